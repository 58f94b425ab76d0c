// Four-word arithmetics on the device: QQW (quasi quadruple-word), its
// unnormalised variant and QW (quadruple-word).
//
// The paper lists QW (Hida et al.) and QQW (Ozaki and Imamura) among the
// multi-word arithmetics (Sec. I) without printing algorithms.  Definitions
// (the same as the CPU oracle's, operation for operation):
//  * QQW continues QTW's Algorithms 7-10 one level down: at each level the
//    level's own terms are combined by TwoSum / TwoProd and every error of the
//    level above is folded in by TwoSum; the lowest level (order u^3) is
//    summed plainly, left to right, its products taken by FMA together with
//    the first errors.  Normalisation: VecSum4 (Algorithm 9 continued).
//  * QW is every QQW operation followed by the error-free VecSum and the TW
//    renormalisation with branches, continued to four non-overlapping words.
// The error-free transformations are the ones of mw_device.cuh (integer-pipe
// error terms by default; the bits equal the printed sequences).
#pragma once
#include "mw_device.cuh"

namespace mw {


template <bool NORM>
struct QQWt {
  static constexpr int ILP = 1;
  static constexpr int CHUNK = 1;
  static constexpr int ILP_SPMV = 1;
  static constexpr int MINB = 3;
  static constexpr int W = 4;
  static constexpr bool QUASI = true;
  static constexpr bool NORMALISES = NORM;   // false for the NN variant
  using T = MW<4>;
  static __device__ __forceinline__ T zero() { return T{{0.0, 0.0, 0.0, 0.0}}; }
  static __device__ __forceinline__ T from(double a) { return T{{a, 0.0, 0.0, 0.0}}; }
  static __device__ __forceinline__ T add(const T& a, const T& b) {
    T c;
    double e1, e2, e3, e4, e5, e6;
    two_sum(a.w[0], b.w[0], c.w[0], e1);
    two_sum(a.w[1], b.w[1], c.w[1], e2);
    two_sum(c.w[1], e1, c.w[1], e3);
    two_sum(a.w[2], b.w[2], c.w[2], e4);
    two_sum(c.w[2], e2, c.w[2], e5);
    two_sum(c.w[2], e3, c.w[2], e6);
    c.w[3] = dadd(dadd(dadd(dadd(a.w[3], b.w[3]), e4), e5), e6);
    return c;
  }
  static __device__ __forceinline__ T mul(const T& a, const T& b) {
    T c;
    double e1, t2, e2, t3, e3, e4, e5;
    two_prod(a.w[0], b.w[0], c.w[0], e1);                     // order 1
    two_prod(a.w[0], b.w[1], t2, e2);                         // order u
    two_prod(a.w[1], b.w[0], t3, e3);
    two_sum(t2, t3, c.w[1], e4);
    two_sum(c.w[1], e1, c.w[1], e5);
    double t4, e6, t5, e7, t6, e8, e9, e10, e11, e12, e13, e14;
    two_prod(a.w[0], b.w[2], t4, e6);                         // order u^2
    two_prod(a.w[1], b.w[1], t5, e7);
    two_prod(a.w[2], b.w[0], t6, e8);
    two_sum(t4, t5, c.w[2], e9);
    two_sum(c.w[2], t6, c.w[2], e10);
    two_sum(c.w[2], e2, c.w[2], e11);
    two_sum(c.w[2], e3, c.w[2], e12);
    two_sum(c.w[2], e4, c.w[2], e13);
    two_sum(c.w[2], e5, c.w[2], e14);
    const double f1 = dfma(a.w[3], b.w[0], e6);               // order u^3
    const double f2 = dfma(a.w[2], b.w[1], e7);
    const double f3 = dfma(a.w[1], b.w[2], e8);
    const double f4 = dfma(a.w[0], b.w[3], e9);
    const double s3 = dadd(dadd(dadd(f1, f2), f3), f4);
    c.w[3] = dadd(dadd(dadd(dadd(dadd(s3, e10), e11), e12), e13), e14);
    return c;
  }
  // FP64 x QQW (Algorithm 10 continued).  A power-of-two a scales every word
  // exactly on the integer pipe (the same bits as the sequence below).
  static __device__ __forceinline__ T dxmul(double a, const T& b) {
    T c;
    if (mwi::pow2_product<4>(a, b.w, c.w))
      return c;
    double e1, e2, e3, e4, e5, e6;
    two_prod(a, b.w[0], c.w[0], e1);
    two_prod(a, b.w[1], c.w[1], e2);
    two_sum(c.w[1], e1, c.w[1], e3);
    two_prod(a, b.w[2], c.w[2], e4);
    two_sum(c.w[2], e2, c.w[2], e5);
    two_sum(c.w[2], e3, c.w[2], e6);
    c.w[3] = dadd(dadd(dfma(a, b.w[3], e4), e5), e6);
    return c;
  }
  static __device__ __forceinline__ T muladd(const T& c, const T& a, const T& b) { return add(c, mul(a, b)); }
  static __device__ __forceinline__ T dxmuladd(const T& c, double a, const T& b) { return add(c, dxmul(a, b)); }
  static __device__ __forceinline__ T neg(const T& a) {
    return T{{dneg(a.w[0]), dneg(a.w[1]), dneg(a.w[2]), dneg(a.w[3])}};
  }
  // VecSum4: TwoSum(c1,c2), TwoSum(c2,c3), TwoSum(c3,c4).
  static __device__ __forceinline__ void renorm(T& a) {
    two_sum(a.w[0], a.w[1], a.w[0], a.w[1]);
    two_sum(a.w[1], a.w[2], a.w[1], a.w[2]);
    two_sum(a.w[2], a.w[3], a.w[2], a.w[3]);
  }
  // Long division with four quotient digits; the remainder is normalised
  // before its leading word is read.
  static __device__ __forceinline__ T div(const T& a, const T& b) {
    double q[4];
    T r = a;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      q[k] = __ddiv_rn(r.w[0], b.w[0]);
      if (k < 3) {
        r = add(r, neg(dxmul(q[k], b)));
        renorm(r);
      }
    }
    T c{{q[0], q[1], q[2], q[3]}};
    renorm(c);
    return c;
  }
  static __device__ __forceinline__ void normalize(T& a) { if (NORM) renorm(a); }
  static __device__ __forceinline__ double collapse(const T& a) {
    return dadd(a.w[0], dadd(a.w[1], dadd(a.w[2], a.w[3])));
  }
};
using QQW = QQWt<true>;
using QQW_NN = QQWt<false>;

struct QW {
  static constexpr int ILP = 1;
  static constexpr int CHUNK = 1;
  static constexpr int ILP_SPMV = 1;
  static constexpr int MINB = 3;
  static constexpr int W = 4;
  static constexpr bool QUASI = false;
  static constexpr bool NORMALISES = false;   // results are always normalised
  using T = MW<4>;
  using Q = QQWt<false>;
  static __device__ __forceinline__ T zero() { return Q::zero(); }
  static __device__ __forceinline__ T from(double a) { return Q::from(a); }
  // Error-free VecSum of the four words, then the running-QuickTwoSum
  // renormalisation (a nonzero error closes an output word), written without
  // dynamic register indexing.
  static __device__ __forceinline__ T fix(const T& c) {
    double z[4] = {c.w[0], c.w[1], c.w[2], c.w[3]};
    TW::vecsum<4>(z);
    double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
    int j = 0;
    double eps = z[0];
    bool stop = false;
#pragma unroll
    for (int i = 0; i + 1 < 4; ++i) {
      if (!stop) {
        double hi, lo;
        quick_two_sum(eps, z[i + 1], hi, lo);
        if (j == 0) r0 = hi; else if (j == 1) r1 = hi; else if (j == 2) r2 = hi; else r3 = hi;
        if (nonzero(lo)) {
          if (j >= 3) stop = true;
          else { ++j; eps = lo; }
        } else {
          eps = hi;
        }
      }
    }
    if (!stop) { if (j == 0) r0 = eps; else if (j == 1) r1 = eps; else if (j == 2) r2 = eps; else r3 = eps; }
    return T{{r0, r1, r2, r3}};
  }
  static __device__ __forceinline__ T add(const T& a, const T& b) { return fix(Q::add(a, b)); }
  static __device__ __forceinline__ T mul(const T& a, const T& b) { return fix(Q::mul(a, b)); }
  static __device__ __forceinline__ T dxmul(double a, const T& b) { return fix(Q::dxmul(a, b)); }
  static __device__ __forceinline__ T muladd(const T& c, const T& a, const T& b) { return add(c, mul(a, b)); }
  static __device__ __forceinline__ T dxmuladd(const T& c, double a, const T& b) { return add(c, dxmul(a, b)); }
  static __device__ __forceinline__ T neg(const T& a) { return Q::neg(a); }
  static __device__ __forceinline__ T div(const T& a, const T& b) {
    double q[4];
    T r = a;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      q[k] = __ddiv_rn(r.w[0], b.w[0]);
      if (k < 3) r = add(r, neg(dxmul(q[k], b)));
    }
    return fix(T{{q[0], q[1], q[2], q[3]}});
  }
  static __device__ __forceinline__ void normalize(T&) {}
  static __device__ __forceinline__ double collapse(const T& a) { return Q::collapse(a); }
};

}  // namespace mw
