// Device word algebra for multi-word arithmetic on sm_103a.
//
// Sources: Sec. III of Mukunoki & Ozaki, "Sparse Iterative Solvers Using
// High-Precision Arithmetic with Quasi Multi-Word Algorithms" -- TwoSum
// (Algorithm 2), QuickTwoSum (Algorithm 3), TwoProdFMA (Algorithm 4), DWadd
// (Algorithm 5), DWmul (Algorithm 6), QTWadd (Algorithm 7), QTWmul
// (Algorithm 8), VecSum3 (Algorithm 9), DxQTWmul (Algorithm 10); QDW is DW
// without the closing QuickTwoSum; FP64 x MW drops the work on zero lower
// words.  Triple-word (TW) follows the Fabiano-Muller-Picot scheme the paper
// cites without printing it (VecSum + renormalisation with branches).
//
// Every FP64 operation is an explicit round-to-nearest intrinsic
// (__dadd_rn, __dsub_rn, __dmul_rn, __fma_rn, __ddiv_rn, __dsqrt_rn): those are
// never contracted or reassociated, so the sequences below are executed
// exactly as written.  Negation and zero/magnitude tests are done on the bit
// pattern (integer pipe), which is exact and keeps them off the FP64 pipe:
// on GB300 the FP64 pipe retires 2 operations per clock per SM while the
// integer pipe retires 64, so the FP64 instruction count is the cost model.
#pragma once
#include <cstdint>
#include "mw_int.cuh"

namespace mw {

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double dneg(double a) {
  return mwi::from_bits(mwi::bits_of(a) ^ 0x8000000000000000ULL);
}
// |a| >= |b| on the bit patterns (valid for all non-NaN values).
__device__ __forceinline__ bool mag_ge(double a, double b) {
  return (mwi::bits_of(a) & mwi::kAbs) >= (mwi::bits_of(b) & mwi::kAbs);
}
// a != 0 (either sign of zero counts as zero; NaN counts as nonzero, as != does).
__device__ __forceinline__ bool nonzero(double a) {
  return (mwi::bits_of(a) << 1) != 0ULL;
}

// Algorithm 2, TwoSum.  Its error term is the exact rounding error of
// fl(a+b), so it is recovered from the bit patterns of a, b and fl(a+b) on the
// integer pipe (mwi::add_error, one FP64 operation instead of six), which
// returns the same number as the printed sequence; the printed sequence runs
// for the operands that path declines.  It is kept out of line so that the
// compiler does not execute part of it speculatively on every call (measured
// as two extra FP64 additions per TwoSum).
static __device__ __noinline__ double two_sum_err_slow(double a, double b, double s) {
  const double z = dsub(s, a);
  return dadd(dsub(a, dsub(s, z)), dsub(b, z));
}
static __device__ __noinline__ double quick_two_sum_err_slow(double a, double b, double s) {
  return dadd(dsub(a, s), b);
}

__device__ __forceinline__ void two_sum(double a, double b, double& x, double& y) {
  const double s = dadd(a, b);
  double e;
  if (!mwi::add_error(a, b, s, e)) e = two_sum_err_slow(a, b, s);
  x = s;
  y = e;
}
// Fully integer-pipe variants (mwi::add_rn computes fl(a+b) itself): no FP64
// instruction at all on the common path.  Used at call sites chosen per
// kernel to balance the FP64 and integer pipes (see QTWt's policy P).
static __device__ __noinline__ double dadd_slow(double a, double b) { return dadd(a, b); }
__device__ __forceinline__ double dadd_int(double a, double b) {
  double x;
  if (!mwi::add_rn(a, b, x)) x = dadd_slow(a, b);
  return x;
}
__device__ __forceinline__ void two_sum_fullint(double a, double b, double& x, double& y) {
  double s, e;
  if (!mwi::add_rn(a, b, s)) s = dadd_slow(a, b);
  if (!mwi::add_error(a, b, s, e)) e = two_sum_err_slow(a, b, s);
  x = s;
  y = e;
}

__device__ __forceinline__ void quick_two_sum_fullint(double a, double b, double& x, double& y) {
  double s, e;
  if (!mwi::add_rn(a, b, s)) s = dadd_slow(a, b);
  if (!(mwi::quick_exact(a, b) && mwi::add_error(a, b, s, e))) e = quick_two_sum_err_slow(a, b, s);
  x = s;
  y = e;
}

// Algorithm 3, QuickTwoSum, as printed (3 FP64 operations).
__device__ __forceinline__ void quick_two_sum(double a, double b, double& x, double& y) {
  double s = dadd(a, b);
  y = dadd(dsub(a, s), b);
  x = s;
}
// Algorithm 4, TwoProdFMA.  two_prod_int recovers the error fma(a, b, -p) on
// the integer pipe instead (mwi::mul_error, same bits), the FMA running only
// for the operands that path declines.  Measured on GB300 it pays off where
// the integer pipe has room: the double-word arithmetics use it (two_prod_w2),
// the triple-word ones, whose kernels already keep the integer pipe busy, use
// the FMA (two_prod).
static __device__ __noinline__ double two_prod_err_slow(double a, double b, double p) { return dfma(a, b, -p); }
__device__ __forceinline__ void two_prod(double a, double b, double& x, double& y) {
  const double p = dmul(a, b);
  y = dfma(a, b, -p);
  x = p;
}
__device__ __forceinline__ void two_prod_w2(double a, double b, double& x, double& y) {
  const double p = dmul(a, b);
  double e;
  if (!mwi::mul_error(a, b, p, e)) e = two_prod_err_slow(a, b, p);
  y = e;
  x = p;
}

template <int W> struct MW { double w[W]; };

// ---------------------------------------------------------------- FP64
struct FP64 {
  // Memory bound: 5 blocks per SM (40 registers a thread, the plan's G = 5 x
  // SMs) with one row per thread and 2 SpMV entries loaded ahead per row
  // measured fastest on GB300 (c2 SpMV 63.6 us; 3 blocks with 2 rows x 2
  // entries: 69.8 us; 4 or 6 blocks, 4 entries or 2 rows: 65.7-76.3 us).
  static constexpr int ILP = 1;                // rows in flight per thread
  static constexpr int CHUNK = 2;              // SpMV entries loaded ahead per row
  static constexpr int ILP_SPMV = 1;
  static constexpr int MINB = 5;               // blocks per SM the register budget must allow
  static constexpr int W = 1;
  static constexpr bool QUASI = false;
  static constexpr bool NORMALISES = false;   // A::normalize is the identity
  using T = MW<1>;
  static __device__ __forceinline__ T zero() { return T{{0.0}}; }
  static __device__ __forceinline__ T from(double a) { return T{{a}}; }
  static __device__ __forceinline__ T add(const T& a, const T& b) { return T{{dadd(a.w[0], b.w[0])}}; }
  static __device__ __forceinline__ T mul(const T& a, const T& b) { return T{{dmul(a.w[0], b.w[0])}}; }
  static __device__ __forceinline__ T dxmul(double a, const T& b) { return T{{dmul(a, b.w[0])}}; }
  static __device__ __forceinline__ T muladd(const T& c, const T& a, const T& b) { return T{{dfma(a.w[0], b.w[0], c.w[0])}}; }
  static __device__ __forceinline__ T dxmuladd(const T& c, double a, const T& b) { return T{{dfma(a, b.w[0], c.w[0])}}; }
  static __device__ __forceinline__ T div(const T& a, const T& b) { return T{{__ddiv_rn(a.w[0], b.w[0])}}; }
  static __device__ __forceinline__ void normalize(T&) {}
  static __device__ __forceinline__ double collapse(const T& a) { return a.w[0]; }
};

// Call-site selectors for the pipe-balancing policies below: with a nonzero
// flag the operation runs entirely on the integer pipe (same bits).
template <int P>
__device__ __forceinline__ void qqs_(double a, double b, double& x, double& y) {
  if constexpr (P != 0) quick_two_sum_fullint(a, b, x, y); else quick_two_sum(a, b, x, y);
}
template <int P>
__device__ __forceinline__ void qts_(double a, double b, double& x, double& y) {
  if constexpr (P != 0) two_sum_fullint(a, b, x, y); else two_sum(a, b, x, y);
}
template <int P>
__device__ __forceinline__ double qadd_(double a, double b) {
  if constexpr (P != 0) return dadd_int(a, b); else return dadd(a, b);
}
// ---------------------------------------------------------------- DW
// Policy P (bit mask, same results): bit 0 DWadd's TwoSum, bit 1 DWadd's two
// plain additions, bit 2 DWadd's closing QuickTwoSum, bit 3 the closing
// QuickTwoSum of DWmul / FP64 x DW, run entirely on the integer pipe.
template <int P = 8>
struct DWt {
  static constexpr int ILP = 1;
  static constexpr int CHUNK = 2;              // SpMV entries loaded ahead (c2 SpMV 289.8 -> 285.4 us)
  static constexpr int ILP_SPMV = 1;
  static constexpr int MINB = 3;
  static constexpr int W = 2;
  static constexpr bool QUASI = false;
  static constexpr bool NORMALISES = false;   // A::normalize is the identity
  using T = MW<2>;
  static __device__ __forceinline__ T zero() { return T{{0.0, 0.0}}; }
  static __device__ __forceinline__ T from(double a) { return T{{a, 0.0}}; }
  // Algorithm 5: e = fl((e + a2) + b2), then QuickTwoSum.
  static __device__ __forceinline__ T add(const T& a, const T& b) {
    double s, e;
    qts_<P & 1>(a.w[0], b.w[0], s, e);
    e = qadd_<P & 2>(qadd_<P & 2>(e, a.w[1]), b.w[1]);
    T c;
    qqs_<P & 4>(s, e, c.w[0], c.w[1]);
    return c;
  }
  // Algorithm 6: fma with a1*b2 first, then a2*b1.
  static __device__ __forceinline__ T mul(const T& a, const T& b) {
    double p, e;
    two_prod_w2(a.w[0], b.w[0], p, e);
    e = dfma(a.w[0], b.w[1], e);
    e = dfma(a.w[1], b.w[0], e);
    T c;
    qqs_<P & 8>(p, e, c.w[0], c.w[1]);
    return c;
  }
  // For a = +-2^k, TwoProdFMA(a, b1) = (a*b1, +0) and fma(a, b2, +0) = a*b2
  // (+0 if zero) exactly, so both are formed on the integer pipe; the closing
  // QuickTwoSum runs as printed.
  static __device__ __forceinline__ T dxmul(double a, const T& b) {
    double p, e;
    double pe[2];
    if (mwi::pow2_product<2>(a, b.w, pe)) {
      p = pe[0];
      e = pe[1];
    } else {
      two_prod_w2(a, b.w[0], p, e);
      e = dfma(a, b.w[1], e);
    }
    T c;
    qqs_<P & 8>(p, e, c.w[0], c.w[1]);
    return c;
  }
  static __device__ __forceinline__ T muladd(const T& c, const T& a, const T& b) { return add(c, mul(a, b)); }
  static __device__ __forceinline__ T dxmuladd(const T& c, double a, const T& b) { return add(c, dxmul(a, b)); }
  static __device__ __forceinline__ T neg(const T& a) { return T{{dneg(a.w[0]), dneg(a.w[1])}}; }
  static __device__ __forceinline__ T div(const T& a, const T& b) {
    double q1 = __ddiv_rn(a.w[0], b.w[0]);
    T r = add(a, neg(dxmul(q1, b)));
    double q2 = __ddiv_rn(r.w[0], b.w[0]);
    T c;
    quick_two_sum(q1, q2, c.w[0], c.w[1]);
    return c;
  }
  static __device__ __forceinline__ void normalize(T&) {}
  static __device__ __forceinline__ double collapse(const T& a) { return dadd(a.w[0], a.w[1]); }
};
// Every DW kernel runs the closing QuickTwoSum of its products on the integer
// pipe (policy bit 3; DW's TwoProd error is there already).  Measured on c2:
// SpMV 311.5 -> 289.5 us, update 165.9 -> 141.4 us, p update 54.4 -> 47.4 us;
// bits 0-2 (the addition's operations), alone or with bit 3, make the SpMV
// slower (342-426 us).
using DW = DWt<>;
using DW_S = DWt<8>;

// ---------------------------------------------------------------- QDW
// Policy P: bit 0 QDWadd's TwoSum, bit 1 its two plain additions, bit 2 the
// normalising QuickTwoSum, run entirely on the integer pipe (same bits).
template <bool NORM, int P = 4>
struct QDWt {
  static constexpr int ILP = 1;
  static constexpr int CHUNK = 2;              // SpMV entries loaded ahead (c2 SpMV 156.0 -> 150.8 us)
  static constexpr int ILP_SPMV = 1;
  static constexpr int MINB = 3;
  static constexpr int W = 2;
  static constexpr bool QUASI = true;
  static constexpr bool NORMALISES = NORM;   // false for the NN variants
  using T = MW<2>;
  static __device__ __forceinline__ T zero() { return T{{0.0, 0.0}}; }
  static __device__ __forceinline__ T from(double a) { return T{{a, 0.0}}; }
  static __device__ __forceinline__ T add(const T& a, const T& b) {
    T c;
    qts_<P & 1>(a.w[0], b.w[0], c.w[0], c.w[1]);
    c.w[1] = qadd_<P & 2>(qadd_<P & 2>(c.w[1], a.w[1]), b.w[1]);
    return c;
  }
  static __device__ __forceinline__ T mul(const T& a, const T& b) {
    T c;
    two_prod_w2(a.w[0], b.w[0], c.w[0], c.w[1]);
    c.w[1] = dfma(a.w[0], b.w[1], c.w[1]);
    c.w[1] = dfma(a.w[1], b.w[0], c.w[1]);
    return c;
  }
  static __device__ __forceinline__ T dxmul(double a, const T& b) {
    T c;
    if (mwi::pow2_product<2>(a, b.w, c.w)) return c;
    two_prod_w2(a, b.w[0], c.w[0], c.w[1]);
    c.w[1] = dfma(a, b.w[1], c.w[1]);
    return c;
  }
  static __device__ __forceinline__ T muladd(const T& c, const T& a, const T& b) { return add(c, mul(a, b)); }
  static __device__ __forceinline__ T dxmuladd(const T& c, double a, const T& b) { return add(c, dxmul(a, b)); }
  static __device__ __forceinline__ T neg(const T& a) { return T{{dneg(a.w[0]), dneg(a.w[1])}}; }
  // QDW normalisation: QuickTwoSum(c1, c2).
  static __device__ __forceinline__ void renorm(T& a) { qqs_<P & 4>(a.w[0], a.w[1], a.w[0], a.w[1]); }
  static __device__ __forceinline__ T div(const T& a, const T& b) {
    double q1 = __ddiv_rn(a.w[0], b.w[0]);
    T r = add(a, neg(dxmul(q1, b)));
    renorm(r);
    double q2 = __ddiv_rn(r.w[0], b.w[0]);
    T c;
    quick_two_sum(q1, q2, c.w[0], c.w[1]);
    return c;
  }
  static __device__ __forceinline__ void normalize(T& a) { if (NORM) renorm(a); }
  static __device__ __forceinline__ double collapse(const T& a) { return dadd(a.w[0], a.w[1]); }
};
using QDW = QDWt<true>;
using QDW_NN = QDWt<false>;
// The vector kernels normalise r with QuickTwoSum on the integer pipe (policy
// bit 2; c2 update 102.5 -> 95.9 us); bit 1 (the addition's plain additions)
// is slower (140.3 us).  The SpMV instantiations keep every FP64 operation on
// the FP64 pipe (bits 0 / 1 there: 206 / 285 us against 155 us).
using QDW_S = QDWt<true, 0>;
using QDW_NN_S = QDWt<false, 0>;

// ---------------------------------------------------------------- QTW
// Policy P (bit mask, same results for every value): which TwoSums and plain
// additions run entirely on the integer pipe.  bit 0: QTWadd's TwoSums;
// bit 1: QTWadd's c3 additions; bit 2: DxQTWmul's TwoSum; bit 3: DxQTWmul's
// c3 addition; bit 4: QTWmul's TwoSums; bit 5: QTWmul's c3 additions.
// Measured on GB300 (128^3 Poisson): a full integer addition costs ~50 integer
// instructions, about 25 clocks of the 64-lane integer pipe per warp against 16
// of the FP64 pipe for a DADD, so only the SpMV's FP64 x QTW c3 addition gains
// (2%); every wider choice, and any choice in the vector kernels, is slower.
template <bool NORM, int P = 0>
struct QTWt {
  static constexpr int ILP = 1;
  static constexpr int CHUNK = 1;              // 2 entries loaded ahead: c2 SpMV 325.2 -> 342.8 us
  static constexpr int ILP_SPMV = 1;
  static constexpr int MINB = 3;
  static constexpr int W = 3;
  static constexpr bool QUASI = true;
  static constexpr bool NORMALISES = NORM;   // false for the NN variants
  using T = MW<3>;
  static __device__ __forceinline__ T zero() { return T{{0.0, 0.0, 0.0}}; }
  static __device__ __forceinline__ T from(double a) { return T{{a, 0.0, 0.0}}; }
  // Algorithm 7.
  static __device__ __forceinline__ T add(const T& a, const T& b) {
    T c;
    double e1, e2, e3;
    qts_<P & 1>(a.w[0], b.w[0], c.w[0], e1);
    qts_<P & 1>(a.w[1], b.w[1], c.w[1], e2);
    qts_<P & 1>(c.w[1], e1, c.w[1], e3);
    c.w[2] = qadd_<P & 2>(qadd_<P & 2>(qadd_<P & 2>(a.w[2], b.w[2]), e2), e3);
    return c;
  }
  // Algorithm 8.
  static __device__ __forceinline__ T mul(const T& a, const T& b) {
    T c;
    double e1, t2, e2, t3, e3, e4, e5;
    two_prod(a.w[0], b.w[0], c.w[0], e1);
    two_prod(a.w[0], b.w[1], t2, e2);
    two_prod(a.w[1], b.w[0], t3, e3);
    qts_<P & 16>(t2, t3, c.w[1], e4);
    qts_<P & 16>(c.w[1], e1, c.w[1], e5);
    double f1 = dfma(a.w[2], b.w[0], e2);
    double f2 = dfma(a.w[1], b.w[1], e3);
    double f3 = dfma(a.w[0], b.w[2], e4);
    c.w[2] = qadd_<P & 32>(qadd_<P & 32>(qadd_<P & 32>(f1, f2), f3), e5);
    return c;
  }
  // Algorithm 10.  A power-of-two a (the +-1 entries of a Laplacian, for
  // instance) takes the exact-scaling path on the integer pipe (same bits).
  static __device__ __forceinline__ T dxmul(double a, const T& b) {
    T c;
    if (mwi::pow2_product<3>(a, b.w, c.w)) return c;
    double e1, e2, e5;
    two_prod(a, b.w[0], c.w[0], e1);
    two_prod(a, b.w[1], c.w[1], e2);
    qts_<P & 4>(c.w[1], e1, c.w[1], e5);
    c.w[2] = qadd_<P & 8>(dfma(a, b.w[2], e2), e5);
    return c;
  }
  static __device__ __forceinline__ T muladd(const T& c, const T& a, const T& b) { return add(c, mul(a, b)); }
  static __device__ __forceinline__ T dxmuladd(const T& c, double a, const T& b) { return add(c, dxmul(a, b)); }
  static __device__ __forceinline__ T neg(const T& a) { return T{{dneg(a.w[0]), dneg(a.w[1]), dneg(a.w[2])}}; }
  // Algorithm 9, VecSum3 as printed.
  static __device__ __forceinline__ void renorm(T& a) {
    qts_<P & 1>(a.w[0], a.w[1], a.w[0], a.w[1]);
    qts_<P & 1>(a.w[1], a.w[2], a.w[1], a.w[2]);
  }
  static __device__ __forceinline__ T div(const T& a, const T& b) {
    double q1 = __ddiv_rn(a.w[0], b.w[0]);
    T r = add(a, neg(dxmul(q1, b)));
    renorm(r);
    double q2 = __ddiv_rn(r.w[0], b.w[0]);
    r = add(r, neg(dxmul(q2, b)));
    renorm(r);
    double q3 = __ddiv_rn(r.w[0], b.w[0]);
    T c{{q1, q2, q3}};
    renorm(c);
    return c;
  }
  static __device__ __forceinline__ void normalize(T& a) { if (NORM) renorm(a); }
  static __device__ __forceinline__ double collapse(const T& a) { return dadd(a.w[0], dadd(a.w[1], a.w[2])); }
};
using QTW = QTWt<true>;
using QTW_NN = QTWt<false>;
// SpMV-kernel instantiations: the FP64 x QTW c3 addition on the integer pipe.
using QTW_S = QTWt<true, 8>;
using QTW_NN_S = QTWt<false, 8>;

// ---------------------------------------------------------------- TW
struct TW {
  static constexpr int ILP = 1;
  static constexpr int CHUNK = 1;
  static constexpr int ILP_SPMV = 1;
  static constexpr int MINB = 3;
  static constexpr int W = 3;
  static constexpr bool QUASI = false;
  static constexpr bool NORMALISES = false;   // A::normalize is the identity
  using T = MW<3>;
  static __device__ __forceinline__ T zero() { return T{{0.0, 0.0, 0.0}}; }
  static __device__ __forceinline__ T from(double a) { return T{{a, 0.0, 0.0}}; }

  // Error-free VecSum, bottom-up, in place (N compile-time so the array stays
  // in registers).
  template <int N>
  static __device__ __forceinline__ void vecsum(double (&x)[N]) {
    double s = x[N - 1];
#pragma unroll
    for (int i = N - 2; i >= 0; --i) {
      double hi, lo;
      two_sum(x[i], s, hi, lo);
      x[i + 1] = lo;
      s = hi;
    }
    x[0] = s;
  }
  // Renormalisation to three words with branches on zero errors.  Written
  // without dynamic register indexing: the open word index j selects one of
  // three registers.
  template <int N>
  static __device__ __forceinline__ T renorm3(const double (&e)[N]) {
    double r0 = 0.0, r1 = 0.0, r2 = 0.0;
    int j = 0;
    double eps = e[0];
    bool stop = false;
#pragma unroll
    for (int i = 0; i + 1 < N; ++i) {
      if (!stop) {
        double hi, lo;
        quick_two_sum(eps, e[i + 1], hi, lo);
        if (j == 0) r0 = hi; else if (j == 1) r1 = hi; else r2 = hi;
        if (nonzero(lo)) {
          if (j >= 2) stop = true;
          else { ++j; eps = lo; }
        } else {
          eps = hi;
        }
      }
    }
    if (!stop) { if (j == 0) r0 = eps; else if (j == 1) r1 = eps; else r2 = eps; }
    return T{{r0, r1, r2}};
  }
  static __device__ __forceinline__ T add(const T& a, const T& b) {
    double z[6];
    int i = 0, k = 0;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      // Merge by decreasing magnitude, ties from a first.
      double ai = (i == 0) ? a.w[0] : (i == 1) ? a.w[1] : a.w[2];
      double bk = (k == 0) ? b.w[0] : (k == 1) ? b.w[1] : b.w[2];
      bool take_a = (k >= 3) || (i < 3 && mag_ge(ai, bk));
      z[m] = take_a ? ai : bk;
      if (take_a) ++i; else ++k;
    }
    vecsum<6>(z);
    return renorm3<6>(z);
  }
  static __device__ __forceinline__ T mul(const T& a, const T& b) {
    double p00, e00, p01, e01, p10, e10;
    two_prod(a.w[0], b.w[0], p00, e00);
    two_prod(a.w[0], b.w[1], p01, e01);
    two_prod(a.w[1], b.w[0], p10, e10);
    double t, s3, s1, s2;
    two_sum(p01, p10, t, s3);
    two_sum(e00, t, s1, s2);
    double c = dadd(s2, s3);
    c = dadd(c, e01);
    c = dadd(c, e10);
    c = dfma(a.w[2], b.w[0], c);
    c = dfma(a.w[1], b.w[1], c);
    c = dfma(a.w[0], b.w[2], c);
    double z[3] = {p00, s1, c};
    vecsum<3>(z);
    return renorm3<3>(z);
  }
  static __device__ __forceinline__ T dxmul(double a, const T& b) {
    double p00, e00, p01, e01;
    two_prod(a, b.w[0], p00, e00);
    two_prod(a, b.w[1], p01, e01);
    double s1, s2;
    two_sum(e00, p01, s1, s2);
    double c = dadd(s2, e01);
    c = dfma(a, b.w[2], c);
    double z[3] = {p00, s1, c};
    vecsum<3>(z);
    return renorm3<3>(z);
  }
  static __device__ __forceinline__ T muladd(const T& c, const T& a, const T& b) { return add(c, mul(a, b)); }
  static __device__ __forceinline__ T dxmuladd(const T& c, double a, const T& b) { return add(c, dxmul(a, b)); }
  static __device__ __forceinline__ T neg(const T& a) { return T{{dneg(a.w[0]), dneg(a.w[1]), dneg(a.w[2])}}; }
  static __device__ __forceinline__ T div(const T& a, const T& b) {
    double q1 = __ddiv_rn(a.w[0], b.w[0]);
    T r = add(a, neg(dxmul(q1, b)));
    double q2 = __ddiv_rn(r.w[0], b.w[0]);
    r = add(r, neg(dxmul(q2, b)));
    double q3 = __ddiv_rn(r.w[0], b.w[0]);
    double z[3] = {q1, q2, q3};
    vecsum<3>(z);
    return renorm3<3>(z);
  }
  static __device__ __forceinline__ void normalize(T&) {}
  static __device__ __forceinline__ double collapse(const T& a) { return dadd(a.w[0], dadd(a.w[1], a.w[2])); }
};

template <class A>
__device__ __forceinline__ typename A::T neg(const typename A::T& a) {
  typename A::T c;
#pragma unroll
  for (int k = 0; k < A::W; ++k) c.w[k] = dneg(a.w[k]);
  return c;
}

}  // namespace mw
