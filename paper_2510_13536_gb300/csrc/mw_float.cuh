// QQF on the device: multi-word arithmetic on four FP32 words.
//
// Sec. II notes multi-word arithmetic built from FP32 words where FP64 is
// missing, and Sec. VI names processors with little FP64 throughput; GB300 is
// one (its FP32 pipe retires 64 times the FP64 pipe's operations).  QQF is
// QQW's sequences (mw_device4.cuh: QTW's Algorithms 7-10 continued one level
// down, VecSum4 as the normalisation) with every FP64 word and operation
// replaced by an FP32 one: about 4 x 24 bits, between FP64 and DW.
//  * An FP64 input (a matrix entry, b_i) enters as its exact three-word split
//    (split3, integer pipe plus two exact FP32 subtractions), and FP64 x QQF
//    is the full QQF product with that split.
//  * Division takes four FP32 quotient digits.
//  * collapse sums the words, lowest first, in FP64.
// Every FP32 operation is an explicit round-to-nearest intrinsic (__fadd_rn,
// __fsub_rn, __fmul_rn, __fmaf_rn, __fdiv_rn): never contracted or
// reassociated; subnormals are kept (the library is built without -ftz).
//
// Vectors of QQF values are stored packed: two 8-byte slots per element, slot
// k (k = 0, 1) of element i holding words 2k and 2k+1 as a float2 at slot
// index k n + i -- the [2][n] layout of an FP64 double-word vector.
#pragma once
#include <cstdint>
#include "mw_device.cuh"

namespace mw {

template <int W> struct MWF { float w[W]; };

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float fneg(float a) { return __uint_as_float(__float_as_uint(a) ^ 0x80000000u); }

// Algorithm 2 (TwoSum) and Algorithm 4 (TwoProdFMA) in FP32.
__device__ __forceinline__ void two_sum_f(float a, float b, float& x, float& y) {
  const float s = fadd(a, b);
  const float z = fsub(s, a);
  y = fadd(fsub(a, fsub(s, z)), fsub(b, z));
  x = s;
}
__device__ __forceinline__ void two_prod_f(float a, float b, float& x, float& y) {
  const float p = fmul(a, b);
  y = ffma(a, b, -p);          // the negation folds into the FMA's operand (no extra instruction)
  x = p;
}

// Values the fast split does not cover: FP32 rounding of the value and of
// the two rests (differences in FP64).  Out of line: rare in practice.
static __device__ __noinline__ float3 split3_slow(double a) {
  const float a0 = __double2float_rn(a);
  const double d = __dsub_rn(a, (double)a0);
  const float a1 = __double2float_rn(d);
  return make_float3(a0, a1, __double2float_rn(__dsub_rn(d, (double)a1)));
}
// Exact split of an FP64 value into three FP32 words by significand bits
// (24 + 23 + 6) for 2^-97 <= |a| < 2^128 (biased exponent 926..1150): a0 the
// value truncated to 24 significant bits, built from the bits; an integer
// m < 2^23 times 2^k (the next 23 bits, the last 6) as the FP32 number with
// exponent k + 23 and fraction m minus the one with fraction 0, an exact
// subtraction.  No FP64 instruction on this path.
__device__ __forceinline__ void split3(double a, float& a0, float& a1, float& a2) {
  const uint64_t u = mwi::bits_of(a);      // opaque: keeps the range test off the FP64 pipe
  const uint32_t hi = (uint32_t)(u >> 32);
  const uint32_t sg = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  if (e >= 926 && e <= 1150) {
    const uint32_t lo = (uint32_t)u;
    const uint32_t top23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);       // fraction bits 51..29
    a0 = __uint_as_float(sg | ((uint32_t)(e - 896) << 23) | top23);
    const uint32_t e1 = (uint32_t)(e - 919) << 23, e2 = (uint32_t)(e - 925) << 23;
    a1 = fsub(__uint_as_float(sg | e1 | ((lo >> 6) & 0x7FFFFFu)), __uint_as_float(sg | e1));
    a2 = fsub(__uint_as_float(sg | e2 | (lo & 63u)), __uint_as_float(sg | e2));
  } else {
    const float3 t = split3_slow(a);
    a0 = t.x;
    a1 = t.y;
    a2 = t.z;
  }
}

// 2^k as FP32 (|k| <= 126) and as FP64 (|k| <= 1022), from the bits.
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }
__device__ __forceinline__ double pow2d(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// FP64 x QQF for a power of two a = +-2^k (2^-126 <= |a| < 2^128): split3(a) is
// (a, +0, +0) and the fourth word is +0, so in the full product every TwoProd
// error, every product with a zero word of a and every TwoSum partner is a
// zero, and the sequence returns (a b0, a b1, a b2, a b3), with +0 for a zero
// lower word of b, whenever each nonzero a b_j is an exact FP32 normal number
// (b_j normal and the scaled exponent inside the normal range).  That case is
// four FP32 multiplications; the path declines (returns false) otherwise.
__device__ __forceinline__ bool pow2_dxmul_f(double a, const float (&b)[4], float (&c)[4]) {
  // The bits through an opaque move: a plain reinterpretation lets the
  // compiler turn the tests below into FP64 comparisons (ncu counted one
  // FP64-pipe instruction per stored entry).
  const uint64_t ua = mwi::bits_of(a);
  if ((ua & 0x7FFFFFFFFFFFFFFFULL) == 0x3FF0000000000000ULL) {
    // a = +-1: no exponent changes, so every product (subnormal words
    // included) is exact for any finite b: a b0 (a zero keeps the product's
    // sign), and a b_j + 0 for the lower words, which is a b_j when b_j is
    // nonzero and +0 when it is zero, as the printed sequence returns them.
    // Four FP32 instructions; the finite test is one more chain of four:
    // x * 0 is NaN exactly when x is infinite or NaN.
    const float af = __uint_as_float(((uint32_t)(ua >> 32) & 0x80000000u) | 0x3F800000u);
    c[0] = fmul(af, b[0]);
    c[1] = ffma(af, b[1], 0.0f);
    c[2] = ffma(af, b[2], 0.0f);
    c[3] = ffma(af, b[3], 0.0f);
    const float t = ffma(b[3], 0.0f, ffma(b[2], 0.0f, ffma(b[1], 0.0f, fmul(b[0], 0.0f))));
    return t == t;
  }
  const int ea = (int)((ua >> 52) & 0x7FFu);
  if ((ua & 0xFFFFFFFFFFFFFULL) != 0 || ea < 897 || ea > 1150) return false;
  const float af = __uint_as_float((uint32_t)(ua >> 32 & 0x80000000u) | ((uint32_t)(ea - 896) << 23));
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t eb = (__float_as_uint(b[j]) >> 23) & 0xFFu;
    const float p = fmul(af, b[j]);
    const uint32_t ep = (__float_as_uint(p) >> 23) & 0xFFu;
    const bool zero = (__float_as_uint(b[j]) << 1) == 0u;
    ok = ok && (zero || (eb != 0u && eb != 255u && ep != 0u && ep != 255u));
    c[j] = (zero && j > 0) ? 0.0f : p;
  }
  return ok;
}

struct QQF {
  static constexpr int ILP = 2;               // rows in flight per thread in the vector kernels (memory bound)
  static constexpr int CHUNK = 3;              // SpMV entries loaded ahead (c2 QQF SpMV 95.4 -> 88.2 us; 2: 89.4, 4: 92.2)
  static constexpr int ILP_SPMV = 1;
  static constexpr int MINB = 4;               // blocks per SM (the plan's G = 4 x SMs)
  static constexpr int W = 4;
  static constexpr bool QUASI = true;
  static constexpr bool NORMALISES = false;   // the normalisation policy does not apply
  static constexpr bool PACKED = true;        // FP32 words, two per 8-byte slot
  using T = MWF<4>;
  static __device__ __forceinline__ T zero() { return T{{0.0f, 0.0f, 0.0f, 0.0f}}; }
  static __device__ __forceinline__ T from(double a) {
    T c;
    split3(a, c.w[0], c.w[1], c.w[2]);
    c.w[3] = 0.0f;
    return c;
  }
  static __device__ __forceinline__ T add(const T& a, const T& b) {
    T c;
    float e1, e2, e3, e4, e5, e6;
    two_sum_f(a.w[0], b.w[0], c.w[0], e1);
    two_sum_f(a.w[1], b.w[1], c.w[1], e2);
    two_sum_f(c.w[1], e1, c.w[1], e3);
    two_sum_f(a.w[2], b.w[2], c.w[2], e4);
    two_sum_f(c.w[2], e2, c.w[2], e5);
    two_sum_f(c.w[2], e3, c.w[2], e6);
    c.w[3] = fadd(fadd(fadd(fadd(a.w[3], b.w[3]), e4), e5), e6);
    return c;
  }
  static __device__ __forceinline__ T mul(const T& a, const T& b) {
    T c;
    float e1, t2, e2, t3, e3, e4, e5;
    two_prod_f(a.w[0], b.w[0], c.w[0], e1);                   // order 1
    two_prod_f(a.w[0], b.w[1], t2, e2);                       // order u
    two_prod_f(a.w[1], b.w[0], t3, e3);
    two_sum_f(t2, t3, c.w[1], e4);
    two_sum_f(c.w[1], e1, c.w[1], e5);
    float t4, e6, t5, e7, t6, e8, e9, e10, e11, e12, e13, e14;
    two_prod_f(a.w[0], b.w[2], t4, e6);                       // order u^2
    two_prod_f(a.w[1], b.w[1], t5, e7);
    two_prod_f(a.w[2], b.w[0], t6, e8);
    two_sum_f(t4, t5, c.w[2], e9);
    two_sum_f(c.w[2], t6, c.w[2], e10);
    two_sum_f(c.w[2], e2, c.w[2], e11);
    two_sum_f(c.w[2], e3, c.w[2], e12);
    two_sum_f(c.w[2], e4, c.w[2], e13);
    two_sum_f(c.w[2], e5, c.w[2], e14);
    const float f1 = ffma(a.w[3], b.w[0], e6);                // order u^3
    const float f2 = ffma(a.w[2], b.w[1], e7);
    const float f3 = ffma(a.w[1], b.w[2], e8);
    const float f4 = ffma(a.w[0], b.w[3], e9);
    const float s3 = fadd(fadd(fadd(f1, f2), f3), f4);
    c.w[3] = fadd(fadd(fadd(fadd(fadd(s3, e10), e11), e12), e13), e14);
    return c;
  }
  // One FP32 word times QQF (the quotient digits of the division).
  static __device__ __forceinline__ T smul(float a, const T& b) {
    T c;
    float e1, e2, e3, e4, e5, e6;
    two_prod_f(a, b.w[0], c.w[0], e1);
    two_prod_f(a, b.w[1], c.w[1], e2);
    two_sum_f(c.w[1], e1, c.w[1], e3);
    two_prod_f(a, b.w[2], c.w[2], e4);
    two_sum_f(c.w[2], e2, c.w[2], e5);
    two_sum_f(c.w[2], e3, c.w[2], e6);
    c.w[3] = fadd(fadd(ffma(a, b.w[3], e4), e5), e6);
    return c;
  }
  static __device__ __forceinline__ T dxmul(double a, const T& b) {
    T c;
    if (pow2_dxmul_f(a, b.w, c.w)) return c;
    return mul(from(a), b);
  }
  static __device__ __forceinline__ T muladd(const T& c, const T& a, const T& b) { return add(c, mul(a, b)); }
  static __device__ __forceinline__ T dxmuladd(const T& c, double a, const T& b) { return add(c, dxmul(a, b)); }
  static __device__ __forceinline__ T neg(const T& a) {
    return T{{fneg(a.w[0]), fneg(a.w[1]), fneg(a.w[2]), fneg(a.w[3])}};
  }
  static __device__ __forceinline__ void renorm(T& a) {    // VecSum4 in FP32
    two_sum_f(a.w[0], a.w[1], a.w[0], a.w[1]);
    two_sum_f(a.w[1], a.w[2], a.w[1], a.w[2]);
    two_sum_f(a.w[2], a.w[3], a.w[2], a.w[3]);
  }
  static __device__ __forceinline__ void normalize(T& a) { renorm(a); }
  static __device__ __forceinline__ T div(const T& a, const T& b) {
    float q[4];
    T r = a;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      q[k] = __fdiv_rn(r.w[0], b.w[0]);
      if (k < 3) {
        r = add(r, neg(smul(q[k], b)));
        renorm(r);
      }
    }
    T c{{q[0], q[1], q[2], q[3]}};
    renorm(c);
    return c;
  }
  static __device__ __forceinline__ double collapse(const T& a) {
    return dadd((double)a.w[0], dadd((double)a.w[1], dadd((double)a.w[2], (double)a.w[3])));
  }
  // Every word times 2^k, each correctly rounded (exact unless it underflows):
  // one FP32 multiplication for |k| <= 126, else the exact FP64 product
  // rounded once to FP32 (|k| <= 1000).
  static __device__ __forceinline__ T scale(const T& a, int k) {
    T c;
    if (k >= -126 && k <= 126) {
      const float f = pow2f(k);
#pragma unroll
      for (int j = 0; j < 4; ++j) c.w[j] = fmul(a.w[j], f);
    } else {
      const double d = pow2d(k);
#pragma unroll
      for (int j = 0; j < 4; ++j) c.w[j] = __double2float_rn(__dmul_rn((double)a.w[j], d));
    }
    return c;
  }
};

// QF: QQF with every addition and product (FP64 x QF included) followed by
// VecSum4 -- the non-quasi counterpart of QQF, as DW relates to QDW in Sec.
// III.  A quasi addition's error is relative to its operands, not to its
// result, so on strongly cancelling SpMV rows QQF keeps about FP64's precision
// in the result; renormalising every result keeps the words ordered and the
// precision relative to the result.  Division, scaling and collapse are
// QQF's (the quotient is renormalised by QQF's division).
struct QF {
  static constexpr int ILP = 2;
  static constexpr int CHUNK = 3;              // as QQF (c2 SpMV 107.0 -> 101.1 us)
  static constexpr int ILP_SPMV = 1;
  static constexpr int MINB = 4;               // blocks per SM (the plan's G = 4 x SMs)
  static constexpr int W = 4;
  static constexpr bool QUASI = false;
  static constexpr bool NORMALISES = false;   // the normalisation policy does not apply
  static constexpr bool PACKED = true;        // FP32 words, two per 8-byte slot
  using T = MWF<4>;
  static __device__ __forceinline__ T fix(T c) {
    QQF::renorm(c);
    return c;
  }
  static __device__ __forceinline__ T zero() { return QQF::zero(); }
  static __device__ __forceinline__ T from(double a) { return QQF::from(a); }
  static __device__ __forceinline__ T add(const T& a, const T& b) { return fix(QQF::add(a, b)); }
  static __device__ __forceinline__ T mul(const T& a, const T& b) { return fix(QQF::mul(a, b)); }
  static __device__ __forceinline__ T dxmul(double a, const T& b) { return fix(QQF::dxmul(a, b)); }
  static __device__ __forceinline__ T muladd(const T& c, const T& a, const T& b) { return add(c, mul(a, b)); }
  static __device__ __forceinline__ T dxmuladd(const T& c, double a, const T& b) { return add(c, dxmul(a, b)); }
  static __device__ __forceinline__ T neg(const T& a) { return QQF::neg(a); }
  static __device__ __forceinline__ void renorm(T& a) { QQF::renorm(a); }
  static __device__ __forceinline__ void normalize(T& a) { QQF::renorm(a); }
  static __device__ __forceinline__ T div(const T& a, const T& b) { return QQF::div(a, b); }
  static __device__ __forceinline__ double collapse(const T& a) { return QQF::collapse(a); }
  static __device__ __forceinline__ T scale(const T& a, int k) { return QQF::scale(a, k); }
};

}  // namespace mw
