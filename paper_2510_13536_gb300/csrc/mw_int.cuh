// Exact rounding error of an FP64 addition, computed on the integer pipe.
//
// TwoSum (Algorithm 2 of the paper) and QuickTwoSum (Algorithm 3, when its
// precondition holds) return x = fl(a+b) and the exact error y = (a+b) - x,
// which is an FP64 number whenever no overflow or underflow gets in the way.
// On GB300 the FP64 pipe retires 2 operations per clock per SM and the
// integer pipe 64, so recovering y from the bit patterns of a, b and x with
// ~70 integer instructions is cheaper than the five FP64 operations of the
// printed sequence that follow fl(a+b).  The result is the same number, so the
// bits are identical to the printed sequence (which returns +0, never -0,
// when the error is zero).
//
// Derivation (IEEE binary64, round to nearest even): order the operands by
// magnitude, |h| >= |l|, with biased exponent fields eh >= el.  Every one of
// h, l and x = fl(h+l) is an integer multiple of u = 2^(el-1075) (x is either
// exact or at least 2^52 u in magnitude).  With significands mh, ml, mx
// (hidden bit included) and d = eh - el, dx = ex - el:
//   |h+l| / u = mh*2^d (+|-) ml,    |x| / u = mx*2^dx,
// and |y| <= ulp(x)/2 <= 2^55 u, so Y = (|h+l| - |x|) / u is recovered exactly
// by 64-bit wrap-around arithmetic even though the two terms do not fit.
// Then y = sign(h) * Y * u, packed by locating Y's leading bit.  Special
// cases: l = 0 gives y = +0; d > 55 gives x = h and y = l; x = 0 or dx < 0
// (the sum is exact) gives y = +0.  The integer path declines (returns false)
// when h is not finite or may overflow (eh >= 2046) or when l is tiny
// (el < 110, so that y could be subnormal); callers then run the printed
// FP64 sequence.
//
// Host-compilable (plain C++) so that it can also be checked on the CPU.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define MWI_HD __host__ __device__ __forceinline__
#else
#define MWI_HD inline
#endif

namespace mwi {

// On the device the reinterpretation goes through an opaque move, so that the
// compiler cannot turn the integer tests below back into FP64 comparisons
// (a zero test on the magnitude bits is equivalent to "v == 0.0", and the
// FP64 pipe is the scarce resource).
MWI_HD uint64_t bits_of(double v) {
#if defined(__CUDA_ARCH__)
  uint64_t u;
  asm("mov.b64 %0, %1;" : "=l"(u) : "d"(v));
  return u;
#else
  uint64_t u;
  memcpy(&u, &v, sizeof u);
  return u;
#endif
}

MWI_HD double from_bits(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double v;
  memcpy(&v, &u, sizeof v);
  return v;
#endif
}

// Index of the most significant set bit of v != 0.
MWI_HD int msb64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return 63 - __clzll((long long)v);
#else
  return 63 - __builtin_clzll(v);
#endif
}

constexpr uint64_t kAbs = 0x7fffffffffffffffULL;
constexpr uint64_t kFrac = 0x000fffffffffffffULL;
constexpr uint64_t kHidden = 0x0010000000000000ULL;

// y = (a + b) - x exactly, given x = fl(a + b).  Returns false when the
// integer path does not apply (see above); y is then left untouched.
MWI_HD bool add_error(double a, double b, double x, double& y) {
  const uint64_t ua = bits_of(a), ub = bits_of(b), ux = bits_of(x);
  const bool swap = (ua & kAbs) < (ub & kAbs);
  const uint64_t h = swap ? ub : ua;
  const uint64_t l = swap ? ua : ub;
  const int eh = (int)((h >> 52) & 0x7ff);
  const int el = (int)((l >> 52) & 0x7ff);
  if (eh >= 2046) return false;                 // inf/NaN or possible overflow
  if ((l & kAbs) == 0) { y = 0.0; return true; }  // l = +-0: the sum is exact
  if (el < 110) return false;                   // y might be subnormal
  const int d = eh - el;
  if (d > 55) { y = from_bits(l); return true; }  // l is below half an ulp of h: x = h
  if ((ux & kAbs) == 0) { y = 0.0; return true; }  // exact cancellation
  const int ex = (int)((ux >> 52) & 0x7ff);
  const int dx = ex - el;
  if (dx < 0) { y = 0.0; return true; }         // |x| < 2^52 u: the sum is exact
  const uint64_t mh = (h & kFrac) | kHidden;
  const uint64_t ml = (l & kFrac) | kHidden;
  const uint64_t mx = (ux & kFrac) | kHidden;
  const uint64_t H = mh << d;                   // d <= 55, wraps modulo 2^64
  const uint64_t T = (((ua ^ ub) >> 63) == 0) ? H + ml : H - ml;
  const uint64_t Y = T - (mx << dx);            // dx <= 56
  if (Y == 0) { y = 0.0; return true; }
  const bool neg = (int64_t)Y < 0;
  const uint64_t M = neg ? (uint64_t)0 - Y : Y;   // |Y| < 2^56, at most 53 significant bits
  const int L = msb64(M);
  const uint64_t mant = (L <= 52) ? (M << (52 - L)) : (M >> (L - 52));
  const uint64_t sign = ((h >> 63) ^ (neg ? 1u : 0u)) & 1u;
  y = from_bits((sign << 63) | ((uint64_t)(L + el - 52) << 52) | (mant & kFrac));
  return true;
}

// x = fl(a + b) (IEEE binary64, round to nearest, ties to even) on the integer
// pipe.  Operands ordered by magnitude, |h| >= |l|; significands extended by
// three guard bits; l aligned to h with the bits shifted out folded into a
// sticky bit; added or subtracted; renormalised; rounded to nearest even.
// Zeros follow IEEE (x = -0 only for (-0) + (-0)); l below a quarter ulp of h
// gives x = h.  Declines (returns false) for non-finite, overflow-prone or
// subnormal operands and for a subnormal result; callers then use the FP64 add.
MWI_HD bool add_rn(double a, double b, double& x) {
  const uint64_t ua = bits_of(a), ub = bits_of(b);
  const bool swap = (ua & kAbs) < (ub & kAbs);
  const uint64_t h = swap ? ub : ua;
  const uint64_t l = swap ? ua : ub;
  const int eh = (int)((h >> 52) & 0x7ff);
  const int el = (int)((l >> 52) & 0x7ff);
  if (eh >= 2046) return false;
  if ((l & kAbs) == 0) {                        // l = +-0
    x = ((h & kAbs) == 0) ? from_bits(h & l & ~kAbs) : from_bits(h);
    return true;
  }
  if (el == 0) return false;                    // subnormal operand
  const int d = eh - el;
  if (d > 55) { x = from_bits(h); return true; }
  const uint64_t mh = ((h & kFrac) | kHidden) << 3;          // 56 bits
  const uint64_t ml = ((l & kFrac) | kHidden) << 3;
  const uint64_t lost = (d == 0) ? 0 : (ml & ((1ULL << d) - 1));
  const uint64_t L = (ml >> d) | (lost != 0 ? 1u : 0u);       // sticky in bit 0
  uint64_t S;
  int e = eh;
  if (((ua ^ ub) >> 63) == 0) {
    S = mh + L;                                 // < 2^57
    if (S >> 56) { S = (S >> 1) | (S & 1u); ++e; }
  } else {
    S = mh - L;
    if (S == 0) { x = 0.0; return true; }       // exact cancellation: +0
    const int sh = 55 - msb64(S);               // renormalise (exact when sh > 1)
    S <<= sh;
    e -= sh;
  }
  const uint64_t g = (S >> 2) & 1u, rest = S & 3u, lsb = (S >> 3) & 1u;
  uint64_t m = (S >> 3) + ((g && (rest || lsb)) ? 1u : 0u);
  if (m >> 53) { m >>= 1; ++e; }
  if (e < 1 || e >= 2047) return false;         // subnormal or overflowing result
  x = from_bits((h & ~kAbs) | ((uint64_t)e << 52) | (m & kFrac));
  return true;
}

// Error of an FP64 product, e = a*b - p exactly, given p = fl(a*b): the value
// TwoProdFMA (Algorithm 4) computes as fma(a, b, -p).  With significands ma, mb
// (53 bits, hidden bit included), the exact product is M = ma*mb units of
// u = 2^(ea+eb-2150) and p = mp*2^s units with s in {52, 53}.  |M - mp*2^s| <=
// 2^52, so the low 64 bits of the two terms (one 64-bit multiplication, no
// high half) give it exactly under wrap-around arithmetic.  Declines (returns
// false) for zero, subnormal, non-finite or overflow-prone operands and when
// the error would be subnormal; callers then use the FMA.
MWI_HD bool mul_error(double a, double b, double p, double& e) {
  const uint64_t ua = bits_of(a), ub = bits_of(b), up = bits_of(p);
  const int ea = (int)((ua >> 52) & 0x7ff);
  const int eb = (int)((ub >> 52) & 0x7ff);
  const int ep = (int)((up >> 52) & 0x7ff);
  if (ea == 2047 || eb == 2047) return false;   // inf or NaN operand
  if ((ua & kAbs) == 0 || (ub & kAbs) == 0) { e = 0.0; return true; }  // exact zero product: fma gives +0
  if (ea == 0 || eb == 0 || ep == 0 || ep >= 2046) return false;
  const int k = ea + eb - 2150;                 // exponent of one unit of M
  const int sh = ep - ea - eb + 1075;           // p = mp * 2^sh units
  if (sh < 0 || sh > 63) return false;
  const uint64_t ma = (ua & kFrac) | kHidden;
  const uint64_t mb = (ub & kFrac) | kHidden;
  const uint64_t mp = (up & kFrac) | kHidden;
  const uint64_t D = ma * mb - (mp << sh);      // low 64 bits; |true value| <= 2^52
  if (D == 0) { e = 0.0; return true; }
  const bool neg = (int64_t)D < 0;
  const uint64_t M = neg ? (uint64_t)0 - D : D;
  const int L = msb64(M);
  const int E = L + k + 1023;                   // biased exponent of the error
  if (E < 1) return false;                      // subnormal error: use the FMA
  const uint64_t mant = (L <= 52) ? (M << (52 - L)) : (M >> (L - 52));
  const uint64_t sign = ((ua ^ ub) >> 63 ^ (neg ? 1u : 0u)) & 1u;
  e = from_bits((sign << 63) | ((uint64_t)E << 52) | (mant & kFrac));
  return true;
}

// Multiplication by a power of two.  If a = +-2^k, every product a*b_i is
// exact, every TwoProdFMA error is +0 and every TwoSum with a +0 operand is
// exact, so the printed FP64 x QTW product (Algorithm 10) returns
// (a*b1, a*b2, a*b3) with the two lower words replaced by +0 when they are
// zero (the printed sequence adds +0 to them), and FP64 x QDW returns
// (a*b1, a*b2) likewise.  pow2_scale forms a*b from the bit patterns (an
// exponent add and a sign flip); it declines for a subnormal, infinite or NaN
// b and when the result would leave the normal range.
MWI_HD bool is_pow2(double a) {
  const uint64_t ua = bits_of(a);
  const int ea = (int)((ua >> 52) & 0x7ff);
  return (ua & kFrac) == 0 && ea >= 1 && ea <= 2046;
}
MWI_HD bool pow2_scale(double a, double b, bool plus_zero, double& out) {
  const uint64_t ua = bits_of(a), ub = bits_of(b);
  const uint64_t sign = (ua ^ ub) & ~kAbs;
  if ((ub & kAbs) == 0) { out = plus_zero ? 0.0 : from_bits(sign); return true; }
  const int eb = (int)((ub >> 52) & 0x7ff);
  if (eb == 0 || eb == 2047) return false;
  const int e = eb + (int)((ua >> 52) & 0x7ff) - 1023;
  if (e < 1 || e > 2046) return false;
  out = from_bits(sign | ((uint64_t)e << 52) | (ub & kFrac));
  return true;
}

// FP64 x MW product with a power-of-two FP64 factor a, as the printed
// sequences (Algorithm 10 and its DW / QDW / QQW analogues, before DW's
// closing QuickTwoSum) return it: every TwoProd error and every partner of a
// TwoSum is then zero, so each word is scaled exactly and a zero lower word
// comes out as +0.  For a = +-1 the scaling changes no exponent and holds for
// every finite word, subnormal ones included (a sign flip per word); other
// powers of two need every nonzero scaled word to stay normal (pow2_scale).
// Returns false (the caller runs the printed sequence) for a non-finite word
// or a scaled word that would leave the normal range.
template <int W>
MWI_HD bool pow2_product(double a, const double (&b)[W], double (&c)[W]) {
  const uint64_t ua = bits_of(a);
  if ((ua & kAbs) == 0x3FF0000000000000ULL) {
    const uint64_t sg = ua & ~kAbs;
    bool ok = true;
    for (int k = 0; k < W; ++k) {
      const uint64_t ub = bits_of(b[k]);
      ok = ok && (((ub >> 52) & 0x7ff) != 0x7ff);
      c[k] = (k > 0 && (ub & kAbs) == 0) ? 0.0 : from_bits(ub ^ sg);
    }
    return ok;
  }
  if (!is_pow2(a)) return false;
  for (int k = 0; k < W; ++k)
    if (!pow2_scale(a, b[k], k > 0, c[k])) return false;
  return true;
}

// Precondition under which QuickTwoSum (Algorithm 3) returns the exact error:
// exponent field of a >= exponent field of b, or b = +-0.
MWI_HD bool quick_exact(double a, double b) {
  const uint64_t ua = bits_of(a), ub = bits_of(b);
  return ((ub & kAbs) == 0) || (((ua >> 52) & 0x7ff) >= ((ub >> 52) & 0x7ff));
}

}  // namespace mwi
