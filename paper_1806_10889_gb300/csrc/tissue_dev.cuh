// Device building blocks of the tissue SSA (sm_103a).
//
// Counter-based random numbers, the fixed-point exponential variate, integer
// propensities with exact overflow detection, and warp-level helpers.  All
// arithmetic here is exact integer arithmetic or single IEEE binary64
// operations through the _rn intrinsics, so the results are reproducible bit
// for bit on any IEEE machine.
#pragma once
#include <cstdint>

#include "tissue_internal.h"

namespace tsg {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Checked build (compiled with -DTISSUE_CHECKED; the stand-in for a memory
// sanitizer).  TSG_IDX(i, n, flag) is the array index i when 0 <= i < n;
// otherwise it sets `flag` (reported as a bounds error through the device
// error flag) and gives 0, so the access lands on element 0 instead of
// outside the array.  In the normal build it is i itself: no instruction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long checked_index(long long i, long long n, bool& flag) {
  const bool ok = i >= 0 && i < n;
  flag |= !ok;
  return ok ? i : 0;
}
#ifdef TISSUE_CHECKED
#define TSG_IDX(i, n, flag) ::tsg::checked_index((i), (n), (flag))
constexpr bool kChecked = true;
#else
#define TSG_IDX(i, n, flag) (i)
constexpr bool kChecked = false;
#endif

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications whose high words are xored into the other
// counter words with the round key; the key advances by the golden-ratio and
// sqrt(3)-1 Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// ---------------------------------------------------------------------------
// -ln(k * 2^-53) * 2^58 for k in [1, 2^53], in integer arithmetic.
// Write k = 2^j m, m in [1,2).  With h = (m-1)/2 (m <= sqrt 2) or
// h = (2-m)/4 (m > sqrt 2, one more power of two), ln of the mantissa part is
// +-2 atanh(h / (1 +- h)) (Abramowitz & Stegun 4.1.27).  1/(1 +- h) comes from
// four Newton-Raphson steps y <- y (2 - d y) started at 2 - d; atanh(s)/s is
// the series sum_{i<=11} s^{2i} / (2i+1) evaluated by Horner's rule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mul_q62(uint64_t a, uint64_t b) {
  return (__umul64hi(a, b) << 2) | ((a * b) >> 62);
}

// round(2^63 / (2i + 1)); never a tie since 2i + 1 > 1 is odd.
__host__ __device__ constexpr uint64_t atanh_coef(int i) {
  return (0x8000000000000000ull + static_cast<uint64_t>(i)) / (2ull * i + 1ull);
}

__device__ __forceinline__ uint64_t neg_ln_q58(uint64_t k) {
  const int lz = __clzll(static_cast<long long>(k));
  const uint64_t m = k << lz;  // Q1.63
  const bool upper = m > 0xB504F333F9DE6484ull;  // floor(sqrt 2 * 2^63)
  const uint64_t h = upper ? ((0ull - m) >> 1) : (m - 0x8000000000000000ull);
  const uint64_t d = upper ? (0x4000000000000000ull - (h >> 2)) : (0x4000000000000000ull + (h >> 2));
  uint64_t y = 0x8000000000000000ull - d;
#pragma unroll
  for (int it = 0; it < 4; ++it) y = mul_q62(y, 0x8000000000000000ull - mul_q62(d, y));
  const uint64_t s = mul_q62(h, y);
  const uint64_t z = __umul64hi(s, s);
  constexpr uint64_t kC[12] = {atanh_coef(0), atanh_coef(1), atanh_coef(2),  atanh_coef(3),
                               atanh_coef(4), atanh_coef(5), atanh_coef(6),  atanh_coef(7),
                               atanh_coef(8), atanh_coef(9), atanh_coef(10), atanh_coef(11)};
  uint64_t p = kC[11];
#pragma unroll
  for (int i = 10; i >= 0; --i) p = __umul64hi(p, z) + kC[i];
  const uint64_t two_atanh = mul_q62(s, p);
  const uint64_t nln2 = static_cast<uint64_t>(upper ? 52 - (63 - lz) : 53 - (63 - lz));
  constexpr uint64_t kLn2Q64 = 0xB17217F7D1CF79ACull;  // round(ln 2 * 2^64)
  uint64_t lo = nln2 * kLn2Q64, hi = __umul64hi(nln2, kLn2Q64);
  if (upper) {
    const uint64_t t = lo + two_atanh;
    hi += (t < lo);
    lo = t;
  } else {
    hi -= (lo < two_atanh);
    lo -= two_atanh;
  }
  return (hi << 58) | (lo >> 6);
}

// Unit-mean exponential from Philox words 0,1: u1 = (bits53 + 1) 2^-53.
__device__ __forceinline__ double exp_variate(uint32_t w0, uint32_t w1) {
  const uint64_t bits = ((static_cast<uint64_t>(w1) << 32) | w0) >> 11;
  return __dmul_rn(__ull2double_rn(neg_ln_q58(bits + 1)), 0x1p-58);
}

// ---------------------------------------------------------------------------
// Integer propensities.  a*x is exact; the flag records whether the exact
// product reached 2^52 (the per-voxel / per-channel limit).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mul_lim(uint64_t a, uint64_t x, bool& ovf) {
  const uint64_t lo = a * x;
  ovf |= (__umul64hi(a, x) != 0ull) | ((lo >> 52) != 0ull);
  return lo;
}

// Hill-repressed Delta production kD / (1 + (R/K)^2), binary64, quantised.
__device__ __forceinline__ uint64_t hill_direct(const QRates& q, uint32_t R) {
  const double x = __ddiv_rn(static_cast<double>(R), q.K);
  const double den = __dadd_rn(1.0, __dmul_rn(x, x));
  return __double2ull_rn(__dmul_rn(__ddiv_rn(q.kD, den), 4294967296.0));
}

__device__ __forceinline__ uint64_t hill_q(const QRates& q, uint32_t R) {
  return R < kHillTab ? __ldg(q.hill + R) : hill_direct(q, R);
}

// ---------------------------------------------------------------------------
// Binary64 time arithmetic in integer registers.
//
// tau = E / (A 2^-32) must be the IEEE round-to-nearest quotient.  The
// hardware division costs ~140 cycles of the SM's FP64 pipe per warp on
// GB300 even with one active lane, so the event loop computes the same
// correctly rounded result with integer instructions:
//   1. E (Q.58) and A are rounded to 53-bit significands exactly as the
//      integer-to-binary64 conversion does (round half to even).
//   2. Y ~ 2^115 / mA from a single-precision reciprocal estimate refined by
//      one third-order Newton-Raphson (Householder) step in fixed point; the
//      quotient estimate floor(mE 2^sh / mA) is then corrected with the exact
//      remainder (long division with a reciprocal, Knuth, TAOCP vol. 2,
//      4.3.1; Moller & Granlund, IEEE TC 60(2), 2011).
//   3. The 53-bit quotient is rounded to nearest with the remainder
//      (a binary division can never land exactly half-way) and assembled.
// ---------------------------------------------------------------------------
struct F53 {
  uint64_t m;  // significand in [2^52, 2^53)
  int k;       // x ~ m * 2^(k - 52)
};

// Round x >= 1 to 53 significant bits, half to even: by definition the
// u64 -> binary64 conversion, so the hardware conversion does it in one
// instruction; the significand (with its leading bit) and the exponent are
// then read from the bits.
__device__ __forceinline__ F53 round53(uint64_t x) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(__ull2double_rn(x)));
  return F53{(b & ((1ull << 52) - 1ull)) | (1ull << 52), static_cast<int>(b >> 52) - 1023};
}

// floor(2^115 / d) within +-2, d in (2^52, 2^53).  Seed y0 = m24 * 2^39 from
// the single-precision reciprocal of d's top 24 bits (relative error < 2^-21),
// then one third-order step y = y0 (1 + e + e^2), e = 1 - d y0 / 2^115, which
// leaves a relative error near e^3 < 2^-63.  The reciprocal of d >> 29, a
// value in [2^23, 2^24), lies in (2^-24, 2^-23]; capping it just below 2^-23
// keeps its exponent, and so every shift below, constant.  d*y0 differs from
// 2^115 by less than 2^94 (|e'| < 2^55 below), so e is exact from the low 64
// bits of d*m24.
__device__ __forceinline__ uint64_t recip115(uint64_t d) {
  const float df = static_cast<float>(static_cast<uint32_t>(d >> 29));  // exact: < 2^24
  float f;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"(df));
  f = fminf(f, __uint_as_float(0x33FFFFFFu));  // largest float below 2^-23
  const uint32_t m24 = (__float_as_uint(f) & 0x7FFFFFu) | 0x800000u;  // y0 = m24 * 2^39
  // e * 2^76 = 2^76 - d*m24; the power of two vanishes mod 2^64
  const int64_t e = -static_cast<int64_t>(d * static_cast<uint64_t>(m24));
  const uint64_t ae = static_cast<uint64_t>(e < 0 ? -e : e);
  // t1 = y0 |e| = m24 |e'| / 2^37, from the 32-bit halves of |e'|
  const uint64_t P1 = static_cast<uint64_t>(m24) * static_cast<uint32_t>(ae >> 32);
  const uint64_t P0 = static_cast<uint64_t>(m24) * static_cast<uint32_t>(ae);
  const uint64_t t1 = (P1 >> 5) + ((((P1 & 31ull) << 32) + P0) >> 37);
  // t2 = y0 e^2 = m24 e'^2 / 2^113 >= 0, to a fraction of a unit
  const uint64_t e24 = ae >> 24;            // < 2^31
  const uint64_t e2 = (e24 * e24) >> 24;    // e'^2 / 2^72
  const uint64_t t2 = (static_cast<uint64_t>(m24) * e2) >> 41;
  const uint64_t y0 = static_cast<uint64_t>(m24) << 39;
  return (e >= 0 ? y0 + t1 : y0 - t1) + t2;
}

// IEEE binary64 RN quotient (E_q58 * 2^-58) / (RN(A) * 2^-32), as a double.
// E_q58 = 0 gives +0.  eq = round53(E_q58) is passed in (it is per draw).
__device__ __forceinline__ double tau_from(const F53 eq, bool e_zero, uint64_t A) {
  if (e_zero) return 0.0;
  const F53 a = round53(A);
  const uint64_t mE = eq.m, d = a.m;
  const int sh = mE >= d ? 52 : 53;  // quotient significand lands in [2^52, 2^53)
  // h = floor(mE 2^(sh+1) / d): the quotient with one more bit.  The quotient
  // of two 53-bit significands is never exactly half-way between two 53-bit
  // values, so the rounded quotient is (h + 1) >> 1.
  uint64_t h;
  if (d == (1ull << 52)) {           // power-of-two divisor: exact shift
    h = mE << (sh - 51);
  } else {
    const uint64_t y = recip115(d);
    const uint64_t plo = mE * y, phi = __umul64hi(mE, y);
    h = sh == 52 ? ((phi << 2) | (plo >> 62)) : ((phi << 3) | (plo >> 61));
    // |y - 2^115/d| <= 2 makes the estimate off by at most one either way
    int64_t r = static_cast<int64_t>((mE << (sh + 1)) - h * d);  // exact: |r| < 2^56
    if (r < 0) { h -= 1; r += static_cast<int64_t>(d); }
    if (r >= static_cast<int64_t>(d)) h += 1;
  }
  const uint64_t q = (h + 1ull) >> 1;
  // tau = q * 2^X with X = (kE - 110) - (kA - 84) - sh; a carry of q into
  // 2^53 moves into the exponent field by itself.
  const int X = eq.k - a.k - 26 - sh;
  const uint64_t bits = (static_cast<uint64_t>(X + 1075) << 52) + (q - (1ull << 52));
  return __longlong_as_double(static_cast<long long>(bits));
}

// t < dt for non-negative doubles: the IEEE order is the integer order of the bits.
__device__ __forceinline__ bool before(double t, double dt) {
  return __double_as_longlong(t) < __double_as_longlong(dt);
}

// One lane's draw for event e: the exponential variate as a rounded
// 53-bit significand and exponent (exponent -1 encodes E = 0) and the 64
// selection bits.
__device__ __forceinline__ void draw_event(uint32_t e, uint32_t step, uint32_t unit,
                                           uint32_t word3, uint32_t key0, uint32_t key1,
                                           uint64_t& Em, int& Ek, uint64_t& Rb) {
  const U4 w = philox10(e, step, unit, word3, key0, key1);
  const uint64_t q = neg_ln_q58((((static_cast<uint64_t>(w.y) << 32) | w.x) >> 11) + 1);
  const F53 f = round53(q | static_cast<uint64_t>(q == 0ull));
  Em = f.m;
  Ek = q ? f.k : -1;
  Rb = (static_cast<uint64_t>(w.w) << 32) | w.z;
}

// v / n for v < 1024, n <= 32: (v * ceil(2^16 / n)) >> 16 is exact there.
__device__ __forceinline__ int div_n(int v, uint32_t magic) {
  return static_cast<int>((static_cast<uint32_t>(v) * magic) >> 16);
}

}  // namespace tsg
