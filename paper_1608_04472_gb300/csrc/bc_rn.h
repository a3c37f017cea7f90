// bc_rn.h -- the double operations of the per-vertex dependency step (Theorem 1
// in factored form) evaluated with integer instructions only, each rounded once
// to nearest, ties to even, exactly as IEEE-754 binary64 arithmetic rounds:
//
//   rn_u53_to_double(s)   s exactly (s < 2^53)
//   rn_mul_u53(s, y)      RN(s * y)      s integer in [1, 2^53), y >= 0
//   rn_one_plus(x)        RN(1 + x)      x >= 0
//   rn_div_u53(x, s)      RN(x / s)      x >= 1, s integer in [1, 2^53)
//
// Why: on GB300 the FP64 pipe retires about two operations per SM per clock,
// so one warp-wide double divide (a reciprocal and several fused multiply-adds)
// holds it for hundreds of cycles, while the integer pipes are wide. Operands
// here are positive, finite and normal, and no result leaves the normal range
// (x >= 1, s < 2^53), so no subnormal, infinity or NaN case arises.
//
// Division (rn_div_u53): with b the bit length of s (s not a power of two),
// Q = floor(m_x * 2^(b+2) / s) has 55-56 bits; it is estimated from a 64-bit
// fixed-point reciprocal r ~ 2^(63+b)/s, refined from a single-precision seed
// by two Newton-Raphson steps r <- r + r*(1 - s*r/2^(63+b)), then made exact
// by the remainder m_x*2^(b+2) - Q*s (computed modulo 2^64: it is small) and
// at most a few +-1 corrections; the remainder's sign and zero test give the
// rounding. Written for host (tests against the platform's IEEE division) and
// device alike.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define RN_HD __host__ __device__ __forceinline__
#else
#define RN_HD static inline
#endif

namespace bcrn {

constexpr uint64_t MANT = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t HIDDEN = 0x0010000000000000ull;

RN_HD uint64_t bits_of(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
  return b;
#endif
}

RN_HD double double_of(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}

RN_HD uint64_t mulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

RN_HD int clz64(uint64_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

// Correctly rounded single-precision reciprocal (IEEE division on the host,
// the round-to-nearest reciprocal on the device: the same value).
RN_HD float rcp_f32(float x) {
#if defined(__CUDA_ARCH__)
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}

// 2^k as a float, -126 <= k <= 127 (exact).
RN_HD float pow2f(int k) {
  const uint32_t u = (uint32_t)(127 + k) << 23;
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

// Rounds the integer mant * 2^sh + (lower bits: round bit rb, sticky st) to 53
// bits, where mant in [2^52, 2^53), and returns the double
// mant' * 2^(e - 1075) with e the biased exponent the unrounded mant has: the
// carry of a mantissa that rounds up to 2^53 moves into the exponent field.
RN_HD double pack_rne(uint64_t mant, bool rb, bool st, int biased) {
  if (rb && (st || (mant & 1ull))) mant += 1ull;
  return double_of(((uint64_t)(biased - 1) << 52) + mant);
}

// s exactly, s in [1, 2^53).
RN_HD double rn_u53_to_double(uint64_t s) {
  const int b = 64 - clz64(s);  // 2^(b-1) <= s < 2^b
  return double_of(((uint64_t)(1021 + b) << 52) + (s << (53 - b)));
}

// RN(s * y), s in [1, 2^53), y >= 0 finite and normal (or zero).
RN_HD double rn_mul_u53(uint64_t s, double y) {
  const uint64_t yb = bits_of(y);
  if (yb == 0ull) return 0.0;
  const int ey = (int)(yb >> 52);
  const uint64_t my = (yb & MANT) | HIDDEN;
  const uint64_t lo = s * my, hi = mulhi(s, my);  // P = hi:lo in [2^52, 2^106)
  const int L = hi ? 128 - clz64(hi) : 64 - clz64(lo);
  const int sh = L - 53;  // 0 .. 53
  if (sh == 0) return pack_rne(lo, false, false, ey);
  const uint64_t mant = (lo >> sh) | (hi << (64 - sh));
  const bool rb = ((lo >> (sh - 1)) & 1ull) != 0ull;
  const bool st = (lo & ((1ull << (sh - 1)) - 1ull)) != 0ull;
  return pack_rne(mant, rb, st, ey + sh);
}

// RN(1 + x), x >= 0 finite and normal (or zero).
RN_HD double rn_one_plus(double x) {
  const uint64_t xb = bits_of(x);
  if (xb == 0ull) return 1.0;
  const int ex = (int)(xb >> 52);
  const uint64_t mx = (xb & MANT) | HIDDEN;
  if (ex >= 1023) {
    // x >= 1: the sum has x's exponent or one more; 1 is 2^(1075-ex) units of x
    const int k = ex - 1023;  // x in [2^k, 2^(k+1))
    if (k <= 52) {
      const uint64_t S = mx + (1ull << (52 - k));  // exact, < 2^54
      if (S < (HIDDEN << 1)) return pack_rne(S, false, false, ex);
      return pack_rne(S >> 1, (S & 1ull) != 0ull, false, ex + 1);
    }
    // 1 is below one unit of x: a tie at exactly half a unit (k == 53), else x
    return pack_rne(mx, k == 53, false, ex);
  }
  // x < 1: the sum lies in [1, 2) before rounding; x is m_x * 2^(ex-1075),
  // i.e. m_x >> (1023 - ex) units of 2^-52
  const int sh = 1023 - ex;  // >= 1
  uint64_t q;
  bool rb, st;
  if (sh <= 63) {
    q = mx >> sh;
    rb = ((mx >> (sh - 1)) & 1ull) != 0ull;
    st = (mx & ((1ull << (sh - 1)) - 1ull)) != 0ull;
  } else {
    q = 0ull;
    rb = (sh == 64) && ((mx >> 63) & 1ull);  // m_x < 2^53: never set
    st = true;
  }
  return pack_rne(HIDDEN + q, rb, st, 1023);
}

// RN(x / s), x >= 1 finite, s in [1, 2^53).
RN_HD double rn_div_u53(double x, uint64_t s) {
  const uint64_t xb = bits_of(x);
  const int ex = (int)(xb >> 52);
  const uint64_t mx = (xb & MANT) | HIDDEN;
  const int b = 64 - clz64(s);
  if ((s & (s - 1ull)) == 0ull) {
    // s = 2^(b-1): exact exponent shift
    return double_of(xb - ((uint64_t)(b - 1) << 52));
  }
  // seed: the top 32 bits of s, s32 = s >> max(b - 32, 0), converted from a
  // 32-bit integer (no 64-bit conversion); rf = RN(1/RN(s32)) * 2^min(b, 32)
  // ~ 2^b/s in [1, 2] (relative error < 2^-22); r0 = rf * 2^63 ~ 2^(63+b)/s,
  // read off rf's bits: rf = 1.m (24 bits) gives 2^63 + m * 2^40, rf = 2 the
  // largest 64-bit value
  const int sh32 = b > 32 ? b - 32 : 0;
  const float rf = rcp_f32((float)(uint32_t)(s >> sh32)) * pow2f(b - sh32);
  uint32_t fb;
#if defined(__CUDA_ARCH__)
  fb = __float_as_uint(rf);
#else
  memcpy(&fb, &rf, 4);
#endif
  uint64_t r = (fb >> 23) >= 128u ? ~0ull : ((1ull << 63) | ((uint64_t)(fb & 0x7FFFFFu) << 40));
  // Newton-Raphson: E = 2^(63+b) - s*r (|E| << 2^(63+b)); r += r*E/2^(63+b)
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const uint64_t plo = s * r, phi = mulhi(s, r);
    // E = 2^(63+b) - (phi:plo) as a 128-bit two's complement number; b >= 2
    const uint64_t elo = 0ull - plo;
    const uint64_t ehi = (1ull << (b - 1)) - phi - (plo != 0ull ? 1ull : 0ull);
    // E' = E >> b (arithmetic): |E'| < 2^63 since |E| < 2^(62+b)
    const int64_t e = (int64_t)((elo >> b) | (ehi << (64 - b)));
    // correction r*E/2^(63+b) = r*E'/2^63 = 2*mulhi(r, |E'|) (+ truncation)
    if (e >= 0) {
      r += mulhi(r, (uint64_t)e) << 1;
    } else {
      r -= mulhi(r, (uint64_t)(-e)) << 1;
    }
  }
  // Q ~ m_x * r / 2^61 = m_x * 2^(b+2) / s
  const uint64_t qlo = mx * r, qhi = mulhi(mx, r);
  uint64_t Q = (qhi << 3) | (qlo >> 61);
  // exact remainder N - Q*s, N = m_x * 2^(b+2); |rem| < 2^63, so mod 2^64 is exact
  const uint64_t N_lo = mx << (b + 2);  // b + 2 <= 55
  int64_t rem = (int64_t)(N_lo - Q * s);
  // (the estimate is off by at most one here; two steps leave a margin)
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    if (rem < 0) {
      Q -= 1ull;
      rem += (int64_t)s;
    } else if ((uint64_t)rem >= s) {
      Q += 1ull;
      rem -= (int64_t)s;
    }
  }
  // x/s = (Q + rem/s) * 2^(ex - 1075 - b - 2), Q in [2^54, 2^56)
  const int L = 64 - clz64(Q);  // 55 or 56
  const int sh = L - 53;        // 2 or 3
  const uint64_t mant = Q >> sh;
  const bool rb = ((Q >> (sh - 1)) & 1ull) != 0ull;
  const bool st = rem != 0 || (Q & ((1ull << (sh - 1)) - 1ull)) != 0ull;
  // value = mant * 2^(sh + ex - 1077 - b): biased exponent of mant*2^-52 is sh + ex - b - 2
  return pack_rne(mant, rb, st, sh + ex - b - 2);
}

}  // namespace bcrn
