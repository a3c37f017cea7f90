// bc_common.cuh -- device primitives shared by the GB300 kernels:
// counter-based draws, the exact fixed-point accumulator, warp helpers, and
// host-side launch/error plumbing. Written for sm_103a.
#pragma once

#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "bc_rn.h"

namespace bcg {

constexpr unsigned FULL = 0xffffffffu;

// Error bits raised by kernels into a device status word.
constexpr unsigned ERR_SIGMA_OVERFLOW = 1u;  // a path count exceeded 2^64-1
constexpr unsigned ERR_RANGE = 2u;           // a value left the exact accumulator window
constexpr unsigned ERR_TIMEOUT = 4u;         // a bounded wait ran out

// ------------------------------------------------------------------ Philox --
// Philox4x64 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): per round the
// counter words 0 and 2 are multiplied by the two round constants; high and low
// halves are recombined with words 1 and 3 and the key; between rounds the key
// is bumped by the two Weyl constants.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

// Draw i of stream (seed, qid): uniform source vertex in [0, n).
__device__ __forceinline__ int32_t draw_source(uint64_t seed, uint64_t qid, uint64_t i, int32_t n) {
  uint64_t c[4] = {i, 0, 0, 0};
  philox4x64_10(c, seed, qid);
  return (int32_t)__umul64hi(c[0], (uint64_t)n);
}

// Draw i of stream (seed, qid): ordered pair (u, t) of different vertices, uniform
// over the n(n-1) ordered pairs.
__device__ __forceinline__ void draw_pair(uint64_t seed, uint64_t qid, uint64_t i, int32_t n,
                                          int32_t &u, int32_t &t) {
  uint64_t c[4] = {i, 0, 0, 0};
  philox4x64_10(c, seed, qid);
  const uint64_t a = __umul64hi(c[0], (uint64_t)n);
  const uint64_t w = __umul64hi(c[1], (uint64_t)(n - 1));
  u = (int32_t)a;
  t = (int32_t)(w + (w >= a ? 1ull : 0ull));
}

// --------------------------------------------------------- exact accumulator --
// A 192-bit unsigned fixed-point number, value = (w0 + w1*2^64 + w2*2^128) * 2^-128.
// Every double in [2^-76, 2^63) is an integer multiple of 2^-128 below 2^191, so
// additions are exact and order-independent. Dependencies lie in [2^-64, 2^31]
// and coefficients (1+delta)/sigma in [2^-64, 2^31] while sigma < 2^64, so sums of
// fewer than 2^32 of them fit. acc_round returns the sum rounded once to the
// nearest double, ties to even.
struct Acc {
  uint64_t w0, w1, w2;
};

__device__ __forceinline__ Acc acc_zero() { return Acc{0ull, 0ull, 0ull}; }

__device__ __forceinline__ void acc_add3(Acc &a, uint64_t t0, uint64_t t1, uint64_t t2) {
  const uint64_t s0 = a.w0 + t0;
  const uint64_t c0 = s0 < t0 ? 1ull : 0ull;
  uint64_t s1 = a.w1 + t1;
  uint64_t c1 = s1 < t1 ? 1ull : 0ull;
  s1 += c0;
  c1 |= (s1 < c0) ? 1ull : 0ull;
  a.w0 = s0;
  a.w1 = s1;
  a.w2 = a.w2 + t2 + c1;
}

// Adds x (0, or a normal double in [2^-76, 2^63)). Out-of-window values set
// ERR_RANGE in err and are dropped.
__device__ __forceinline__ void acc_add(Acc &a, double x, unsigned &err) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  if (bits == 0ull) return;
  const int e = (int)(bits >> 52);  // biased exponent (x >= 0)
  const int p = e - 947;            // position of the mantissa's lowest bit
  if (p < 0 || p > 138) { err |= ERR_RANGE; return; }
  const uint64_t m = (bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int q = p >> 6, r = p & 63;
  const uint64_t lo = m << r;
  const uint64_t hi = r ? (m >> (64 - r)) : 0ull;
  const uint64_t t0 = (q == 0) ? lo : 0ull;
  const uint64_t t1 = (q == 0) ? hi : ((q == 1) ? lo : 0ull);
  const uint64_t t2 = (q == 1) ? hi : ((q == 2) ? lo : 0ull);
  acc_add3(a, t0, t1, t2);
}

__device__ __forceinline__ void acc_add_acc(Acc &a, const Acc &b) { acc_add3(a, b.w0, b.w1, b.w2); }

// low 64 bits of (w2:w1:w0) >> s, 0 <= s < 192
__device__ __forceinline__ uint64_t acc_shr64(const Acc &a, int s) {
  const int q = s >> 6, r = s & 63;
  const uint64_t x = (q == 0) ? a.w0 : ((q == 1) ? a.w1 : a.w2);
  const uint64_t y = (q == 0) ? a.w1 : ((q == 1) ? a.w2 : 0ull);
  return r ? ((x >> r) | (y << (64 - r))) : x;
}

// any of the lowest s bits set, 0 <= s <= 192
__device__ __forceinline__ bool acc_any_below(const Acc &a, int s) {
  const int q = s >> 6, r = s & 63;
  bool any = false;
  if (q >= 1) any |= (a.w0 != 0ull);
  if (q >= 2) any |= (a.w1 != 0ull);
  if (q >= 3) any |= (a.w2 != 0ull);
  if (q < 3 && r) {
    const uint64_t w = (q == 0) ? a.w0 : ((q == 1) ? a.w1 : a.w2);
    any |= (w & ((1ull << r) - 1ull)) != 0ull;
  }
  return any;
}

__device__ __forceinline__ double acc_round(const Acc &a) {
  int top;
  if (a.w2) top = 191 - __clzll((long long)a.w2);
  else if (a.w1) top = 127 - __clzll((long long)a.w1);
  else if (a.w0) top = 63 - __clzll((long long)a.w0);
  else return 0.0;
  if (top <= 52) {  // fewer than 54 significant bits: exact, w0 * 2^-128
    return bcrn::double_of(bcrn::bits_of(bcrn::rn_u53_to_double(a.w0)) - (128ull << 52));
  }
  int sh = top - 52;  // 1..139
  uint64_t M = acc_shr64(a, sh) & 0x001FFFFFFFFFFFFFull;
  const bool rbit = (acc_shr64(a, sh - 1) & 1ull) != 0ull;
  const bool sticky = acc_any_below(a, sh - 1);
  if (rbit && (sticky || (M & 1ull))) {
    M += 1ull;
    if (M == 0x0020000000000000ull) { M >>= 1; sh += 1; }
  }
  const uint64_t bits = ((uint64_t)(sh + 947) << 52) | (M & 0x000FFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// Exact butterfly sum over the warp; every lane ends with the total.
__device__ __forceinline__ Acc acc_warp_sum(Acc a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Acc o;
    o.w0 = __shfl_xor_sync(FULL, a.w0, off);
    o.w1 = __shfl_xor_sync(FULL, a.w1, off);
    o.w2 = __shfl_xor_sync(FULL, a.w2, off);
    acc_add_acc(a, o);
  }
  return a;
}

// A narrower exact accumulator for successor sums: 128 bits in 32-bit limbs,
// value = (l3:l2:l1:l0) * 2^-96, holding every double in [2^-44, 2^32). When
// sigma <= 2^44 every coefficient RN((1+delta)/sigma) is >= 2^-44, and a
// successor sum equals delta_v/sigma_v <= n < 2^31 up to rounding, so the
// window is never left; out-of-window values set ERR_RANGE.
struct Acc2 {
  uint32_t l0, l1, l2, l3;
};

__device__ __forceinline__ Acc2 acc2_zero() { return Acc2{0u, 0u, 0u, 0u}; }

__device__ __forceinline__ void acc2_add4(Acc2 &a, uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3) {
  asm("add.cc.u32 %0, %0, %4;\n\t"
      "addc.cc.u32 %1, %1, %5;\n\t"
      "addc.cc.u32 %2, %2, %6;\n\t"
      "addc.u32 %3, %3, %7;"
      : "+r"(a.l0), "+r"(a.l1), "+r"(a.l2), "+r"(a.l3)
      : "r"(t0), "r"(t1), "r"(t2), "r"(t3));
}

__device__ __forceinline__ void acc2_add(Acc2 &a, double x, unsigned &err) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  if (bits == 0ull) return;
  const uint32_t hi = (uint32_t)(bits >> 32), lo = (uint32_t)bits;
  const int p = (int)(hi >> 20) - 979;  // lowest mantissa bit, in units of 2^-96
  if ((unsigned)p > 75u) { err |= ERR_RANGE; return; }
  const uint32_t mh = (hi & 0x000FFFFFu) | 0x00100000u;
  const int r = p & 31, q = p >> 5;
  const uint32_t c0 = lo << r;
  const uint32_t c1 = __funnelshift_l(lo, mh, r);
  const uint32_t c2 = __funnelshift_l(mh, 0u, r);
  const uint32_t t0 = (q == 0) ? c0 : 0u;
  const uint32_t t1 = (q == 0) ? c1 : ((q == 1) ? c0 : 0u);
  const uint32_t t2 = (q == 0) ? c2 : ((q == 1) ? c1 : c0);
  const uint32_t t3 = (q == 1) ? c2 : ((q == 2) ? c1 : 0u);
  acc2_add4(a, t0, t1, t2, t3);
}

// The same value in the 192-bit format (unit 2^-128).
__device__ __forceinline__ Acc acc2_widen(const Acc2 &a) {
  return Acc{(uint64_t)a.l0 << 32, (uint64_t)a.l1 | ((uint64_t)a.l2 << 32), (uint64_t)a.l3};
}

// ------------------------------------------------------ Brandes arithmetic --
// The per-vertex step of Theorem 1 in factored form, every operation rounded
// once: delta = RN(RN(sigma) * sum), coef = RN(RN(1 + delta) / RN(sigma)).
// Counts below 2^53 (every count of the narrow backward path) go through the
// integer-only forms of bc_rn.h, which round exactly as the FP64 instructions
// do but keep the slow FP64 pipe free; larger counts use the FP64 instructions.
// BCG_RN_INT=0 at compile time takes the FP64 instructions throughout (the
// same results; for measuring what the integer forms save).
#ifndef BCG_RN_INT
#define BCG_RN_INT 1
#endif
constexpr uint64_t EXACT53 = BCG_RN_INT ? (1ull << 53) : 0ull;

__device__ __forceinline__ double sigma_to_double(uint64_t s) {
  if (s == 0ull) return 0.0;
  return s < EXACT53 ? bcrn::rn_u53_to_double(s) : __ull2double_rn(s);
}

// RN(RN(sigma) * sum), sum >= 0 normal or zero, sigma >= 1.
__device__ __forceinline__ double delta_rn(uint64_t sigma, double sum) {
  return sigma < EXACT53 ? bcrn::rn_mul_u53(sigma, sum) : __dmul_rn(sigma_to_double(sigma), sum);
}

// RN(RN(1 + delta) / RN(sigma)), delta >= 0 normal or zero, sigma >= 1.
__device__ __forceinline__ double coef_of(double delta, uint64_t sigma) {
  const double x = BCG_RN_INT ? bcrn::rn_one_plus(delta) : __dadd_rn(1.0, delta);
  if ((sigma & (sigma - 1ull)) == 0ull) {  // power of two: exact scaling
    const int k = 63 - __clzll((long long)sigma);
    return __longlong_as_double((long long)((uint64_t)__double_as_longlong(x) - ((uint64_t)k << 52)));
  }
  return sigma < EXACT53 ? bcrn::rn_div_u53(x, sigma) : __ddiv_rn(x, sigma_to_double(sigma));
}

// The same two values by the FP64 instructions. The one-source-per-CTA
// engines (lane-major, weighted) take these: they issue few FP64 operations
// per memory access, and there the integer forms measured 4.5 % slower.
__device__ __forceinline__ double delta_rn_fp(uint64_t sigma, double sum) {
  return __dmul_rn(__ull2double_rn(sigma), sum);
}

__device__ __forceinline__ double coef_of_fp(double delta, uint64_t sigma) {
  const double x = __dadd_rn(1.0, delta);
  if ((sigma & (sigma - 1ull)) == 0ull) {  // power of two: exact scaling
    const int k = 63 - __clzll((long long)sigma);
    return __longlong_as_double((long long)((uint64_t)__double_as_longlong(x) - ((uint64_t)k << 52)));
  }
  return __ddiv_rn(x, __ull2double_rn(sigma));
}

}  // namespace bcg
