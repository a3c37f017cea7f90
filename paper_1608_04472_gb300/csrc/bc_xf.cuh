// bc_xf.cuh -- doubles with an unbounded exponent (value = m * 2^e, m in
// [1,2), or 0): the arithmetic of the extended form used for samples whose
// shortest-path counts exceed 2^64-1. Every operation rounds once to 53 bits
// as IEEE round-to-nearest-even would without an exponent limit.
#pragma once

#include <cstdint>

namespace bcg {

struct Xf {
  double m;
  int e;
};

// 2^k as a double, k in [-1022, 1023]
__device__ __forceinline__ double pow2(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// x * 2^e normalised; x a positive normal double, or 0
__device__ __forceinline__ Xf xf_make(double x, int e) {
  if (x == 0.0) return Xf{0.0, 0};
  const long long b = __double_as_longlong(x);
  const int k = (int)((b >> 52) & 0x7ff) - 1023;
  return Xf{__longlong_as_double((b & 0x000fffffffffffffLL) | (1023LL << 52)), e + k};
}

// RN(a + b), a, b >= 0: a term more than 60 binades below the other is under a
// quarter ulp of it; otherwise both mantissas are exact on a common scale and
// one double addition rounds their exact sum.
__device__ __forceinline__ Xf xf_add(Xf a, Xf b) {
  if (a.m == 0.0) return b;
  if (b.m == 0.0) return a;
  if (a.e < b.e) {
    const Xf t = a;
    a = b;
    b = t;
  }
  const long long d = (long long)a.e - (long long)b.e;
  if (d > 60) return a;
  return xf_make(__dadd_rn(a.m, __dmul_rn(b.m, pow2(-(int)d))), a.e);
}

// RN(a * b) as a double: the mantissa product rounds once; steps of 2^1000 are
// exact while the value stays normal and only the last one can round.
__device__ __forceinline__ double xf_mul_to_double(Xf a, Xf b) {
  if (a.m == 0.0 || b.m == 0.0) return 0.0;
  double p = __dmul_rn(a.m, b.m);
  long long k = (long long)a.e + (long long)b.e;
  while (k > 1000) {
    p = __dmul_rn(p, pow2(1000));
    k -= 1000;
  }
  while (k < -1000) {
    p = __dmul_rn(p, pow2(-1000));
    k += 1000;
  }
  return __dmul_rn(p, pow2((int)k));
}

// RN(x / b) for a double x >= 1/2 and b > 0
__device__ __forceinline__ Xf xf_div(double x, Xf b) { return xf_make(__ddiv_rn(x, b.m), -b.e); }

__device__ __forceinline__ Xf xf_load(const double *xm, const int32_t *xe, size_t i) { return Xf{xm[i], xe[i]}; }
__device__ __forceinline__ void xf_store(double *xm, int32_t *xe, size_t i, Xf x) {
  xm[i] = x.m;
  xe[i] = x.e;
}

// RN(a * b) and RN(a / b) in the extended form; the value as a double (only
// the last power-of-two step can round).
__device__ __forceinline__ Xf xf_mul(Xf a, Xf b) {
  if (a.m == 0.0 || b.m == 0.0) return Xf{0.0, 0};
  return xf_make(__dmul_rn(a.m, b.m), a.e + b.e);
}
__device__ __forceinline__ Xf xf_div_xf(Xf a, Xf b) {
  if (a.m == 0.0) return Xf{0.0, 0};
  return xf_make(__ddiv_rn(a.m, b.m), a.e - b.e);
}
__device__ __forceinline__ double xf_to_double(Xf a) { return xf_mul_to_double(a, Xf{1.0, 0}); }
__device__ __forceinline__ Xf xf_of_u64(uint64_t x) { return xf_make(__ull2double_rn(x), 0); }

// Pair dependency sigma_sv * sigma_vt / sigma_st (Eq. 2) from counts that are
// exact uint64 or, when flagged, extended (mantissa bits + exponent):
// RN(RN(a * b) / c) without an exponent limit; with no flag set this equals
// the double formula RN(RN(a * b) / c) on the rounded counts.
__device__ __forceinline__ double pair_y(bool vx, uint64_t a, int ae, uint64_t b, int be, bool px, uint64_t c,
                                         int ce) {
  const Xf A = vx ? Xf{__longlong_as_double((long long)a), ae} : xf_of_u64(a);
  const Xf B = vx ? Xf{__longlong_as_double((long long)b), be} : xf_of_u64(b);
  const Xf C = px ? Xf{__longlong_as_double((long long)c), ce} : xf_of_u64(c);
  return xf_to_double(xf_div_xf(xf_mul(A, B), C));
}

}  // namespace bcg
