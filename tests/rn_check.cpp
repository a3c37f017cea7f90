// Checks the integer-only double operations of the library's dependency step
// (paper_1608_04472_gb300/csrc/bc_rn.h) against the platform's IEEE-754 binary64
// arithmetic (round to nearest even): random operands over the ranges the step
// uses and beyond, operands next to powers of two, all-ones and all-zeros
// mantissas, and half-way cases. Prints the number of mismatches; exit status 1
// if there is any.
#include "../paper_1608_04472_gb300/csrc/bc_rn.h"

#include <cstdio>
#include <random>

using namespace bcrn;

static long bad = 0, cases = 0;

static void check(const char *what, double got, double want, double a, double b) {
  ++cases;
  if (bits_of(got) != bits_of(want)) {
    if (bad < 10) std::printf("%s(%.17g, %.17g): got %.17g, IEEE %.17g\n", what, a, b, got, want);
    ++bad;
  }
}

static double make(std::mt19937_64 &g, int e_lo, int e_hi, int form) {
  const uint64_t m = form == 0 ? MANT : (form == 1 ? 0ull : (g() & MANT));
  const int e = e_lo + (int)(g() % (uint64_t)(e_hi - e_lo + 1));
  return double_of(((uint64_t)e << 52) | m);
}

int main() {
  std::mt19937_64 g(20161608);
  for (long i = 0; i < 4000000; ++i) {
    const int b = 1 + (int)(g() % 53);
    uint64_t s;
    switch (i % 6) {
      case 0: s = (1ull << (b - 1)) + (uint64_t)(i / 6) % 5; break;
      case 1: s = (b == 53 ? (1ull << 53) : (1ull << b)) - 1 - (uint64_t)(i / 6) % 5; break;
      default: s = (g() >> (64 - b)) | (1ull << (b - 1));
    }
    if (s == 0 || s >= (1ull << 53)) s = (1ull << 53) - 1;
    const int form = (int)(i % 7 < 2 ? i % 7 : 2);
    const double x = make(g, 1023, 1023 + 60, form);
    const double y = make(g, 700, 1300, form);
    const double z = make(g, 940, 1100, form);
    check("div", rn_div_u53(x, s), x / (double)s, x, (double)s);
    check("mul", rn_mul_u53(s, y), (double)s * y, (double)s, y);
    check("one_plus", rn_one_plus(z), 1.0 + z, z, 0.0);
    check("u53", rn_u53_to_double(s), (double)s, (double)s, 0.0);
  }
  // half-way products: small s times mantissas with few low bits
  for (uint64_t s = 1; s < 3000; ++s)
    for (int k = 0; k < 64; ++k) {
      const double y = double_of(((uint64_t)(1000 + k) << 52) | (g() & MANT & ~0x1FFull) | (uint64_t)(k & 3));
      check("mul", rn_mul_u53(s, y), (double)s * y, (double)s, y);
    }
  // 1 + x at exact ties: x = 2^53 (+ units), x = 2^-53 (+ units)
  for (int k = 0; k < 8; ++k) {
    check("one_plus", rn_one_plus(9007199254740992.0 + 2.0 * k), 1.0 + (9007199254740992.0 + 2.0 * k), 0, 0);
    const double t = double_of(((uint64_t)(1023 - 53) << 52) | (uint64_t)k);
    check("one_plus", rn_one_plus(t), 1.0 + t, t, 0);
  }
  check("one_plus", rn_one_plus(0.0), 1.0, 0, 0);
  check("mul", rn_mul_u53(5, 0.0), 0.0, 5, 0);
  std::printf("cases %ld mismatches %ld\n", cases, bad);
  return bad != 0 ? 1 : 0;
}
