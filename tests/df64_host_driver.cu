// Host check of the double-float arithmetic of df64.cuh.  Prints, as exact
// hexadecimal floats, one case per line:
//   split <d> <hi> <lo>                   df64(d) of a double d
//   add|sub|mul <ahi> <alo> <bhi> <blo> <rhi> <rlo>
//   scale <ahi> <alo> <p2> <rhi> <rlo>    ldexp_pow2(a, p2)
//   conv <f> <d>                          float_bits_to_double(f)
// The test recomputes every result in exact rational arithmetic.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "df64.cuh"

using namespace fockx;

namespace {

uint64_t g_state = 0x2545f4914f6cdd1dull;

// uniform in [0, 1) from a 64-bit linear congruential generator (Knuth's MMIX constants)
double uniform() {
  g_state = g_state * 6364136223846793005ull + 1442695040888963407ull;
  return (double)(g_state >> 11) * (1.0 / 9007199254740992.0);
}

// a signed value of magnitude 2^e, e uniform in [-emax, emax], with 53 random bits
double value(int emax) {
  const double m = 1.0 + uniform();
  const int e = (int)std::floor(uniform() * (2 * emax + 1)) - emax;
  return (uniform() < 0.5 ? -1.0 : 1.0) * std::ldexp(m, e);
}

void put(df64 a) { std::printf(" %a %a", (double)a.hi, (double)a.lo); }

}  // namespace

int main() {
  for (int i = 0; i < 2000; ++i) {
    const double d = value(30);
    const df64 s(d);
    std::printf("split %a %a %a\n", d, (double)s.hi, (double)s.lo);
  }
  for (int i = 0; i < 4000; ++i) {
    // operands of similar and of very different magnitudes, and near-cancellation
    const int emax = i % 3 == 0 ? 2 : 20;
    const df64 a(value(emax));
    df64 b(value(emax));
    if (i % 7 == 0) b = df64(-(double)a.hi - (double)a.lo * (1.0 + 0x1p-20), 0.0f) + df64(value(1) * 0x1p-40);
    std::printf("add");
    put(a);
    put(b);
    put(a + b);
    std::printf("\nsub");
    put(a);
    put(b);
    put(a - b);
    std::printf("\nmul");
    put(a);
    put(b);
    put(a * b);
    std::printf("\n");
  }
  for (int i = 0; i < 200; ++i) {
    const df64 a(value(20));
    const float p2 = std::ldexp(1.0f, (int)std::floor(uniform() * 21) - 10);
    std::printf("scale");
    put(a);
    std::printf(" %a", (double)p2);
    put(ldexp_pow2(a, p2));
    std::printf("\n");
  }
  const float special[] = {0.0f, -0.0f, FLT_MIN, -FLT_MIN, FLT_MAX, -FLT_MAX, 1.0f, -1.5f, 0x1p-127f, -0x1p-140f,
                           0x1.fffffep-1f, 3.14159265f, 1e-30f, -7e20f};
  for (float f : special) std::printf("conv %a %a\n", (double)f, float_bits_to_double(f));
  for (int i = 0; i < 500; ++i) {
    const float f = (float)value(100);
    std::printf("conv %a %a\n", (double)f, float_bits_to_double(f));
  }
  return 0;
}
