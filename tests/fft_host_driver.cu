// Host check of the in-register DFTs of fft_core.cuh.  For every radix R, sign
// and real type it prints seeded inputs x_r, twiddles w_r and the butterfly's
// outputs y_q, one case per line:
//   <type 0 float | 1 double> <R> <SIGN> <mode> then R values each of x, w, y
//   (real and imaginary parts)
// mode 0: Dft::run (y = DFT of x), 1: Dft::run_tw<R, false> (DFT of x_0,
// w_1 x_1, ..., w_{R-1} x_{R-1}), 2: Dft::run_tw<R, true> (w_0 x_0 as well).
// The DFT is y_q = sum_r x_r exp(SIGN 2 pi i r q / R); the test recomputes it.
//
// With the argument "plans" it prints instead the radix plan make_radix_plan
// picks for every compiled grid size and (CTA size limit, elements per thread)
// pair the kernels use:
//   plan <N> <maxt> <emax> <stages> <radix 0..3, 0: none> <tl_plane> <tl_colh>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "fft_core.cuh"

using namespace fockx;

namespace {

uint64_t g_state = 0x9e3779b97f4a7c15ull;

// uniform in [-1, 1) from a 64-bit linear congruential generator (Knuth's MMIX constants)
double uniform() {
  g_state = g_state * 6364136223846793005ull + 1442695040888963407ull;
  return (double)(g_state >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

template <class T> void put(T v) { std::printf(" %.17g", (double)v); }

template <class T, int SIGN, int R, int MODE>
void one_case() {
  using C = cplx<T>;
  using D = Dft<SIGN, T>;
  C x[R], w[R], y[R];
  for (int r = 0; r < R; ++r) {
    x[r] = cmake<T>((T)uniform(), (T)uniform());
    const double a = 3.14159265358979323846 * uniform();  // a unit twiddle
    w[r] = cmake<T>((T)std::cos(a), (T)std::sin(a));
    y[r] = x[r];
  }
  if constexpr (MODE == 0) D::template run<R>(y);
  else D::template run_tw<R, MODE == 2>(y, w);
  std::printf("%d %d %d %d", sizeof(T) == 8 ? 1 : 0, R, SIGN, MODE);
  for (int r = 0; r < R; ++r) { put(x[r].x); put(x[r].y); }
  for (int r = 0; r < R; ++r) { put(w[r].x); put(w[r].y); }
  for (int r = 0; r < R; ++r) { put(y[r].x); put(y[r].y); }
  std::printf("\n");
}

template <class T, int SIGN, int R>
void cases() {
  for (int rep = 0; rep < 3; ++rep) {
    one_case<T, SIGN, R, 0>();
    one_case<T, SIGN, R, 1>();
    one_case<T, SIGN, R, 2>();
  }
}

template <class T, int SIGN>
void all_radices() {
  cases<T, SIGN, 2>();
  cases<T, SIGN, 3>();
  cases<T, SIGN, 4>();
  cases<T, SIGN, 6>();
  cases<T, SIGN, 8>();
  cases<T, SIGN, 9>();
  cases<T, SIGN, 12>();
  cases<T, SIGN, 16>();
}

// evaluated at compile time, as the kernels do
template <int N, int MAXT, int EMAX>
void plan_line() {
  constexpr RadixPlan p = make_radix_plan(N, MAXT, EMAX);
  std::printf("plan %d %d %d %d", N, MAXT, EMAX, p.nst);
  for (int s = 0; s < 4; ++s) std::printf(" %d", s < p.nst ? p.r[s] : 0);
  std::printf(" %d %d\n", p.tl_plane, p.tl_colh);
}

template <int N>
void plan_lines() {
  plan_line<N, kMaxThreads, 24>();
  plan_line<N, kMaxThreads, 12>();
  plan_line<N, 416, 24>();
  plan_line<N, 800, 12>();
}

void plans() {
  plan_lines<8>();
  plan_lines<12>();
  plan_lines<16>();
  plan_lines<24>();
  plan_lines<32>();
  plan_lines<36>();
  plan_lines<48>();
  plan_lines<64>();
  plan_lines<72>();
  plan_lines<96>();
}

}  // namespace

int main(int argc, char** argv) {
  if (argc > 1 && std::strcmp(argv[1], "plans") == 0) {
    plans();
    return 0;
  }
  all_radices<float, -1>();
  all_radices<float, +1>();
  all_radices<double, -1>();
  all_radices<double, +1>();
  return 0;
}
