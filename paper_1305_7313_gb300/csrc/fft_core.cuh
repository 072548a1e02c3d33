// fft_core.cuh — batched mixed-radix (2, 3, 4, 8) Stockham FFT on lines held in
// shared memory, specialised at compile time for one line length N.
//
// The 3D FFTs of the Fock apply (orbitals to real space, pair densities to G
// space and back, V_x psi back to G space; §4 of the paper computes all of
// them "via Fast Fourier Transform") are done as one pass over planes and one
// pass over columns.  Inside a pass, every CTA owns whole lines in shared
// memory and runs the Stockham autosort recursion on them:
//
//   stage (radix R, P = product of the radices of the earlier stages):
//     for every butterfly b in [0, N/R):  k = b mod P
//       x_r = in[b + r N/R] * w_N^(SIGN r k N/(PR)),   r = 0..R-1
//       y   = DFT_R(x)                                  (exp(SIGN 2 pi i r q / R))
//       out[(b - k) R + k + q P] = y_q,                 q = 0..R-1
//
// which leaves the result in natural order after the last stage.  A stage is
// done in place: each thread loads all its butterfly inputs into registers,
// the CTA synchronises, then the outputs are written back.  In float and
// double the products x_r w are not rounded on their own but folded into the
// first butterfly sums as fused multiply-adds (Dft::run_tw).
//
// Thread mapping: thread `tid` works on line (tid mod NLINES) as sub-thread
// (tid / NLINES) of TL sub-threads per line; consecutive threads therefore
// touch consecutive lines, which keeps shared-memory accesses conflict-free
// when lines are contiguous (column FFTs) or when the line stride is odd
// (row FFTs with a padded stride).  Sub-thread t owns butterflies t, t + TL, ...
// of every stage, so it holds N / TL elements between the two barriers.
//
// Twiddles come from a table w[t] = exp(-2 pi i t / N), t < N, computed on the
// host in FP64 and staged in shared memory together with its conjugate
// (tw[N + t]), which the SIGN = +1 transforms read.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "df64.cuh"

// The butterflies and their complex helpers compile for the host too, so that
// they can be checked on a CPU; the kernels use them on the device only.
#define FFT_HD __host__ __device__ __forceinline__

namespace fockx {

constexpr int kMaxStages = 8;
// The shared-memory twiddle table holds the forward table e^{-2 pi i t/N}
// (t < N) followed by its conjugate for the inverse transforms.
constexpr int kTwiddleTable = 2;
constexpr int kMaxThreads = 1024;
constexpr int kEmax = 24;  // elements a thread may hold across a stage

struct RadixPlan {
  int nst;                 // number of stages
  int r[kMaxStages];       // radices, in stage order
  int tl_plane;            // sub-threads per line, plane passes (N lines)
  int tl_colh;             // sub-threads per line, half-spectrum column pass (2(N/2+1) lines)
};

// sin and cos of 2 pi m / R for integers, evaluated at compile time from their
// Taylor series after reducing the angle to [0, pi/4] with the octant
// symmetries (exact for the multiples of pi/4).
__host__ __device__ constexpr double ct_taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double ct_taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// cos(2 pi m / R) (want_sin = false) or sin(2 pi m / R) (want_sin = true)
__host__ __device__ constexpr double ct_trig(int m, int R, bool want_sin) {
  m = ((m % R) + R) % R;
  // angle = 2 pi m / R = (pi / 4) * (8 m / R): octant o and remainder in [0, 1)
  const int num = 8 * m;
  const int o = num / R;
  const double f = (double)(num - o * R) / (double)R;  // fraction of an octant
  const double quarter_pi = 0.78539816339744830961566084581987572;
  double c = 0.0, s = 0.0;
  // angle within the octant, measured from its start (even octant) or its end (odd)
  const double y = ((o & 1) ? (1.0 - f) : f) * quarter_pi;
  const double cy = ct_taylor_cos(y), sy = ct_taylor_sin(y);
  switch (o) {  // angle = o * pi/4 + f * pi/4
    case 0: c = cy; s = sy; break;      // [0, 45)
    case 1: c = sy; s = cy; break;      // [45, 90): 90 - y
    case 2: c = -sy; s = cy; break;     // [90, 135): 90 + y
    case 3: c = -cy; s = sy; break;     // [135, 180): 180 - y
    case 4: c = -cy; s = -sy; break;    // [180, 225): 180 + y
    case 5: c = -sy; s = -cy; break;    // [225, 270): 270 - y
    case 6: c = sy; s = -cy; break;     // [270, 315): 270 + y
    default: c = cy; s = -sy; break;    // [315, 360): 360 - y
  }
  return want_sin ? s : c;
}

__host__ __device__ constexpr int cgcd(int a, int b) {
  while (b != 0) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return a;
}

__host__ __device__ constexpr int best_tl(int n, const int* r, int nst, int nlines, int maxt, int emax) {
  int g = 0;
  for (int s = 0; s < nst; ++s) g = cgcd(g, n / r[s]);
  for (int t = g; t >= 1; --t)
    if (g % t == 0 && n / t <= emax && (nlines * t + 31) / 32 * 32 <= maxt) return t;
  return 0;
}

constexpr int kRadices[8] = {16, 12, 9, 8, 6, 4, 3, 2};

// Depth-first search over radix multisets (in descending order) whose product
// is n; keeps the plan with the fewest stages, then the most threads per line.
__host__ __device__ constexpr void radix_search(int n, int rem, int first, RadixPlan& cur, RadixPlan& best,
                                                int& best_score, int maxt, int emax) {
  if (rem == 1) {
    RadixPlan p = cur;
    p.tl_plane = best_tl(n, p.r, p.nst, n, maxt, emax);
    p.tl_colh = best_tl(n, p.r, p.nst, 2 * (n / 2 + 1), maxt, emax);
    if (p.tl_plane == 0 || p.tl_colh == 0) return;
    const int score = p.nst * 4096 - p.tl_plane;
    if (score < best_score) {
      best_score = score;
      best = p;
    }
    return;
  }
  if (cur.nst >= 4) return;
  for (int k = first; k < 8; ++k) {
    const int r = kRadices[k];
    if (rem % r != 0) continue;
    cur.r[cur.nst++] = r;
    radix_search(n, rem / r, k, cur, best, best_score, maxt, emax);
    --cur.nst;
  }
}

// Fewest stages first, then the most threads per line, with CTAs of at most
// maxt threads.  Radices 6, 9, 12 and 16 are done in registers as two small
// DFTs, so a plan such as 96 = 12 x 8 needs two shared-memory stages.
__host__ __device__ constexpr RadixPlan make_radix_plan(int n, int maxt = kMaxThreads, int emax = kEmax) {
  RadixPlan best{};
  best.nst = 0;
  RadixPlan cur{};
  cur.nst = 0;
  int best_score = 1 << 30;
  radix_search(n, n, 0, cur, best, best_score, maxt, emax);
  return best;
}

// Per working type.  emax: elements a thread may hold across a stage (24 in
// FP32; 12 in FP64 and double-float, whose values take twice the registers of
// a float, so their plans use more threads per line: 96 = 12 x 4 x 2 with 8
// threads per line instead of 12 x 8 with 4).  fused: the type has a hardware
// fused multiply-add, so twiddle products are folded into the butterfly sums
// (Dft::run_tw) instead of being rounded on their own.
template <class T> struct FftTraits {
  static constexpr int emax = kEmax;
  static constexpr bool fused = true;
};

template <class T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <> struct CplxOf<df64> { using type = cdf64; };
// FP64: the 12-element plans keep twice the warps of the 24-element ones in
// flight on the FP64 pipe at the same instruction count
template <> struct FftTraits<double> {
  static constexpr int emax = 12;
  static constexpr bool fused = true;
};
template <> struct FftTraits<df64> {
  static constexpr int emax = 12;
  static constexpr bool fused = false;
};
template <class T> using cplx = typename CplxOf<T>::type;

// Elements a thread may hold across a stage for radix-plan variant EMAX (0:
// the type's own, FftTraits<T>::emax).  A plan is named by (N, MAXT, EMAX).
template <class T, int EMAX> __host__ __device__ constexpr int plan_emax() {
  return EMAX > 0 ? EMAX : FftTraits<T>::emax;
}

// S * x for S = +1 or -1 (a sign flip, never a multiplication)
template <int S, class T> FFT_HD T sgn(T x) {
  if constexpr (S > 0) return x;
  else return -x;
}
// x / 2, exact
FFT_HD float half_of(float x) { return 0.5f * x; }
FFT_HD double half_of(double x) { return 0.5 * x; }
__device__ __forceinline__ df64 half_of(df64 x) { return ldexp_pow2(x, 0.5f); }

// a * b + c with one rounding
FFT_HD float fmadd(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
FFT_HD double fmadd(double a, double b, double c) {
#ifdef __CUDA_ARCH__
  return __fma_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

template <class T>
FFT_HD cplx<T> cmake(T x, T y) {
  cplx<T> r;
  r.x = x;
  r.y = y;
  return r;
}
template <class C> FFT_HD C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <class C> FFT_HD C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <class C> FFT_HD C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// S * i * a for S = +1 or -1
template <int S, class C> FFT_HD C cmul_si(C a) {
  C r;
  r.x = S > 0 ? -a.y : a.y;
  r.y = S > 0 ? a.x : -a.x;
  return r;
}

// In-register DFTs, y_q = sum_r x_r exp(SIGN 2 pi i r q / R).
template <int SIGN, class T> struct Dft {
  using C = cplx<T>;
  static FFT_HD void r2(C* x) {
    C a = x[0];
    x[0] = cadd(a, x[1]);
    x[1] = csub(a, x[1]);
  }
  static FFT_HD void r3(C* x) { r3_sd(x, cadd(x[1], x[2]), csub(x[1], x[2])); }
  // the length-3 DFT from x0, s = x1 + x2 and d = x1 - x2
  static FFT_HD void r3_sd(C* x, C s, C d) {
    constexpr T h0 = T(0.86602540378443864676372317075293618);  // sin(2 pi / 3)
    const T h = sgn<SIGN>(h0);
    C m = cmake<T>(x[0].x - half_of(s.x), x[0].y - half_of(s.y));
    C u = cmake<T>(-h * d.y, h * d.x);
    x[0] = cadd(x[0], s);
    x[1] = cadd(m, u);
    x[2] = csub(m, u);
  }
  static FFT_HD void r4v(C& x0, C& x1, C& x2, C& x3) {
    C a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = cmul_si<SIGN>(csub(x1, x3));
    x0 = cadd(a, c);
    x2 = csub(a, c);
    x1 = cadd(b, d);
    x3 = csub(b, d);
  }
  static FFT_HD void r4(C* x) { r4v(x[0], x[1], x[2], x[3]); }
  static FFT_HD void r8(C* x) {
    constexpr T c = T(0.70710678118654752440084436210484904);  // cos(pi / 4)
    C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    r4v(e0, e1, e2, e3);
    r4v(o0, o1, o2, o3);
    // o_q *= exp(SIGN 2 pi i q / 8)
    C t1 = cmake<T>(c * (o1.x - sgn<SIGN>(o1.y)), c * (o1.y + sgn<SIGN>(o1.x)));
    C t2 = cmul_si<SIGN>(o2);
    C t3 = cmake<T>(-(c * (o3.x + sgn<SIGN>(o3.y))), c * (sgn<SIGN>(o3.x) - o3.y));
    x[0] = cadd(e0, o0);
    x[4] = csub(e0, o0);
    x[1] = cadd(e1, t1);
    x[5] = csub(e1, t1);
    x[2] = cadd(e2, t2);
    x[6] = csub(e2, t2);
    x[3] = cadd(e3, t3);
    x[7] = csub(e3, t3);
  }
  // x *= exp(SIGN 2 pi i M / R) with compile-time M, R (exact for the quarter turns)
  template <int M, int R> static FFT_HD C twiddle(C x) {
    constexpr int m = ((M % R) + R) % R;
    if constexpr (m == 0) {
      return x;
    } else if constexpr (4 * m == R) {
      return cmul_si<SIGN>(x);
    } else if constexpr (2 * m == R) {
      return cmake<T>(-x.x, -x.y);
    } else if constexpr (4 * m == 3 * R) {
      return cmul_si<-SIGN>(x);
    } else {
      constexpr T c = T(ct_trig(m, R, false));
      constexpr T s = T(SIGN * ct_trig(m, R, true));
      return cmake<T>(c * x.x - s * x.y, c * x.y + s * x.x);
    }
  }
  // ---- twiddled inputs, for types with a fused multiply-add (FftTraits::fused).
  // DFT of (x_0, w_1 x_1, ..., w_{R-1} x_{R-1}): each twiddle product is folded
  // into the first sum it feeds (a + w x as two fused multiply-adds per
  // component), and the matching difference is taken as 2 a - (a + w x), which
  // saves the separate rounding of w x and a quarter of the instructions of the
  // twiddled sums.
  // a + w x
  static FFT_HD C cfma(C a, C w, C x) {
    return cmake<T>(fmadd(w.x, x.x, fmadd(-w.y, x.y, a.x)), fmadd(w.x, x.y, fmadd(w.y, x.x, a.y)));
  }
  // 2 a - b
  static FFT_HD C ctwice_sub(C a, C b) {
    return cmake<T>(fmadd(T(2), a.x, -b.x), fmadd(T(2), a.y, -b.y));
  }
  // a - 2 b
  static FFT_HD C csub_twice(C a, C b) {
    return cmake<T>(fmadd(T(-2), b.x, a.x), fmadd(T(-2), b.y, a.y));
  }
  static FFT_HD void r2_tw(C& x0, C& x1, C w1) {
    const C a = cfma(x0, w1, x1);
    x1 = ctwice_sub(x0, a);
    x0 = a;
  }
  static FFT_HD void r3_tw(C* x, C w1, C w2) {
    const C x1w = cmul(x[1], w1);
    const C s = cfma(x1w, w2, x[2]);  // w1 x1 + w2 x2
    r3_sd(x, s, ctwice_sub(x1w, s));
  }
  static FFT_HD void r4v_tw(C& x0, C& x1, C& x2, C& x3, C w1, C w2, C w3) {
    const C a = cfma(x0, w2, x2);      // x0 + w2 x2
    const C b = ctwice_sub(x0, a);     // x0 - w2 x2
    const C x3w = cmul(x3, w3);
    const C c = cfma(x3w, w1, x1);     // w1 x1 + w3 x3
    const C d = cmul_si<SIGN>(csub_twice(c, x3w));  // S i (w1 x1 - w3 x3)
    x0 = cadd(a, c);
    x2 = csub(a, c);
    x1 = cadd(b, d);
    x3 = csub(b, d);
  }
  static FFT_HD void r8_tw(C* x, const C* w) {
    constexpr T c = T(0.70710678118654752440084436210484904);  // cos(pi / 4)
    C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    C o0 = cmul(x[1], w[1]), o1 = x[3], o2 = x[5], o3 = x[7];
    r4v_tw(e0, e1, e2, e3, w[2], w[4], w[6]);
    r4v_tw(o0, o1, o2, o3, w[3], w[5], w[7]);
    // x_q = e_q +- exp(SIGN 2 pi i q / 8) o_q, the pi/4 rotations as c * p
    const C p = cmake<T>(o1.x - sgn<SIGN>(o1.y), o1.y + sgn<SIGN>(o1.x));
    const C q = cmake<T>(o3.x + sgn<SIGN>(o3.y), sgn<SIGN>(o3.x) - o3.y);
    const C t2 = cmul_si<SIGN>(o2);
    x[0] = cadd(e0, o0);
    x[4] = csub(e0, o0);
    x[1] = cmake<T>(fmadd(c, p.x, e1.x), fmadd(c, p.y, e1.y));
    x[5] = cmake<T>(fmadd(-c, p.x, e1.x), fmadd(-c, p.y, e1.y));
    x[2] = cadd(e2, t2);
    x[6] = csub(e2, t2);
    x[3] = cmake<T>(fmadd(-c, q.x, e3.x), fmadd(c, q.y, e3.y));
    x[7] = cmake<T>(fmadd(c, q.x, e3.x), fmadd(-c, q.y, e3.y));
  }
  // W0: x_0 carries a twiddle w_0 too
  template <int R, bool W0> static FFT_HD void run_tw(C* x, const C* w) {
    if constexpr (W0) x[0] = cmul(x[0], w[0]);
    if constexpr (R == 2) r2_tw(x[0], x[1], w[1]);
    else if constexpr (R == 3) r3_tw(x, w[1], w[2]);
    else if constexpr (R == 4) r4v_tw(x[0], x[1], x[2], x[3], w[1], w[2], w[3]);
    else if constexpr (R == 8) r8_tw(x, w);
    else if constexpr (R == 6) composite<2, 3, true>(x, w);
    else if constexpr (R == 9) composite<3, 3, true>(x, w);
    else if constexpr (R == 12) composite<4, 3, true>(x, w);
    else composite<4, 4, true>(x, w);  // R == 16
  }

  // w_R^m is a quarter turn (a sign change or a swap, no arithmetic)
  static __host__ __device__ constexpr bool quarter_turn(int m, int R) { return (4 * (((m % R) + R) % R)) % R == 0; }
  // every twiddle w_R^(n2 k1), 0 < n2 < R2, needs arithmetic
  template <int R2, int R> static __host__ __device__ constexpr bool all_general(int k1) {
    for (int n2 = 1; n2 < R2; ++n2)
      if (quarter_turn(n2 * k1, R)) return false;
    return true;
  }

  // R = R1 R2 in registers: R2 DFTs of length R1 over x[R2 n1 + n2] (TW: with
  // the stage twiddles w[R2 n1 + n2] on their inputs), twiddle w_R^(n2 k1),
  // R1 DFTs of length R2; output k = k1 + R1 k2.
  template <int R1, int R2, bool TW, int N2 = 0>
  static FFT_HD void inner(C* x, const C* w, C* a) {
    if constexpr (N2 < R2) {
      C t[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) t[n1] = x[R2 * n1 + N2];
      if constexpr (TW) {
        C wt[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) wt[n1] = w[R2 * n1 + N2];
        run_tw<R1, (N2 > 0)>(t, wt);
      } else {
        run<R1>(t);
      }
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) a[N2 * R1 + k1] = t[k1];
      inner<R1, R2, TW, N2 + 1>(x, w, a);
    }
  }
  template <int R1, int R2, int K1 = 0>
  static FFT_HD void outer(const C* a, C* x) {
    if constexpr (K1 < R1) {
      C t[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) t[n2] = a[n2 * R1 + K1];
      if constexpr (FftTraits<T>::fused && K1 > 0 && all_general<R2, R1 * R2>(K1)) {
        C wc[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2)
          wc[n2] = cmake<T>(T(ct_trig(n2 * K1, R1 * R2, false)), T(SIGN * ct_trig(n2 * K1, R1 * R2, true)));
        run_tw<R2, false>(t, wc);
      } else {
        twiddle_col<R1, R2, K1, 1>(t);
        run<R2>(t);
      }
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) x[K1 + R1 * k2] = t[k2];
      outer<R1, R2, K1 + 1>(a, x);
    }
  }
  template <int R1, int R2, int K1, int N2>
  static FFT_HD void twiddle_col(C* t) {
    if constexpr (N2 < R2) {
      t[N2] = twiddle<N2 * K1, R1 * R2>(t[N2]);
      twiddle_col<R1, R2, K1, N2 + 1>(t);
    }
  }
  template <int R1, int R2, bool TW = false>
  static FFT_HD void composite(C* x, const C* w = nullptr) {
    C a[R1 * R2];
    inner<R1, R2, TW>(x, w, a);
    outer<R1, R2>(a, x);
  }
  template <int R> static FFT_HD void run(C* x) {
    if constexpr (R == 2) r2(x);
    else if constexpr (R == 3) r3(x);
    else if constexpr (R == 4) r4(x);
    else if constexpr (R == 8) r8(x);
    else if constexpr (R == 6) composite<2, 3>(x);
    else if constexpr (R == 9) composite<3, 3>(x);
    else if constexpr (R == 12) composite<4, 3>(x);
    else composite<4, 4>(x);  // R == 16
  }
};

// Position of output element k of a line in shared memory: OMAP 0 natural
// order; OMAP 1 "quad phases": the line is stored as four runs of N/4, run
// k mod 4 holding elements k mod 4, k mod 4 + 4, ... (so that element 4c + u
// sits at u N/4 + c).  Only the last stage of a transform applies a map.
template <int N, int OMAP> FFT_HD constexpr int out_pos(int k) {
  if constexpr (OMAP == 1) return (k & 3) * (N / 4) + (k >> 2);
  else return k;
}

// One Stockham stage on one line (base, element stride ES) for sub-thread t of TL.
template <class T, int N, int R, int P, int TL, int ES, int SIGN, int OMAP = 0>
__device__ __forceinline__ void fft_stage(cplx<T>* base, int t, bool active, const cplx<T>* tw) {
  using C = cplx<T>;
  constexpr int NB = N / R;
  constexpr int PER = NB / TL;
  constexpr int TWS = N / (P * R);
  const C* twt = SIGN > 0 ? tw + N : tw;  // the conjugate table for inverse transforms
  C x[PER][R];
  if (active) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int b = t + TL * k;
#pragma unroll
      for (int r = 0; r < R; ++r) x[k][r] = base[(b + r * NB) * ES];
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int b = t + TL * k;
      const int kk = b % P;
      if constexpr (P > 1 && FftTraits<T>::fused) {
        C w[R];
#pragma unroll
        for (int r = 1; r < R; ++r) w[r] = twt[r * kk * TWS];
        w[0] = w[1];  // not read: x_0 carries no twiddle
        Dft<SIGN, T>::template run_tw<R, false>(x[k], w);
      } else {
        if constexpr (P > 1) {
#pragma unroll
          for (int r = 1; r < R; ++r) x[k][r] = cmul(x[k][r], twt[r * kk * TWS]);
        }
        Dft<SIGN, T>::template run<R>(x[k]);
      }
      const int j = (b - kk) * R + kk;
#pragma unroll
      for (int q = 0; q < R; ++q) base[out_pos<N, OMAP>(j + q * P) * ES] = x[k][q];
    }
  }
  __syncthreads();
}

// The first stage (P = 1, no twiddles) with its inputs taken from a loader
// (element m of line `line`: load(line, m)) instead of shared memory: the
// caller's data never pass through shared memory before the transform.
template <class T, int N, int R, int TL, int ES, int SIGN, class Load>
__device__ __forceinline__ void fft_stage_first(cplx<T>* base, int t, bool active, int line, const Load& load) {
  using C = cplx<T>;
  constexpr int NB = N / R;
  constexpr int PER = NB / TL;
  C x[PER][R];
  if (active) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int b = t + TL * k;
#pragma unroll
      for (int r = 0; r < R; ++r) x[k][r] = load(line, b + r * NB);
    }
  }
  if (active) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int b = t + TL * k;
      Dft<SIGN, T>::template run<R>(x[k]);
#pragma unroll
      for (int q = 0; q < R; ++q) base[(b * R + q) * ES] = x[k][q];
    }
  }
  __syncthreads();
}

template <class T, int N, int SIGN, int TL, int ES, int S, int P, int MAXT, int EMAX = 0, int OMAP = 0>
__device__ __forceinline__ void fft_stages(cplx<T>* base, int t, bool active, const cplx<T>* tw) {
  constexpr RadixPlan pl = make_radix_plan(N, MAXT, plan_emax<T, EMAX>());
  if constexpr (S < pl.nst) {
    constexpr int R = pl.r[S];
    fft_stage<T, N, R, P, TL, ES, SIGN, (S + 1 == pl.nst) ? OMAP : 0>(base, t, active, tw);
    fft_stages<T, N, SIGN, TL, ES, S + 1, P * R, MAXT, EMAX, OMAP>(base, t, active, tw);
  }
}

// FFT of NLINES lines of length N whose input comes from load(line, m) and
// whose output lands in shared memory (line l at buf + l*LS, stride ES).
template <class T, int N, int SIGN, int NLINES, int TL, int LS, int ES, int MAXT, int EMAX = 0, class Load>
__device__ __forceinline__ void fft_lines_from(cplx<T>* buf, const cplx<T>* tw, const Load& load) {
  constexpr RadixPlan pl = make_radix_plan(N, MAXT, plan_emax<T, EMAX>());
  constexpr int R0 = pl.r[0];
  const int tid = threadIdx.x;
  const int line = tid % NLINES;
  const int t = tid / NLINES;
  const bool active = t < TL;
  fft_stage_first<T, N, R0, TL, ES, SIGN>(buf + line * LS, t, active, line, load);
  fft_stages<T, N, SIGN, TL, ES, 1, R0, MAXT, EMAX>(buf + line * LS, t, active, tw);
}

// FFT of `nlines` lines (a run-time count) whose input comes from
// load(line, m) and whose output lands in shared memory at buf + off(line)
// (elements ES apart).  Consecutive threads take consecutive lines, as in
// fft_lines_from; threads beyond nlines * TL idle, so whole warps drop out when
// fewer lines are transformed.
template <class T, int N, int SIGN, int TL, int ES, int MAXT, int EMAX = 0, class Load, class Off>
__device__ __forceinline__ void fft_lines_from_rt(cplx<T>* buf, const cplx<T>* tw, int nlines, const Load& load,
                                                  const Off& off) {
  constexpr RadixPlan pl = make_radix_plan(N, MAXT, plan_emax<T, EMAX>());
  constexpr int R0 = pl.r[0];
  const int tid = threadIdx.x;
  const int line = tid % nlines;
  const int t = tid / nlines;
  const bool active = t < TL;
  cplx<T>* base = buf + off(line);
  fft_stage_first<T, N, R0, TL, ES, SIGN>(base, t, active, line, load);
  fft_stages<T, N, SIGN, TL, ES, 1, R0, MAXT, EMAX>(base, t, active, tw);
}

// FFT in place of `nlines` lines (a run-time count) in shared memory, line l
// at buf + off(l), elements ES apart; as fft_lines otherwise.
template <class T, int N, int SIGN, int TL, int ES, int MAXT, int EMAX = 0, class Off>
__device__ __forceinline__ void fft_lines_rt(cplx<T>* buf, const cplx<T>* tw, int nlines, const Off& off) {
  const int tid = threadIdx.x;
  const int line = tid % nlines;
  const int t = tid / nlines;
  const bool active = t < TL;
  fft_stages<T, N, SIGN, TL, ES, 0, 1, MAXT, EMAX>(buf + off(line), t, active, tw);
}

// FFT of NLINES lines of length N in shared memory: line l starts at buf + l*LS,
// its elements are ES apart.  Every thread of the CTA must call this (it
// synchronises); threads with tid >= NLINES*TL idle.
// MAXT and EMAX name the radix plan (make_radix_plan(N, MAXT, plan_emax<T,
// EMAX>())) that TL was chosen for.
// OMAP: the order the last stage leaves the elements of a line in (out_pos).
template <class T, int N, int SIGN, int NLINES, int TL, int LS, int ES, int MAXT = kMaxThreads, int EMAX = 0,
          int OMAP = 0>
__device__ __forceinline__ void fft_lines(cplx<T>* buf, const cplx<T>* tw) {
  const int tid = threadIdx.x;
  const int line = tid % NLINES;
  const int t = tid / NLINES;
  const bool active = t < TL;
  fft_stages<T, N, SIGN, TL, ES, 0, 1, MAXT, EMAX, OMAP>(buf + line * LS, t, active, tw);
}

}  // namespace fockx
