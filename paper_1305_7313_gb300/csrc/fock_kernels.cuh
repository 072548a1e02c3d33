// fock_kernels.cuh — the CUDA kernels of the Gamma-point Fock apply, templated
// on the working real type T (double: FP64 form; float: mixed form; df64:
// double-float form, FP64-class accuracy on the FP32 pipe).
//
// Data layout in HBM (all row-major, last index fastest):
//   psi  [nb][N][N][N]  real T      orbitals in real space, psi(r) of §4
//   W    [nb][N][N][N]  real A      accumulators of V_x psi_j(r) (A = T, or
//                                   double for df64)
//   H    [chain][N][N][2][N/2+1]    complex T: per plane i1 and row k2, the
//        stored half (k3 <= N/2) of the 2D transforms of the two pair densities
//        of a chain (index 0: pair a, 1: pair b)
//   X    [q][N][N][N]   complex T   full grids for the O(nb) transforms
//
// Hot path per chain of two pairs (a = (ai, aj), b = (bi, bj)):
//   pair_fwd  (plane i1):  z = psi_ai psi_aj + i psi_bi psi_bj, 2D FFT over
//             (i2, i3) (columns first; the first stage forms z from the orbital
//             planes in global memory), split z = A + iB by Hermitian symmetry
//             (A, B are the transforms of real planes), store the kept columns
//             of the k3 <= N/2 half of A and B.
//   Every pass reads the first stage of its first transform straight from
//   global memory (fft_lines_from), so no input is staged in shared memory
//   (the double-float inverse pass stages its plane with cp.async instead).
//   pair_col  (NC columns): FFT along i1 of the stored columns a pair density
//             reaches (DevPlan::colmap: NC = 2 (N/2+1) lines per CTA), energy partials
//             sum w(k3) v |A|^2 and sum w(k3) v |B|^2 (w = 1 on the k3 = 0, N/2
//             planes, 2 elsewhere: the k3 > N/2 half is the mirror image), times
//             v/Ntot, inverse FFT along k1.
//   pair_inv  (plane i1):  inverse FFT along k2 of the stored half plane (A and B
//             columns), rebuild each row z = A + iB over all k3 (the k3 > N/2
//             half from the conjugates), inverse FFT along k3 -> phi_a + i phi_b, then
//             W_aj -= f_ai psi_ai phi_a, W_ai -= f_aj psi_aj phi_a (i != j), same for b.
#pragma once

#include "fft_core.cuh"
#include "fock_internal.h"

namespace fockx {

__device__ __forceinline__ int freq_of(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

// Rounds of global loads each thread issues before storing them to shared
// memory in the pass prologues (memory-level parallelism).
constexpr int kLoadUnroll = 4;

// Per working type: the precision code of the plan (0 FP64, 1 mixed FP32,
// 2 double-float) and the type of the accumulators W.
template <class T> struct RealTraits;
template <> struct RealTraits<double> { static constexpr int prec = 0; using acc = double; };
template <> struct RealTraits<float> { static constexpr int prec = 1; using acc = float; };
template <> struct RealTraits<df64> { static constexpr int prec = 2; using acc = double; };
template <class T> using acc_t = typename RealTraits<T>::acc;

// Load through L2 only (ld.global.cg) of one complex value.
template <class C> __device__ __forceinline__ C ldcg_c(const C* p) { return __ldcg(p); }
template <> __device__ __forceinline__ cdf64 ldcg_c<cdf64>(const cdf64* p) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  cdf64 r;
  r.x = df64(v.x, v.y);
  r.y = df64(v.z, v.w);
  return r;
}

// L2 eviction priorities (createpolicy): evict_first for data read for the last
// time (the transform buffer in the inverse pass), evict_last for data the next
// chains of a band block read again (orbital and accumulator planes).
__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_policy_evict_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// ld.global.cg of one complex value with an L2 eviction policy.
template <class C> __device__ __forceinline__ C ldcg_hint(const C* p, unsigned long long pol);
template <> __device__ __forceinline__ float2 ldcg_hint<float2>(const float2* p, unsigned long long pol) {
  float2 v;
  asm volatile("ld.global.cg.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
  return v;
}
template <> __device__ __forceinline__ double2 ldcg_hint<double2>(const double2* p, unsigned long long pol) {
  double2 v;
  asm volatile("ld.global.cg.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}
// Four floats with an L2 eviction policy (16-byte aligned).
__device__ __forceinline__ float4 ld_f4_hint(const float* p, unsigned long long pol) {
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

template <class T> __device__ __forceinline__ void atomic_add_real(T* p, T v) { atomicAdd(p, v); }
// df64 into an FP64 accumulator: both parts become doubles by integer
// instructions, one FP64 add joins them (exact to the rounding of that add).
__device__ __forceinline__ void atomic_add_real(double* p, df64 v) {
  atomicAdd(p, float_bits_to_double(v.hi) + float_bits_to_double(v.lo));
}

// Sum of four doubles over the CTA; the result is valid in thread 0.
__device__ inline void block_sum4(double v[4], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) red[warp * 4 + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w * 4 + k];
      v[k] = s;
    }
  }
}

// CTA sum of four double-float values in double-float arithmetic (warp
// shuffles of both parts, then warp 0 over the per-warp sums): no FP64
// instruction.  The result is valid in thread 0.  red: 2 * 4 * 32 floats.
__device__ inline void block_sum4_df(df64 v[4], float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_down_sync(0xffffffffu, v[k].hi, o);
      const float l2 = __shfl_down_sync(0xffffffffu, v[k].lo, o);
      v[k] += df64(h2, l2);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      red[(warp * 4 + k) * 2] = v[k].hi;
      red[(warp * 4 + k) * 2 + 1] = v[k].lo;
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = lane < nw ? df64(red[(lane * 4 + k) * 2], red[(lane * 4 + k) * 2 + 1]) : df64(0.f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, v[k].hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, v[k].lo, o);
        v[k] += df64(h2, l2);
      }
    }
  }
}

// Shared memory of one SM on sm_103 (228 KB; each resident CTA also reserves 1 KB).
constexpr size_t kSmemPerSM = 233472;

// Compile-time geometry of the passes for grid size N and radix-plan variant
// EMAX (elements a thread holds across a stage; 0: the type's own).
template <class T, int N, int MAXT = kMaxThreads, int EMAX = 0>
struct Geo {
  using C = cplx<T>;
  static constexpr RadixPlan pl = make_radix_plan(N, MAXT, plan_emax<T, EMAX>());
  static_assert(pl.nst > 0, "grid size must be 2^a 3^b and fit the FFT kernels");
  static constexpr int KH = N / 2 + 1;                    // stored half of the last axis
  static constexpr int NC = 2 * KH;                       // stored columns per row (A and B)
  static constexpr int RP = (N % 2 == 0) ? N + 1 : N;     // odd padded row stride of a plane
  static constexpr int TLP = pl.tl_plane;
  static constexpr int TLC = pl.tl_colh;
  // CTA sizes rounded up to whole warps (the extra threads idle in the FFT
  // stages), so warp shuffles always see 32 live lanes
  static constexpr int THR_PLANE = (N * TLP + 31) / 32 * 32;
  // NC lines at the column tiling: the inverse plane pass's CTA (its k2
  // transform of up to NC stored columns); the column pass sizes its own below
  static constexpr int THR_COLH = (NC * TLC + 31) / 32 * 32;
  static constexpr int THR_COLF = (N * TLP + 31) / 32 * 32;
  // lines per CTA of the column pass: the NC columns of a row's width, or
  // about half as many, rounded up to 8 lines (whole warps at 4 and 8 threads
  // a line), where two CTAs of that width do not fit the SM's shared memory
  // (FP64 and double-float at N = 96: 153 KB each; halved, two share an SM)
  // and in FP32 from N = 96 (four CTAs of 46 KB an SM instead of two of 78
  // KB): more CTAs an SM, so that the barriers of one overlap the arithmetic
  // of the others
  static constexpr int NLC_HALF = (KH + 7) / 8 * 8;
  static constexpr bool COL_SPLIT =
      (2 * (sizeof(C) * (size_t)(N * NC + kTwiddleTable * N) + 32 * 4 * sizeof(double) + NC * sizeof(int) + 1024) >
           kSmemPerSM ||
       (sizeof(C) == 8 && N >= 96)) &&
      NLC_HALF < NC;
  static constexpr int NLC = COL_SPLIT ? NLC_HALF : NC;
  static constexpr int THR_COL = (NLC * TLC + 31) / 32 * 32;
  static_assert(THR_PLANE <= 1024 && THR_COLH <= 1024, "CTA too large");
  // CTAs per SM the column and inverse passes are register-budgeted for
  // (shared memory allows two in FP32 up to N = 96, one in FP64): two when two
  // CTAs of 72 registers a thread fit the register file
  static constexpr int MIN_CTAS = (sizeof(T) == 4 && 2 * 72 * THR_COLH <= 65536) ? 2 : 1;
  // CTAs per SM the column pass is register-budgeted for where its CTAs take
  // half a row's width of lines: in FP32 as many as fit at 72 registers a
  // thread; in FP64 and double-float two above 256 threads (72 registers), and
  // no bound below (two 224-thread CTAs fit the 142 registers FP64 takes)
  static constexpr int MIN_CTAS_COL =
      NLC < NC ? (sizeof(C) == 8 ? 65536 / (72 * THR_COL) : (THR_COL > 256 ? 2 : MIN_CTAS)) : MIN_CTAS;
  // CTAs per SM the k-point inverse plane pass is register-budgeted for: in
  // FP32, eight where eight CTAs of 40 registers a thread fit the register file
  // (its shared memory allows that many up to N = 48); 0 leaves the choice to
  // the compiler, as a bound without a minimum does (a minimum of 1 changes
  // its register allocation: 89 instead of 78 registers at 96^3 in FP32)
  static constexpr int MIN_CTAS_KINV = (sizeof(T) == 4 && 8 * 40 * THR_PLANE <= 65536) ? 8 : 0;
  // twiddle table in shared memory: e^{-2 pi i t/N} and its conjugate (2N values)
  static constexpr int TWN = kTwiddleTable * N;
  static constexpr size_t SMEM_PLANE = sizeof(C) * (size_t)(N * RP + TWN);
  static constexpr size_t SMEM_COLH =
      sizeof(C) * (size_t)(N * NLC + TWN) + 32 * 4 * sizeof(double) + NLC * sizeof(int);
  static constexpr size_t SMEM_COLF = sizeof(C) * (size_t)(N * N + TWN);
  // inverse plane pass: the stored half plane with an odd row stride NC + 1,
  // the twiddles and the column map's row lengths
  static constexpr int NCP = NC + 1;
  static constexpr size_t SMEM_INV = sizeof(C) * (size_t)(N * NCP + TWN) + N * sizeof(int);
};

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += (h2, l2) in float-float arithmetic (about 48 significant bits).
__device__ __forceinline__ void ff_add(float& hi, float& lo, float h2, float l2) {
  float s, e;
  two_sum(hi, h2, s, e);
  e += lo + l2;
  hi = s + e;
  lo = e - (hi - s);
}

// CTA sum of four float partials in float-float arithmetic across threads and
// warps; thread 0 receives (hi, lo) per value.  Uses no FP64 instruction, so
// the FP64 pipe stays out of the FP32 kernels.  red: 2 * 4 * 32 floats.
__device__ inline void block_sum4_ff(const float v[4], float hi[4], float lo[4], float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    hi[k] = v[k];
    lo[k] = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_down_sync(0xffffffffu, hi[k], o);
      const float l2 = __shfl_down_sync(0xffffffffu, lo[k], o);
      ff_add(hi[k], lo[k], h2, l2);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      red[(warp * 4 + k) * 2] = hi[k];
      red[(warp * 4 + k) * 2 + 1] = lo[k];
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      hi[k] = lane < nw ? red[(lane * 4 + k) * 2] : 0.f;
      lo[k] = lane < nw ? red[(lane * 4 + k) * 2 + 1] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi[k], o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo[k], o);
        ff_add(hi[k], lo[k], h2, l2);
      }
    }
  }
}

// One kernel term of the smallest |m| (|m|^2 <= msmall2: 27 points per pair)
// of the mixed-form column pass, in FP64: element e of the CTA's lines, at
// (k1, k2, k3) of pair s.  Adds its energy terms to the pair slot itself.
// Kept out of line so the FP64 instructions are not predicated into every
// warp of the kernel.
template <class T, int N>
__device__ __noinline__ void small_g_term_fp64(const DevPlan& g, cplx<T>* S, int e, int k1, int k2, int k3,
                                               int s, const Chain& ch, double* epair, double* dpair) {
  constexpr int KH = N / 2 + 1;
  const int64_t vi = ((int64_t)k1 * N + k2) * KH + k3;
  const double wgt = (k3 == 0 || 2 * k3 == N) ? 1.0 : 2.0;
  cplx<T> z = S[e];
  double zx = z.x, zy = z.y;
  if (g.ovl != nullptr && k1 == 0 && k2 == 0 && k3 == 0) {
    // G = 0: the sum of the pair density over the grid, from the FP64 overlap
    // of the pair's coefficients instead of the FP32 transform (real)
    const int i = s ? ch.bi : ch.ai, j = s ? ch.bj : ch.aj;
    zx = g.ovl_scale * g.ovl[(int64_t)i * g.ovl_ld + (j - g.ovl_j0)];
    zy = 0.0;
  }
  const double a2 = zx * zx + zy * zy;
  const double v = g.vtab64[vi];
  const int slot = s ? ch.pb : ch.pa;
  if (slot >= 0) {
    atomicAdd(&epair[slot], wgt * v * a2);
    if (g.dvtab64) atomicAdd(&dpair[slot], wgt * g.dvtab64[vi] * a2);
  }
  const double vs = v * g.inv_ntot;
  z.x = T(zx * vs);
  z.y = T(zy * vs);
  S[e] = z;
}

// Stage the twiddle table in shared memory: tw[t] = e^{-2 pi i t/N} for the
// forward transforms, tw[N + t] = its conjugate for the inverse ones, so no
// transform negates a twiddle where it uses it.
template <class T>
__device__ __forceinline__ void load_twiddles(cplx<T>* tw, const DevPlan& g) {
  const cplx<T>* src = static_cast<const cplx<T>*>(g.tw);
  for (int t = threadIdx.x; t < g.n; t += blockDim.x) {
    const cplx<T> w = src[t];
    tw[t] = w;
    tw[g.n + t] = cmake<T>(w.x, -w.y);
  }
}

// ---------------------------------------------------------------- O(nb) passes

// X[q] = scatter(c_{b0} + i c_{b0+1}) for band pairs q of the batch (X zeroed before).
template <class T>
__global__ void k_scatter(DevPlan g, const double2* __restrict__ psiG, int nb, int band0, int nbat,
                          cplx<T>* __restrict__ X) {
  const int q = blockIdx.y;
  const int b0 = band0 + 2 * q;
  const bool has1 = (2 * q + 1 < nbat) && (b0 + 1 < nb);
  cplx<T>* Xq = X + (int64_t)q * g.ntot;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.npw; k += gridDim.x * blockDim.x) {
    const double2 c0 = psiG[(int64_t)b0 * g.npw + k];
    const double2 c1 = has1 ? psiG[(int64_t)(b0 + 1) * g.npw + k] : make_double2(0.0, 0.0);
    Xq[g.gidx[k]] = cmake<T>(T(c0.x - c1.y), T(c0.y + c1.x));
  }
}

// FFT along i1 of the slab X[q][:, i2, :] (all N columns).
template <class T, int N, int SIGN>
__global__ void __launch_bounds__(Geo<T, N>::THR_COLF) k_col_full(DevPlan g, cplx<T>* __restrict__ X) {
  using C = cplx<T>;
  using G = Geo<T, N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* S = reinterpret_cast<C*>(smem_raw);
  C* tw = S + N * N;
  const int i2 = blockIdx.x;
  C* Xq = X + (int64_t)blockIdx.y * g.ntot;
  load_twiddles<T>(tw, g);
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i1 = e / N, i3 = e - i1 * N;
    S[e] = Xq[((int64_t)i1 * N + i2) * N + i3];
  }
  __syncthreads();
  fft_lines<T, N, SIGN, N, G::TLP, 1, N>(S, tw);
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i1 = e / N, i3 = e - i1 * N;
    Xq[((int64_t)i1 * N + i2) * N + i3] = S[e];
  }
}

// 2D FFT over (i2, i3) of plane i1 of X[q].  PRO 0: load from X; PRO 1: z = W_b0 + i W_b0+1.
// EPI 0: store to X; EPI 1: psi_b0 = Re z * psi_scale, psi_b0+1 = Im z * psi_scale.
template <class T, int N, int SIGN, int PRO, int EPI>
__global__ void __launch_bounds__(Geo<T, N>::THR_PLANE)
    k_plane_full(DevPlan g, cplx<T>* __restrict__ X, const acc_t<T>* __restrict__ W, T* __restrict__ psi,
                 int band0, int nb, int nbat) {
  using C = cplx<T>;
  using G = Geo<T, N>;
  constexpr int RP = G::RP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);
  C* tw = P + N * RP;
  const int i1 = blockIdx.x, q = blockIdx.y;
  const int b0 = band0 + 2 * q;
  const bool has1 = (2 * q + 1 < nbat) && (b0 + 1 < nb);
  C* Xq = X + (int64_t)q * g.ntot + (int64_t)i1 * N * N;
  const int64_t plane0 = (int64_t)i1 * N * N;
  load_twiddles<T>(tw, g);
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i2 = e / N, i3 = e - i2 * N;
    C z;
    if (PRO == 0) {
      z = Xq[e];
    } else {
      z.x = T(W[(int64_t)b0 * g.ntot + plane0 + e]);
      z.y = has1 ? T(W[(int64_t)(b0 + 1) * g.ntot + plane0 + e]) : T(0);
    }
    P[i2 * RP + i3] = z;
  }
  __syncthreads();
  fft_lines<T, N, SIGN, N, G::TLP, RP, 1>(P, tw);  // along i3
  fft_lines<T, N, SIGN, N, G::TLP, 1, RP>(P, tw);  // along i2
  const T s = T(g.psi_scale);
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i2 = e / N, i3 = e - i2 * N;
    const C z = P[i2 * RP + i3];
    if (EPI == 0) {
      Xq[e] = z;
    } else {
      psi[(int64_t)b0 * g.ntot + plane0 + e] = z.x * s;
      if (has1) psi[(int64_t)(b0 + 1) * g.ntot + plane0 + e] = z.y * s;
    }
  }
}

// (V_x psi)(G) of the band pair q: Y = fft(W_b0 + i W_b0+1); X_b0(G) = (Y(G) + Y(-G)*)/2,
// X_b0+1(G) = (Y(G) - Y(-G)*)/(2i); both scaled by sqrt(Omega)/Ntot.
template <class T>
__global__ void k_gather(DevPlan g, const cplx<T>* __restrict__ X, int nb, int band0, int nbat,
                         double2* __restrict__ vpsiG) {
  const int q = blockIdx.y;
  const int b0 = band0 + 2 * q;
  const bool has1 = (2 * q + 1 < nbat) && (b0 + 1 < nb);
  const cplx<T>* Xq = X + (int64_t)q * g.ntot;
  const double s = 0.5 * g.out_scale;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.npw; k += gridDim.x * blockDim.x) {
    const cplx<T> y = Xq[g.gidx[k]], ym = Xq[g.gidxneg[k]];
    const double yx = to_double(y.x), yy = to_double(y.y), mx = to_double(ym.x), my = to_double(ym.y);
    vpsiG[(int64_t)b0 * g.npw + k] = make_double2(s * (yx + mx), s * (yy - my));
    if (has1) vpsiG[(int64_t)(b0 + 1) * g.npw + k] = make_double2(s * (yy + my), s * (mx - yx));
  }
}

// ------------------------------------------------------------------ pair passes

// One task of the forward plane pass: plane i1 of chain `ch`, whose transform
// buffer is Hc.  Shared memory: Geo::SMEM_PLANE bytes at smem_raw.
template <class T, int N, int MAXT, int EMAX = 0>
__device__ __forceinline__ void pair_fwd_task(const DevPlan& g, const T* __restrict__ psi,
                                              const Chain& ch, cplx<T>* __restrict__ Hc, int i1,
                                              unsigned char* smem_raw) {
  using C = cplx<T>;
  using G = Geo<T, N, MAXT, EMAX>;
  constexpr int RP = G::RP, KH = G::KH, NC = G::NC;
  C* P = reinterpret_cast<C*>(smem_raw);
  C* tw = P + N * RP;
  load_twiddles<T>(tw, g);
  const int64_t plane0 = (int64_t)i1 * N * N;
  const bool hb = ch.bi >= 0;
  const T* pai = psi + (int64_t)ch.ai * g.ntot + plane0;
  const T* paj = psi + (int64_t)ch.aj * g.ntot + plane0;
  const T* pbi = psi + (int64_t)(hb ? ch.bi : 0) * g.ntot + plane0;
  const T* pbj = psi + (int64_t)(hb ? ch.bj : 0) * g.ntot + plane0;
  // Columns first: the first stage along i2 reads the pair product straight
  // from the orbital planes (a warp's lines are consecutive columns i3, so the
  // loads coalesce) and leaves its outputs in shared memory; then the rows.
  // this thread's column i3 (line-fast mapping of the transform along i2)
  const int c3 = threadIdx.x % N;
  const T* qai = pai + c3;
  const T* qaj = paj + c3;
  const T* qbi = pbi + c3;
  const T* qbj = pbj + c3;
  if (hb && ch.ai == ch.bi) {
    // the usual chain, pairs (i, j) and (i, j'): psi_i is read once
    const auto product = [&](int, int i2) {
      const T x = qai[i2 * N];
      return cmake<T>(x * qaj[i2 * N], x * qbj[i2 * N]);
    };
    fft_lines_from<T, N, -1, N, G::TLP, 1, RP, MAXT, EMAX>(P, tw, product);  // along i2
  } else {
    const auto product = [&](int, int i2) {
      return cmake<T>(qai[i2 * N] * qaj[i2 * N], hb ? qbi[i2 * N] * qbj[i2 * N] : T(0));
    };
    fft_lines_from<T, N, -1, N, G::TLP, 1, RP, MAXT, EMAX>(P, tw, product);  // along i2
  }
  // along i3: only the rows k2 that hold kept columns, [0, row_lo) and
  // [N - row_hi, N) (the split below reads row k2 and its mirror N - k2, both in)
  const int rlo = g.row_lo, nrows = g.row_lo + g.row_hi;
  const auto row_off = [&](int l) { return (l < rlo ? l : l + (N - nrows)) * RP; };
  fft_lines_rt<T, N, -1, G::TLP, 1, MAXT, EMAX>(P, tw, nrows, row_off);
  C* Hp = Hc + (int64_t)i1 * N * NC;
  // split by Hermitian symmetry over the list of kept columns (k2, k3): every
  // lane busy, consecutive threads on consecutive k3 of a row
  for (int e = threadIdx.x; e < g.nkept; e += blockDim.x) {
    const int code = __ldg(g.kept + e);
    const int k2 = code >> 16, k3 = code & 0xffff;
    const int m2 = k2 == 0 ? 0 : N - k2, m3 = k3 == 0 ? 0 : N - k3;
    const C z = P[k2 * RP + k3], zm = P[m2 * RP + m3];
    Hp[k2 * NC + k3] = cmake<T>(half_of(z.x + zm.x), half_of(z.y - zm.y));
    Hp[k2 * NC + KH + k3] = cmake<T>(half_of(z.y + zm.y), half_of(zm.x - z.x));
  }
}

template <class T, int N, int EMAX = 0>
__global__ void __launch_bounds__(Geo<T, N, kMaxThreads, EMAX>::THR_PLANE)
    k_pair_fwd(DevPlan g, const T* __restrict__ psi, const Chain* __restrict__ chains,
               cplx<T>* __restrict__ H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Chain ch = chains[blockIdx.y];
  pair_fwd_task<T, N, kMaxThreads, EMAX>(g, psi, ch, H + (int64_t)blockIdx.y * g.hsize, blockIdx.x, smem_raw);
}

// Publish a CTA's energy partials (thread 0): atomically into the pair slots,
// or, in deterministic mode, into slot [pair * ncta_col + cta] for a sum in a
// fixed order afterwards.
__device__ __forceinline__ void put_energies(const DevPlan& g, const Chain& ch, int cta, const double acc[4],
                                             bool want_d, double* epair, double* dpair) {
  if (g.det) {
    const int64_t nc = g.ncta_col;
    if (ch.pa >= 0) epair[ch.pa * nc + cta] = acc[0];
    if (ch.pb >= 0) epair[ch.pb * nc + cta] = acc[1];
    if (want_d) {
      if (ch.pa >= 0) dpair[ch.pa * nc + cta] = acc[2];
      if (ch.pb >= 0) dpair[ch.pb * nc + cta] = acc[3];
    }
    return;
  }
  if (ch.pa >= 0) atomicAdd(&epair[ch.pa], acc[0]);
  if (ch.pb >= 0) atomicAdd(&epair[ch.pb], acc[1]);
  if (want_d) {
    if (ch.pa >= 0) atomicAdd(&dpair[ch.pa], acc[2]);
    if (ch.pb >= 0) atomicAdd(&dpair[ch.pb], acc[3]);
  }
}

// Deterministic accumulation: one contribution as 64-bit fixed point (scale
// 2^s), added with an integer atomic (exact, so the order does not matter).
__device__ __forceinline__ void det_add(double* p, double v, double scale) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double2ll_rn(v * scale));
}
__device__ __forceinline__ void det_add(double* p, df64 v, double scale) {
  const float sf = (float)scale;  // a power of two, exact in float
  const long long q = __float2ll_rn(v.hi * sf) + __float2ll_rn(v.lo * sf);
  atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)q);
}
__device__ __forceinline__ void det_add(float*, float, double) {}  // not offered for the mixed form

// Line code of the column pass: (k2 << 16) | (s << 15) | k3, or -1 (no line).
__device__ __forceinline__ int line_k2(int code) { return code >> 16; }
__device__ __forceinline__ int line_s(int code) { return (code >> 15) & 1; }
__device__ __forceinline__ int line_k3(int code) { return code & 0x7fff; }

// Asynchronous global-to-shared copies (cp.async) for the double-float
// inverse plane pass of the stand-alone kernels: every element of a thread is
// in flight at once, no register holds it.  Inside the persistent kernel the
// loads stay ld.global.cg (the buffer was written earlier by the same launch,
// so L1 must not serve it).
constexpr bool kColAsync = true;
// The column and inverse passes read their first transform stage straight from
// the transform buffer (no staging pass through shared memory).  Measured at
// 96^3: column pass -2..-6% in every form, inverse pass -13% (mixed) and -3%
// (FP64) but +9% in double-float, whose inverse pass keeps the cp.async staging.
constexpr bool kFirstStageDirect = true;
template <class T> __host__ __device__ constexpr bool inv_first_stage_direct() {
  return kFirstStageDirect && RealTraits<T>::prec != 2;
}

// Stage the column pass's line codes (NL a CTA) in shared memory.
template <int NL>
__device__ __forceinline__ void col_codes(const DevPlan& g, int cta, int* codes) {
  for (int l = threadIdx.x; l < NL; l += blockDim.x) codes[l] = __ldg(g.colmap + cta * NL + l);
  __syncthreads();
}

// The column of Hc (NC stored columns a row) that this thread's line of the
// column pass reads and writes (the line-fast thread mapping of the
// transforms: line tid mod NL), or NULL for a line without a code.  codes
// must be staged.
template <class C, int N, int NC, int NL>
__device__ __forceinline__ C* col_line_ptr(C* Hc, const int* codes) {
  constexpr int KH = NC / 2;
  const int code = codes[threadIdx.x % NL];
  return code >= 0 ? Hc + line_k2(code) * NC + line_s(code) * KH + line_k3(code) : nullptr;
}

// Store the transformed lines: thread (line l, sub-thread t) writes elements
// i1 = t, t + TL, ... of its own line (consecutive lanes hold consecutive
// lines, so both the shared reads and the global writes are contiguous).
template <class C, int N, int NC, int NL, int TL>
__device__ __forceinline__ void col_store_lines(C* lp, const C* S) {
  const int l = threadIdx.x % NL, t = threadIdx.x / NL;
  if (lp != nullptr && t < TL) {
#pragma unroll 4
    for (int i1 = t; i1 < N; i1 += TL) lp[(int64_t)i1 * N * NC] = S[i1 * NL + l];
  }
}

// The column pass in double-float arithmetic: the df64 tables of v / Ntot and
// dv/domega, per-thread double-float energy sums that are reduced (in FP64)
// before the inverse transform, so they hold no registers across it.
template <int N, int MAXT, int EMAX = 0>
__device__ __forceinline__ void pair_col_task_df(const DevPlan& g, cdf64* __restrict__ Hc, const Chain& ch,
                                                 int cta, double* __restrict__ epair, double* __restrict__ dpair,
                                                 unsigned char* smem_raw) {
  using C = cdf64;
  using G = Geo<df64, N, MAXT, EMAX>;
  constexpr int KH = G::KH, NC = G::NC, NL = G::NLC;
  C* S = reinterpret_cast<C*>(smem_raw);
  C* tw = S + N * NL;
  double* red = reinterpret_cast<double*>(tw + G::TWN);
  int* codes = reinterpret_cast<int*>(red + 32 * 4);
  load_twiddles<df64>(tw, g);
  const bool want_d = g.dvtab64 != nullptr;
  const df64* vt = static_cast<const df64*>(g.vtab);  // v / Ntot
  const df64* dvt = static_cast<const df64*>(g.dvtab);  // dv/domega
  col_codes<NL>(g, cta, codes);
  {
    const C* lp = col_line_ptr<C, N, NC, NL>(Hc, codes);
    const auto val = [&](int, int i1) {
      C v;
      if (lp != nullptr) {
        v = ldcg_c(lp + (int64_t)i1 * N * NC);
      } else {
        v.x = df64(0.f);
        v.y = df64(0.f);
      }
      return v;
    };
    fft_lines_from<df64, N, -1, NL, G::TLC, 1, NL, MAXT, EMAX>(S, tw, val);  // along i1
  }
  {
    df64 accd[4] = {df64(0.f), df64(0.f), df64(0.f), df64(0.f)};
    // one line per thread (decoded once), walking k1
    const int l = threadIdx.x % NL, kstep = blockDim.x / NL;
    const int code = threadIdx.x < kstep * NL ? codes[l] : -1;
    if (code >= 0) {
      const int k2 = line_k2(code), s = line_s(code), k3 = line_k3(code);
      const float wgt = (k3 == 0 || 2 * k3 == N) ? 1.0f : 2.0f;
      df64 e_sum(0.f), d_sum(0.f);
      for (int k1 = threadIdx.x / NL; k1 < N; k1 += kstep) {
        const int e = k1 * NL + l;
        const int vi = (k1 * N + k2) * KH + k3;
        C z = S[e];
        const df64 a2 = z.x * z.x + z.y * z.y;
        const df64 v = vt[vi];
        e_sum += v * a2;
        if (want_d) d_sum += dvt[vi] * a2;
        z.x *= v;
        z.y *= v;
        S[e] = z;
      }
      e_sum = ldexp_pow2(e_sum, wgt);
      d_sum = ldexp_pow2(d_sum, wgt);
      if (s) {
        accd[1] = e_sum;
        accd[3] = d_sum;
      } else {
        accd[0] = e_sum;
        accd[2] = d_sum;
      }
    }
    block_sum4_df(accd, reinterpret_cast<float*>(red));  // synchronises the CTA
    if (threadIdx.x == 0) {
      const double ntot = double(g.ntot);  // the energy table holds v / Ntot
      const double acc[4] = {to_double(accd[0]) * ntot, to_double(accd[1]) * ntot, to_double(accd[2]),
                             to_double(accd[3])};
      put_energies(g, ch, cta, acc, want_d, epair, dpair);
    }
  }
  fft_lines<df64, N, +1, NL, G::TLC, 1, NL, MAXT, EMAX>(S, tw);  // inverse along k1
  col_store_lines<C, N, NC, NL, G::TLC>(col_line_ptr<C, N, NC, NL>(Hc, codes), S);
}

// The column pass in FP64 or in the mixed form.
template <class T, int N, int MAXT, int EMAX = 0>
__device__ __forceinline__ void pair_col_task_std(const DevPlan& g, cplx<T>* __restrict__ Hc,
                                                  const Chain& ch, int cta, double* __restrict__ epair,
                                                  double* __restrict__ dpair, unsigned char* smem_raw) {
  using C = cplx<T>;
  using G = Geo<T, N, MAXT, EMAX>;
  constexpr int KH = G::KH, NC = G::NC, NL = G::NLC;
  C* S = reinterpret_cast<C*>(smem_raw);
  C* tw = S + N * NL;
  double* red = reinterpret_cast<double*>(tw + G::TWN);
  int* codes = reinterpret_cast<int*>(red + 32 * 4);
  load_twiddles<T>(tw, g);
  col_codes<NL>(g, cta, codes);
  {
    // the first stage reads this thread's line straight from the transform
    // buffer: one base pointer per thread, compile-time offsets per element
    const C* lp = col_line_ptr<C, N, NC, NL>(Hc, codes);
    const auto val = [&](int, int i1) {
      C v;
      if (lp != nullptr) {
        v = ldcg_c(lp + (int64_t)i1 * N * NC);
      } else {
        v.x = 0;
        v.y = 0;
      }
      return v;
    };
    fft_lines_from<T, N, -1, NL, G::TLC, 1, NL, MAXT, EMAX>(S, tw, val);  // along i1
  }

  // kernel multiply and energy partials
  const bool want_d = g.dvtab64 != nullptr;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // e_a, e_b, d_a, d_b (FP64 terms)
  float acc_f32[4] = {0.f, 0.f, 0.f, 0.f};  // the same from the FP32 terms (mixed form)
  // one line per thread (decoded once), walking k1
  const int l = threadIdx.x % NL, kstep = blockDim.x / NL;
  const int code = threadIdx.x < kstep * NL ? codes[l] : -1;
  if constexpr (RealTraits<T>::prec == 0) {
    if (code >= 0) {
      const int k2 = line_k2(code), s = line_s(code), k3 = line_k3(code);
      const double wgt = (k3 == 0 || 2 * k3 == N) ? 1.0 : 2.0;
      const double* v64 = g.vtab64 + k2 * KH + k3;
      const double* dv64 = g.dvtab64 ? g.dvtab64 + k2 * KH + k3 : nullptr;
      // v / Ntot, or -f0 v / Ntot when the occupations are uniform (vtab_f set)
      const double* vs64 = static_cast<const double*>(g.vtab) + k2 * KH + k3;
      double e_sum = 0.0, d_sum = 0.0;
      for (int k1 = threadIdx.x / NL; k1 < N; k1 += kstep) {
        const int e = k1 * NL + l;
        const int vo = k1 * N * KH;
        C z = S[e];
        const double a2 = z.x * z.x + z.y * z.y;
        e_sum += v64[vo] * a2;
        if (want_d) d_sum += dv64[vo] * a2;
        const double vs = vs64[vo];
        z.x *= vs;
        z.y *= vs;
        S[e] = z;
      }
      if (s) {  // explicit selects: a runtime index would put acc in local memory
        acc[1] = wgt * e_sum;
        acc[3] = wgt * d_sum;
      } else {
        acc[0] = wgt * e_sum;
        acc[2] = wgt * d_sum;
      }
    }
  } else {
    const T* vt = static_cast<const T*>(g.vtab);    // v / Ntot
    const T* dvt = static_cast<const T*>(g.dvtab);  // dv/domega
    T accf[4] = {T(0), T(0), T(0), T(0)};
    if (code >= 0) {
      const int k2 = line_k2(code), s = line_s(code), k3 = line_k3(code);
      const int m2 = freq_of(k2, N), m3 = freq_of(k3, N);
      const int r23 = m2 * m2 + m3 * m3;
      const T wgt = (k3 == 0 || 2 * k3 == N) ? T(1) : T(2);
      const T* vl = vt + k2 * KH + k3;
      const T* dvl = dvt + k2 * KH + k3;
      T e_sum = T(0), d_sum = T(0);
      if (r23 > g.msmall2) {  // no term of this line is a small-|G| one
        const int k10 = threadIdx.x / NL;
        const T* vp = vl + k10 * N * KH;
        const T* dvp = dvl + k10 * N * KH;
        C* sp = S + k10 * NL + l;
        const int vstep = kstep * N * KH, sstep = kstep * NL;
        // batches of U elements: the U table loads are in flight together
        constexpr int U = 8;
        int k1 = k10;
        for (; k1 + (U - 1) * kstep < N; k1 += U * kstep, vp += U * vstep, dvp += U * vstep, sp += U * sstep) {
          T v[U], dv[U];
          C z[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            v[u] = vp[u * vstep];
            dv[u] = want_d ? dvp[u * vstep] : T(0);
            z[u] = sp[u * sstep];
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const T a2 = z[u].x * z[u].x + z[u].y * z[u].y;
            e_sum += v[u] * a2;
            d_sum += dv[u] * a2;
            sp[u * sstep] = cmake<T>(z[u].x * v[u], z[u].y * v[u]);
          }
        }
        for (; k1 < N; k1 += kstep, vp += vstep, dvp += vstep, sp += sstep) {
          C z = *sp;
          const T a2 = z.x * z.x + z.y * z.y;
          const T v = *vp;
          e_sum += v * a2;
          if (want_d) d_sum += *dvp * a2;
          z.x *= v;
          z.y *= v;
          *sp = z;
        }
      } else {
        for (int k1 = threadIdx.x / NL; k1 < N; k1 += kstep) {
          const int e = k1 * NL + l;
          const int m1 = freq_of(k1, N);
          if (m1 * m1 + r23 <= g.msmall2) {
            if (s == 0 || ch.bi >= 0) small_g_term_fp64<T, N>(g, S, e, k1, k2, k3, s, ch, epair, dpair);
            continue;
          }
          const int vo = k1 * N * KH;
          C z = S[e];
          const T a2 = z.x * z.x + z.y * z.y;
          const T v = vl[vo];
          e_sum += v * a2;
          if (want_d) d_sum += dvl[vo] * a2;
          z.x *= v;
          z.y *= v;
          S[e] = z;
        }
      }
      if (s) {
        accf[1] = wgt * e_sum;
        accf[3] = wgt * d_sum;
      } else {
        accf[0] = wgt * e_sum;
        accf[2] = wgt * d_sum;
      }
    }
    // per-thread FP32 sums of at most N (N+2) / blockDim non-negative terms;
    // the table holds v / Ntot, undone in FP64 after the CTA reduction
    acc_f32[0] = accf[0];
    acc_f32[1] = accf[1];
    acc_f32[2] = accf[2];
    acc_f32[3] = accf[3];
  }
  __syncthreads();
  fft_lines<T, N, +1, NL, G::TLC, 1, NL, MAXT, EMAX>(S, tw);  // inverse along k1
  col_store_lines<C, N, NC, NL, G::TLC>(col_line_ptr<C, N, NC, NL>(Hc, codes), S);
  if constexpr (RealTraits<T>::prec != 1) {
    block_sum4(acc, red);
  } else {
    float hi[4], lo[4];
    block_sum4_ff(acc_f32, hi, lo, reinterpret_cast<float*>(red));
    if (threadIdx.x == 0) {
      const double ntot = double(g.ntot);  // the FP32 table holds v / Ntot
      for (int k = 0; k < 4; ++k) acc[k] = ((double)hi[k] + (double)lo[k]) * (k < 2 ? ntot : 1.0);
    }
  }
  if (threadIdx.x == 0) put_energies(g, ch, cta, acc, want_d, epair, dpair);
}

// One task of the column pass: the NLC lines `cta` of the column map for chain
// `ch` (transform buffer Hc).  Shared memory: Geo::SMEM_COLH bytes at smem_raw.
template <class T, int N, int MAXT, int EMAX = 0>
__device__ __forceinline__ void pair_col_task(const DevPlan& g, cplx<T>* __restrict__ Hc,
                                              const Chain& ch, int cta, double* __restrict__ epair,
                                              double* __restrict__ dpair, unsigned char* smem_raw) {
  if constexpr (RealTraits<T>::prec == 2) {
    pair_col_task_df<N, MAXT, EMAX>(g, Hc, ch, cta, epair, dpair, smem_raw);
  } else {
    pair_col_task_std<T, N, MAXT, EMAX>(g, Hc, ch, cta, epair, dpair, smem_raw);
  }
}

template <class T, int N, int EMAX = 0>
__global__ void __launch_bounds__(Geo<T, N, kMaxThreads, EMAX>::THR_COL, Geo<T, N, kMaxThreads, EMAX>::MIN_CTAS_COL)
    k_pair_col(DevPlan g, cplx<T>* __restrict__ H, const Chain* __restrict__ chains,
               double* __restrict__ epair, double* __restrict__ dpair) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Chain ch = chains[blockIdx.y];
  pair_col_task<T, N, kMaxThreads, EMAX>(g, H + (int64_t)blockIdx.y * g.hsize, ch, blockIdx.x, epair, dpair,
                                         smem_raw);
}

// One task of the inverse plane pass: plane i1 of chain `ch` (transform buffer
// Hc), accumulating into W.  Shared memory: Geo::SMEM_PLANE bytes at smem_raw.
template <class T, int N, int MAXT, int EMAX = 0>
__device__ __forceinline__ void pair_inv_task(const DevPlan& g, const T* __restrict__ psi,
                                              acc_t<T>* __restrict__ W, const T* __restrict__ occ,
                                              const Chain& ch, const cplx<T>* __restrict__ Hc, int i1,
                                              unsigned char* smem_raw) {
  using C = cplx<T>;
  using G = Geo<T, N, MAXT, EMAX>;
  constexpr int KH = G::KH, NC = G::NC, NCP = G::NCP;
  C* Q = reinterpret_cast<C*>(smem_raw);
  C* tw = Q + N * NCP;
  int* ncol = reinterpret_cast<int*>(tw + G::TWN);
  load_twiddles<T>(tw, g);
  for (int r = threadIdx.x; r < N; r += blockDim.x) ncol[r] = __ldg(g.ncol + r);
  __syncthreads();
  const C* Hp = Hc + (int64_t)i1 * N * NC;
  // 1-2. the stored half plane, row k2 = [A(k2, 0..N/2) | B(k2, 0..N/2)],
  //    columns no pair density reaches (never written) read as zero, and its
  //    inverse transform along k2 into Q[k2][c] (odd row stride NCP).  Only
  //    the columns k3 < col_max of A and B hold anything: 2 col_max lines are
  //    transformed, line l being column l (A) or KH + l - col_max (B).
  const int cm = g.col_max;
  const auto col_of = [&](int l) { return l < cm ? l : KH + (l - cm); };
  if constexpr (inv_first_stage_direct<T>()) {
    const unsigned long long last_use = l2_policy_evict_first();  // H is dead after this read
    const auto val = [&](int l, int k2) {
      C v;
      if ((l < cm ? l : l - cm) < ncol[k2]) {
        v = ldcg_hint(Hp + k2 * NC + col_of(l), last_use);
      } else {
        v.x = 0;
        v.y = 0;
      }
      return v;
    };
    fft_lines_from_rt<T, N, +1, G::TLC, NCP, MAXT, EMAX>(Q, tw, 2 * cm, val, col_of);
  } else {
  if constexpr (kColAsync && MAXT == kMaxThreads) {
    for (int e = threadIdx.x; e < N * NC; e += blockDim.x) {
      const int k2 = e / NC, c = e - k2 * NC;
      const int keep = (c < KH ? c : c - KH) < ncol[k2];
      const unsigned dst = (unsigned)__cvta_generic_to_shared(Q + k2 * NCP + c);
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(Hp + e), "n"((int)sizeof(C)),
                   "r"(keep ? (int)sizeof(C) : 0)
                   : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else {
    for (int e0 = threadIdx.x; e0 < N * NC; e0 += kLoadUnroll * blockDim.x) {
      C v[kLoadUnroll];
#pragma unroll
      for (int u = 0; u < kLoadUnroll; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < N * NC) {
          const int k2 = e / NC, c = e - k2 * NC;
          v[u] = ldcg_c(Hp + e);
          if (!((c < KH ? c : c - KH) < ncol[k2])) v[u] = cmake<T>(T(0), T(0));
        }
      }
#pragma unroll
      for (int u = 0; u < kLoadUnroll; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < N * NC) {
          const int k2 = e / NC, c = e - k2 * NC;
          Q[k2 * NCP + c] = v[u];
        }
      }
    }
  }
  __syncthreads();
  fft_lines_rt<T, N, +1, G::TLC, NCP, MAXT, EMAX>(Q, tw, 2 * cm, col_of);  // inverse transform along k2
  }
  // 3. rows: z(k3) = A^(k3) + i B^(k3) for k3 <= N/2 and, from the Hermitian
  //    symmetry of the transforms of the real planes, z(N - k3) =
  //    conj(A^(k3)) + i conj(B^(k3)); one warp per row (reads, then writes);
  //    columns k3 >= col_max were not transformed and hold nothing
  {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    static_assert(N / 2 + 1 <= 64, "two stored columns per lane");
    for (int i2 = threadIdx.x >> 5; i2 < N; i2 += nw) {
      C* row = Q + i2 * NCP;
      C av[2], bv[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int k = lane + 32 * t;
        if (k < cm) {
          av[t] = row[k];
          bv[t] = row[KH + k];
        } else {
          av[t] = cmake<T>(T(0), T(0));
          bv[t] = av[t];
        }
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int k = lane + 32 * t;
        if (k < KH) {
          row[k] = cmake<T>(av[t].x - bv[t].y, av[t].y + bv[t].x);
          if (k > 0 && 2 * k < N) row[N - k] = cmake<T>(av[t].x + bv[t].y, bv[t].x - av[t].y);
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // 4. inverse transform along k3 of the N rows: Q[i2][i3] = phi_a + i phi_b,
  //    in FP32 with each row left in quad phases (element 4c + u of row i2 at
  //    i2 NCP + u N/4 + c): the four-point groups of the accumulator update
  //    are then read with consecutive lanes on consecutive addresses
  constexpr int OMAP = (RealTraits<T>::prec == 1 && N % 4 == 0) ? 1 : 0;
  fft_lines<T, N, +1, N, G::TLP, NCP, 1, MAXT, EMAX, OMAP>(Q, tw);
  const int64_t plane0 = (int64_t)i1 * N * N;
  const bool hb = ch.bi >= 0;
  // Up to four updates k, W[tgt_k] -= f[src_k] psi[src_k] phi:
  //   k = 0: W_aj -= f_ai psi_ai phi_a      k = 1: W_ai -= f_aj psi_aj phi_a (i != j)
  //   k = 2: W_bj -= f_bi psi_bi phi_b      k = 3: W_bi -= f_bj psi_bj phi_b (i != j)
  // Updates of the same band are summed first (into[k] = first slot with that
  // band), so each distinct band costs one atomic per point.
  int tgt[4] = {ch.aj, (ch.ai != ch.aj && !(ch.flags & kChainOneSidedA)) ? ch.ai : -1, hb ? ch.bj : -1,
                (hb && ch.bi != ch.bj && !(ch.flags & kChainOneSidedB)) ? ch.bi : -1};
  const int src[4] = {ch.ai, ch.aj, hb ? ch.bi : 0, hb ? ch.bj : 0};
  const T f[4] = {occ[ch.ai], occ[ch.aj], hb ? occ[ch.bi] : T(0), hb ? occ[ch.bj] : T(0)};
  int into[4] = {0, 1, 2, 3};  // which slot a contribution is added to
#pragma unroll
  for (int k = 1; k < 4; ++k)
#pragma unroll
    for (int m = 0; m < k; ++m)
      if (into[k] == k && tgt[k] >= 0 && tgt[m] == tgt[k]) into[k] = m;
  const T* ps[4];
  acc_t<T>* wt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ps[k] = psi + (int64_t)src[k] * g.ntot + plane0;
    wt[k] = W + (int64_t)(tgt[k] >= 0 ? tgt[k] : 0) * g.ntot + plane0;
  }
  if constexpr (RealTraits<T>::prec == 1) {
    // four consecutive points per thread: 16-byte loads of the orbitals and
    // one red.global.add.v4.f32 per target
    static_assert(N % 4 == 0, "vector updates need N divisible by 4");
    const unsigned long long keep = l2_policy_evict_last();  // orbitals and accumulators of the band block
    // The usual chain of the band-blocked schedule: pairs (i, j) and (i, j')
    // with i, j, j' distinct and both updates wanted.  Three orbitals, three
    // targets: W_j -= f_i psi_i phi_a, W_j' -= f_i psi_i phi_b and
    // W_i -= f_j psi_j phi_a + f_j' psi_j' phi_b, without per-point bookkeeping.
    const bool shared_i = hb && ch.ai == ch.bi && ch.ai != ch.aj && ch.ai != ch.bj && ch.aj != ch.bj &&
                          !(ch.flags & (kChainOneSidedA | kChainOneSidedB));
    if (shared_i) {
      const float mi = -f[0], mj = -f[1], mj2 = -f[3];
      const float* pi = ps[0];
      const float* pj = ps[1];
      const float* pj2 = ps[3];
      float* wj = wt[0];
      float* wj2 = wt[2];
      float* wi = wt[1];
      for (int e4 = threadIdx.x; e4 < N * N / 4; e4 += blockDim.x) {
        const int e = 4 * e4;
        const int i2 = e4 / (N / 4), c = e4 - i2 * (N / 4);
        const C* q = Q + i2 * NCP + c;  // quad phases: element 4c + u at u N/4 + c
        const C z0 = q[0], z1 = q[N / 4], z2 = q[2 * (N / 4)], z3 = q[3 * (N / 4)];
        const float4 vi = ld_f4_hint(pi + e, keep);
        const float4 vj = ld_f4_hint(pj + e, keep);
        const float4 vj2 = ld_f4_hint(pj2 + e, keep);
        const float4 a = make_float4(mi * vi.x * z0.x, mi * vi.y * z1.x, mi * vi.z * z2.x, mi * vi.w * z3.x);
        const float4 b = make_float4(mi * vi.x * z0.y, mi * vi.y * z1.y, mi * vi.z * z2.y, mi * vi.w * z3.y);
        const float4 ci = make_float4(mj * vj.x * z0.x + mj2 * vj2.x * z0.y, mj * vj.y * z1.x + mj2 * vj2.y * z1.y,
                                      mj * vj.z * z2.x + mj2 * vj2.z * z2.y, mj * vj.w * z3.x + mj2 * vj2.w * z3.y);
        asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(wj + e), "f"(a.x),
                     "f"(a.y), "f"(a.z), "f"(a.w), "l"(keep)
                     : "memory");
        asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(wj2 + e), "f"(b.x),
                     "f"(b.y), "f"(b.z), "f"(b.w), "l"(keep)
                     : "memory");
        asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(wi + e), "f"(ci.x),
                     "f"(ci.y), "f"(ci.z), "f"(ci.w), "l"(keep)
                     : "memory");
      }
      return;
    }
    for (int e4 = threadIdx.x; e4 < N * N / 4; e4 += blockDim.x) {
      const int e = 4 * e4;
      const int i2 = e4 / (N / 4), cq = e4 - i2 * (N / 4);
      float4 phia, phib;
      {
        const C* q = Q + i2 * NCP + cq;  // quad phases
        const C z0 = q[0], z1 = q[N / 4], z2 = q[2 * (N / 4)], z3 = q[3 * (N / 4)];
        phia = make_float4(z0.x, z1.x, z2.x, z3.x);
        phib = make_float4(z0.y, z1.y, z2.y, z3.y);
      }
      float4 c[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        c[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tgt[k] < 0) continue;
        const float4 p = ld_f4_hint(ps[k] + e, keep);
        const float4 ph = k < 2 ? phia : phib;
        const float m = -f[k];
        c[k] = make_float4(m * p.x * ph.x, m * p.y * ph.y, m * p.z * ph.z, m * p.w * ph.w);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (tgt[r] < 0 || into[r] != r) continue;
        float4 a = c[r];
#pragma unroll
        for (int k = r + 1; k < 4; ++k) {
          if (into[k] == r) {
            a.x += c[k].x;
            a.y += c[k].y;
            a.z += c[k].z;
            a.w += c[k].w;
          }
        }
        float* dst = wt[r] + e;
        asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(dst), "f"(a.x),
                     "f"(a.y), "f"(a.z), "f"(a.w), "l"(keep)
                     : "memory");
      }
    }
  } else {
    const bool det = g.det != 0;
    const double dscale = det ? g.det_scale[0] : 0.0;
    // both sources of each pair equally occupied (the usual case): -f phi is
    // formed once per pair and point, one multiplication fewer per update
    const bool same_f = f[0] == f[1] && f[2] == f[3];
    // FP64: phi carries -f0 already (uniform occupations)
    const bool prescaled = RealTraits<T>::prec == 0 && g.vtab_f != nullptr;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
      const int i2 = e / N, i3 = e - i2 * N;
      const C z = Q[i2 * NCP + i3];
      T c[4];
      if (RealTraits<T>::prec == 0 && prescaled) {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = tgt[k] < 0 ? T(0) : ps[k][e] * (k < 2 ? z.x : z.y);
      } else if (same_f) {
        const T ga = -f[0] * z.x, gb = -f[2] * z.y;
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = tgt[k] < 0 ? T(0) : ps[k][e] * (k < 2 ? ga : gb);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = tgt[k] < 0 ? T(0) : -f[k] * ps[k][e] * (k < 2 ? z.x : z.y);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (tgt[r] < 0 || into[r] != r) continue;
        T a = c[r];
#pragma unroll
        for (int k = r + 1; k < 4; ++k)
          if (into[k] == r) a += c[k];
        if (det) det_add(wt[r] + e, a, dscale);
        else atomic_add_real(wt[r] + e, a);
      }
    }
  }
}

template <class T, int N, int EMAX = 0>
__global__ void __launch_bounds__(Geo<T, N, kMaxThreads, EMAX>::THR_COLH, Geo<T, N, kMaxThreads, EMAX>::MIN_CTAS)
    k_pair_inv(DevPlan g, const T* __restrict__ psi, acc_t<T>* __restrict__ W, const T* __restrict__ occ,
               const Chain* __restrict__ chains, const cplx<T>* __restrict__ H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Chain ch = chains[blockIdx.y];
  pair_inv_task<T, N, kMaxThreads, EMAX>(g, psi, W, occ, ch, H + (int64_t)blockIdx.y * g.hsize, blockIdx.x,
                                         smem_raw);
}

// ------------------------------------------------------------ FFT tilings
//
// Each pair pass can run one of two radix plans ("tilings"): tile 0 is the
// type's own (FftTraits::emax elements per thread), tile 1 the plan found
// with the other element budget (12 for FP32, 24 for FP64; none for the
// double-float form).  When both budgets give the same plan for N, tile 1 is
// tile 0 and no second kernel is compiled.
template <class T> constexpr int alt_emax() {
  return RealTraits<T>::prec == 1 ? 12 : (RealTraits<T>::prec == 0 ? 24 : 0);
}
constexpr bool same_plan(const RadixPlan& a, const RadixPlan& b) {
  if (a.nst != b.nst || a.tl_plane != b.tl_plane || a.tl_colh != b.tl_colh) return false;
  for (int k = 0; k < a.nst; ++k)
    if (a.r[k] != b.r[k]) return false;
  return true;
}
template <class T, int N> constexpr int tile1_emax() {
  return (alt_emax<T>() == 0 ||
          same_plan(Geo<T, N>::pl, Geo<T, N, kMaxThreads, alt_emax<T>()>::pl))
             ? 0
             : alt_emax<T>();
}

// ------------------------------------------------------------------ launchers

constexpr size_t smem_max(size_t a, size_t b) { return a > b ? a : b; }

template <class T, int N>
struct Launch {
  using C = cplx<T>;
  using G = Geo<T, N>;
  static constexpr int E1 = tile1_emax<T, N>();  // EMAX of tile 1 (0: tile 1 is tile 0)
  using G1 = Geo<T, N, kMaxThreads, E1>;

  static cudaError_t configure(const DevPlan&) {
    const void* fns[] = {(const void*)k_col_full<T, N, +1>, (const void*)k_col_full<T, N, -1>,
                         (const void*)k_plane_full<T, N, +1, 0, 1>,
                         (const void*)k_plane_full<T, N, -1, 1, 0>, (const void*)k_pair_fwd<T, N>,
                         (const void*)k_pair_fwd<T, N, E1>};
    for (const void* f : fns) {
      cudaError_t err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)G::SMEM_PLANE);
      if (err != cudaSuccess) return err;
    }
    for (const void* f : {(const void*)k_pair_inv<T, N>, (const void*)k_pair_inv<T, N, E1>}) {
      cudaError_t err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_INV);
      if (err != cudaSuccess) return err;
    }
    for (const void* f : {(const void*)k_pair_col<T, N>, (const void*)k_pair_col<T, N, E1>}) {
      cudaError_t err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_COLH);
      if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
  }

  // Radix plan of tile `tile` (0 or 1) of pass `pass` (0 forward plane, 1
  // column, 2 inverse plane): stage radices, stage count, threads per line of
  // the pass's first transform and threads per CTA.
  static int tile_plan(int pass, int tile, int* radices, int* nst, int* threads_per_line, int* threads) {
    const RadixPlan pl = tile == 1 ? G1::pl : G::pl;
    *nst = pl.nst;
    for (int k = 0; k < pl.nst; ++k) radices[k] = pl.r[k];
    const bool plane = pass == 0;
    *threads_per_line = plane ? pl.tl_plane : pl.tl_colh;
    const int thr_col = pass == 1 ? G::THR_COL : G::THR_COLH, thr_col1 = pass == 1 ? G1::THR_COL : G1::THR_COLH;
    *threads = tile == 1 ? (plane ? G1::THR_PLANE : thr_col1) : (plane ? G::THR_PLANE : thr_col);
    return E1 != 0 ? 2 : 1;
  }

  static cudaError_t to_real(const DevPlan& g, const double2* psiG, int nb, int band0, int nbat,
                             void* Xv, void* psiv, cudaStream_t s) {
    C* X = static_cast<C*>(Xv);
    const int nq = (nbat + 1) / 2;
    cudaError_t err = cudaMemsetAsync(X, 0, sizeof(C) * (size_t)g.ntot * nq, s);
    if (err != cudaSuccess) return err;
    k_scatter<T><<<dim3((g.npw + 255) / 256, nq), 256, 0, s>>>(g, psiG, nb, band0, nbat, X);
    k_col_full<T, N, +1><<<dim3(N, nq), G::THR_COLF, G::SMEM_COLF, s>>>(g, X);
    k_plane_full<T, N, +1, 0, 1><<<dim3(N, nq), G::THR_PLANE, G::SMEM_PLANE, s>>>(
        g, X, nullptr, static_cast<T*>(psiv), band0, nb, nbat);
    return cudaGetLastError();
  }

  static cudaError_t pair_fwd(const DevPlan& g, const void* psi, const Chain* ch, int nch, void* H,
                              cudaStream_t s) {
    if (E1 != 0 && g.tile[0] == 1)
      k_pair_fwd<T, N, E1><<<dim3(N, nch), G1::THR_PLANE, G::SMEM_PLANE, s>>>(
          g, static_cast<const T*>(psi), ch, static_cast<C*>(H));
    else
      k_pair_fwd<T, N><<<dim3(N, nch), G::THR_PLANE, G::SMEM_PLANE, s>>>(
          g, static_cast<const T*>(psi), ch, static_cast<C*>(H));
    return cudaGetLastError();
  }

  static cudaError_t pair_col(const DevPlan& g, void* H, const Chain* ch, int nch, double* ep,
                              double* dp, cudaStream_t s) {
    if (E1 != 0 && g.tile[1] == 1)
      k_pair_col<T, N, E1><<<dim3(g.ncta_col, nch), G1::THR_COL, G::SMEM_COLH, s>>>(
          g, static_cast<C*>(H), ch, ep, dp);
    else
      k_pair_col<T, N><<<dim3(g.ncta_col, nch), G::THR_COL, G::SMEM_COLH, s>>>(
          g, static_cast<C*>(H), ch, ep, dp);
    return cudaGetLastError();
  }

  static cudaError_t pair_inv(const DevPlan& g, const void* psi, void* W, const void* occ,
                              const Chain* ch, int nch, const void* H, cudaStream_t s) {
    if (E1 != 0 && g.tile[2] == 1)
      k_pair_inv<T, N, E1><<<dim3(N, nch), G1::THR_COLH, G::SMEM_INV, s>>>(
          g, static_cast<const T*>(psi), static_cast<acc_t<T>*>(W), static_cast<const T*>(occ), ch,
          static_cast<const C*>(H));
    else
      k_pair_inv<T, N><<<dim3(N, nch), G::THR_COLH, G::SMEM_INV, s>>>(
          g, static_cast<const T*>(psi), static_cast<acc_t<T>*>(W), static_cast<const T*>(occ), ch,
          static_cast<const C*>(H));
    return cudaGetLastError();
  }

  static cudaError_t to_sphere(const DevPlan& g, const void* W, int nb, int band0, int nbat,
                               void* Xv, double2* vpsiG, cudaStream_t s) {
    C* X = static_cast<C*>(Xv);
    const int nq = (nbat + 1) / 2;
    k_plane_full<T, N, -1, 1, 0><<<dim3(N, nq), G::THR_PLANE, G::SMEM_PLANE, s>>>(
        g, X, static_cast<const acc_t<T>*>(W), nullptr, band0, nb, nbat);
    k_col_full<T, N, -1><<<dim3(N, nq), G::THR_COLF, G::SMEM_COLF, s>>>(g, X);
    k_gather<T><<<dim3((g.npw + 255) / 256, nq), 256, 0, s>>>(g, X, nb, band0, nbat, vpsiG);
    return cudaGetLastError();
  }

  static constexpr KernelOps ops() {
    return KernelOps{(int)sizeof(T), RealTraits<T>::prec, N, G::NLC,
                     smem_max(smem_max(G::SMEM_COLH, G::SMEM_PLANE), G::SMEM_INV),
                     configure, to_real, pair_fwd, pair_col, pair_inv, to_sphere, tile_plan};
  }
};

}  // namespace fockx
