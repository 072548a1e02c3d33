// Size-independent device code: the energy reduction and the table of the
// compiled (precision, grid size) kernel sets.
#include "fock_kernels.cuh"
#include "fock_sizes.h"

namespace fockx {

#define FOCK_DECLARE(N)                 \
  extern const KernelOps kOps_f64_##N; \
  extern const KernelOps kOps_f32_##N; \
  extern const KernelOps kOps_df_##N;  \
  extern const KOps kKOps_f64_##N;     \
  extern const KOps kKOps_f32_##N;
FOCK_GRID_SIZES(FOCK_DECLARE)
#undef FOCK_DECLARE

const KernelOps* find_kernel_ops(int prec, int n) {
#define FOCK_FIND(N) \
  if (n == N) return prec == 0 ? &kOps_f64_##N : prec == 1 ? &kOps_f32_##N : prec == 2 ? &kOps_df_##N : nullptr;
  FOCK_GRID_SIZES(FOCK_FIND)
#undef FOCK_FIND
  return nullptr;
}

const KOps* find_kops(int prec, int n) {
#define FOCK_FINDK(N) \
  if (n == N) return prec == 0 ? &kKOps_f64_##N : prec == 1 ? &kKOps_f32_##N : nullptr;
  FOCK_GRID_SIZES(FOCK_FINDK)
#undef FOCK_FINDK
  return nullptr;
}

extern const PersistOps kPersist_f64;
extern const PersistOps kPersist_f32;

const PersistOps* find_persist_ops(int prec) { return prec == 0 ? &kPersist_f64 : &kPersist_f32; }

bool persist_supports(int n) {
  return n == 24 || n == 32 || n == 48 || n == 64 || n == 72 || n == 96;
}

// E_x = scale * sum over the unique pairs of f_i f_j (2 if i != j) e_ij, with
// scale = -(Omega/2) / Ntot^2; summed by one CTA in a fixed order, so the
// result does not depend on launch timing.
__global__ void k_energy(const int2* __restrict__ pairs, int npairs, const double* __restrict__ occ,
                         const double* __restrict__ ep, const double* __restrict__ dp,
                         double scale, double* __restrict__ out) {
  __shared__ double red[32 * 4];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
    const int2 ij = pairs[p];
    const double w = occ[ij.x] * occ[ij.y] * (ij.x == ij.y ? 1.0 : 2.0);
    v[0] += w * ep[p];
    if (dp) v[1] += w * dp[p];
  }
  block_sum4(v, red);
  if (threadIdx.x == 0) {
    out[0] = scale * v[0];
    out[1] = scale * v[1];
  }
}

// ------------------------------------------------ deterministic accumulation

template <class T>
__global__ void k_orbital_stats(const T* __restrict__ psi, int64_t ntot, double* __restrict__ stats) {
  __shared__ double red[32 * 4];
  const T* p = psi + (int64_t)blockIdx.x * ntot;
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // max |x|, sum x^2
  for (int64_t e = threadIdx.x; e < ntot; e += blockDim.x) {
    const double x = to_double(p[e]);
    v[0] = fmax(v[0], fabs(x));
    v[1] += x * x;
  }
  // max over the CTA: warp shuffles then one pass over the warps
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v[0] = fmax(v[0], __shfl_down_sync(0xffffffffu, v[0], o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v[0];
  __syncthreads();
  double m = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
  __syncthreads();
  v[0] = 0.0;
  block_sum4(v, red);
  if (threadIdx.x == 0) {
    stats[2 * blockIdx.x] = m;
    stats[2 * blockIdx.x + 1] = v[1];
  }
}

// B = vnorm / sqrt(Ntot) * max_t ||psi_t||_2 * sum_{s < nsrc} |f_s| max|psi_s|^2 bounds
// every partial sum of an accumulator; the scale 2^s keeps 4 B 2^s < 2^63.
__global__ void k_det_scale(const double* __restrict__ stats, int nbands, const double* __restrict__ occ,
                            int nsrc, double vnorm, int64_t ntot, double* __restrict__ scale) {
  double a = 0.0, t2 = 0.0;
  for (int b = 0; b < nbands; ++b) {
    if (b < nsrc) a += fabs(occ[b]) * stats[2 * b] * stats[2 * b];
    t2 = fmax(t2, stats[2 * b + 1]);
  }
  const double bound = vnorm / sqrt((double)ntot) * sqrt(t2) * a * (1.0 + 1e-6);
  int ex = 0;
  if (bound > 0.0) {
    frexp(bound, &ex);  // bound < 2^ex
  }
  const int s = bound > 0.0 ? 61 - ex : 0;  // 4 * bound * 2^s < 2^63
  scale[0] = ldexp(1.0, s);
  scale[1] = ldexp(1.0, -s);
}

__global__ void k_det_to_double(long long* __restrict__ w, int64_t n, const double* __restrict__ scale) {
  const double inv = scale[1];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)w[e] * inv;
    w[e] = __double_as_longlong(x);
  }
}

__global__ void k_det_pair_sums(const double* __restrict__ part, int npairs, int ncta, double* __restrict__ out) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < ncta; ++c) s += part[(int64_t)p * ncta + c];
    out[p] = s;
  }
}

cudaError_t launch_orbital_stats(int prec, const void* psi, int nbands, int64_t ntot, double* stats,
                                 cudaStream_t s) {
  if (prec == 0)
    k_orbital_stats<double><<<nbands, 512, 0, s>>>(static_cast<const double*>(psi), ntot, stats);
  else if (prec == 2)
    k_orbital_stats<df64><<<nbands, 512, 0, s>>>(static_cast<const df64*>(psi), ntot, stats);
  else
    k_orbital_stats<float><<<nbands, 512, 0, s>>>(static_cast<const float*>(psi), ntot, stats);
  return cudaGetLastError();
}

cudaError_t launch_det_scale(const double* stats, int nbands, const double* occ, int nsrc, double vnorm,
                             int64_t ntot, double* scale, cudaStream_t s) {
  k_det_scale<<<1, 1, 0, s>>>(stats, nbands, occ, nsrc, vnorm, ntot, scale);
  return cudaGetLastError();
}

cudaError_t launch_det_to_double(void* w, int64_t n, const double* scale, cudaStream_t s) {
  k_det_to_double<<<1216, 256, 0, s>>>(static_cast<long long*>(w), n, scale);
  return cudaGetLastError();
}

cudaError_t launch_det_pair_sums(const double* part, int npairs, int ncta, double* out, cudaStream_t s) {
  if (npairs < 1) return cudaSuccess;
  k_det_pair_sums<<<(npairs + 255) / 256, 256, 0, s>>>(part, npairs, ncta, out);
  return cudaGetLastError();
}

#define FOCK_OV_CHECK(call)             \
  do {                                  \
    const cudaError_t e_ = (call);      \
    if (e_ != cudaSuccess) return e_;   \
  } while (0)

namespace {

// Overlap tiles: TB x TB entries of S per CTA (16 x 16 threads, each
// TB/16 x TB/16 entries 16 apart; TB = 64, or 32 for matrices of at most 32
// rows), the sum over the real views of the rows split into chunks over
// gridDim.y and reduced with FP64 atomics.
constexpr int kOvK = 16, kOvThreads = 256;

// K: terms of the sum (real-view entries); with `half`, entry k is component
// k & 1 of sphere position half[k >> 1] (weight 2, weight 1 for k < 2: the
// list's first position is G = 0), else entry k of the row; rows are RS doubles.
template <int TB>
__global__ void __launch_bounds__(kOvThreads)
    k_overlap(const double* __restrict__ A, int na, const double* __restrict__ B, int nbb, int64_t K, int64_t RS,
              const int* __restrict__ half, int sym, int tiles_j, int64_t kchunk, double* __restrict__ S, int ld) {
  constexpr int MT = TB / 16;
  int ti, tj;
  if (sym) {  // blockIdx.x enumerates the tiles ti <= tj row by row
    int rem = blockIdx.x;
    ti = 0;
    while (rem >= tiles_j - ti) {
      rem -= tiles_j - ti;
      ++ti;
    }
    tj = ti + rem;
  } else {
    ti = blockIdx.x / tiles_j;
    tj = blockIdx.x - ti * tiles_j;
  }
  const int i0 = ti * TB, j0 = tj * TB;
  const int64_t k0 = (int64_t)blockIdx.y * kchunk;
  const int64_t k1 = k0 + kchunk < K ? k0 + kchunk : K;
  __shared__ double As[kOvK][TB + 1], Bs[kOvK][TB + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[MT][MT];
#pragma unroll
  for (int u = 0; u < MT; ++u)
#pragma unroll
    for (int v = 0; v < MT; ++v) acc[u][v] = 0.0;
  for (int64_t kb = k0; kb < k1; kb += kOvK) {
    for (int e = threadIdx.x; e < TB * kOvK; e += kOvThreads) {
      const int r = e / kOvK, kk = e - r * kOvK;
      const int64_t k = kb + kk;
      double a = 0.0, b = 0.0;
      if (k < k1) {
        int64_t c = k;
        double w = 1.0;
        if (half != nullptr) {
          c = 2 * (int64_t)half[k >> 1] + (k & 1);
          w = k < 2 ? 1.0 : 2.0;
        }
        if (i0 + r < na) a = w * A[(int64_t)(i0 + r) * RS + c];
        if (j0 + r < nbb) b = B[(int64_t)(j0 + r) * RS + c];
      }
      As[kk][r] = a;
      Bs[kk][r] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kOvK; ++kk) {
      double a[MT], b[MT];
#pragma unroll
      for (int u = 0; u < MT; ++u) {
        a[u] = As[kk][ty + 16 * u];
        b[u] = Bs[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < MT; ++u)
#pragma unroll
        for (int v = 0; v < MT; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < MT; ++u)
#pragma unroll
    for (int v = 0; v < MT; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < na && j < nbb && (!sym || j >= i)) atomicAdd(&S[(int64_t)i * ld + j], acc[u][v]);
    }
}

__global__ void k_overlap_zero(double* S, int na, int nbb, int sym, int ld) {
  const int64_t total = (int64_t)na * nbb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / nbb), j = (int)(e - (int64_t)i * nbb);
    if (!sym || j >= i) S[(int64_t)i * ld + j] = 0.0;
  }
}

}  // namespace

namespace {
__global__ void k_scaled_table(const double* __restrict__ v, int64_t n, double factor, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = factor * v[i];
}
}  // namespace

cudaError_t launch_scaled_table(const double* v, int64_t n, double factor, double* out, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_scaled_table<<<(int)(blocks < 1216 ? blocks : 1216), 256, 0, s>>>(v, n, factor, out);
  return cudaGetLastError();
}

namespace {
cudaError_t overlap_impl(const double2* a, int na, const double2* b, int nbb, int npw, const int* half, int nhalf,
                         bool sym, double* S, int ld, cudaStream_t s);

// Complex overlaps of nsets row sets (set z: rows[z], nb rows of npw[z]
// complex128) with themselves, upper triangles: Sre/Sim[z][i][j] =
// Re/Im sum_G conj(c_i(G)) c_j(G), j >= i.  32 x 32 tiles (16 x 16 threads,
// 2 x 2 entries each, real and imaginary parts from the same loads), the
// sum split into gridDim.y chunks of kchunk complex terms, FP64 atomics.
__global__ void __launch_bounds__(kOvThreads)
    k_overlap_sets(const double2* const* __restrict__ rows, const int* __restrict__ npw, int nb, int tiles_j,
                   int kchunk, double* __restrict__ Sre, double* __restrict__ Sim) {
  constexpr int TB = 32, KC = 16;
  const int z = blockIdx.z;
  int rem = blockIdx.x, ti = 0;
  while (rem >= tiles_j - ti) {
    rem -= tiles_j - ti;
    ++ti;
  }
  const int tj = ti + rem;
  const int i0 = ti * TB, j0 = tj * TB;
  const double2* R = rows[z];
  const int K = npw[z];
  const int k0 = blockIdx.y * kchunk;
  const int k1 = k0 + kchunk < K ? k0 + kchunk : K;
  __shared__ double2 As[KC][TB + 1], Bs[KC][TB + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double re[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, im[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int kb = k0; kb < k1; kb += KC) {
    for (int e = threadIdx.x; e < TB * KC; e += kOvThreads) {
      const int r = e / KC, kk = e - r * KC;
      const int k = kb + kk;
      const double2 zero = make_double2(0.0, 0.0);
      As[kk][r] = (k < k1 && i0 + r < nb) ? R[(int64_t)(i0 + r) * K + k] : zero;
      Bs[kk][r] = (k < k1 && j0 + r < nb) ? R[(int64_t)(j0 + r) * K + k] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      double2 a[2], b[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        a[u] = As[kk][ty + 16 * u];
        b[u] = Bs[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          re[u][v] = fma(a[u].x, b[v].x, fma(a[u].y, b[v].y, re[u][v]));
          im[u][v] = fma(a[u].x, b[v].y, fma(-a[u].y, b[v].x, im[u][v]));
        }
    }
    __syncthreads();
  }
  const int64_t off = (int64_t)z * nb * nb;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < nb && j < nb && j >= i) {
        atomicAdd(&Sre[off + (int64_t)i * nb + j], re[u][v]);
        atomicAdd(&Sim[off + (int64_t)i * nb + j], im[u][v]);
      }
    }
}
}  // namespace

cudaError_t launch_overlap_sets(const double2* const* rows, const int* npw, int npw_max, int nsets, int nb,
                                double* Sre, double* Sim, cudaStream_t s) {
  if (nsets < 1 || nb < 1) return cudaSuccess;
  FOCK_OV_CHECK(cudaMemsetAsync(Sre, 0, sizeof(double) * (size_t)nsets * nb * nb, s));
  FOCK_OV_CHECK(cudaMemsetAsync(Sim, 0, sizeof(double) * (size_t)nsets * nb * nb, s));
  const int tj = (nb + 31) / 32, tiles = tj * (tj + 1) / 2;
  // chunks: two CTAs per SM over all sets, each chunk at least 4 k-blocks,
  // at most 64 chunks adding into one entry
  int splits = (2 * 152 + tiles * nsets - 1) / (tiles * nsets);
  const int max_splits = (npw_max + 63) / 64;
  if (splits > max_splits) splits = max_splits;
  if (splits > 64) splits = 64;
  if (splits < 1) splits = 1;
  int kchunk = (npw_max + splits - 1) / splits;
  kchunk = (kchunk + 15) / 16 * 16;
  splits = (npw_max + kchunk - 1) / kchunk;
  k_overlap_sets<<<dim3(tiles, splits, nsets), kOvThreads, 0, s>>>(rows, npw, nb, tj, kchunk, Sre, Sim);
  return cudaGetLastError();
}

cudaError_t launch_overlap(const double2* a, int na, const double2* b, int nbb, int npw, const int* half,
                           int nhalf, bool sym, double* S, int ld, cudaStream_t s) {
  return overlap_impl(a, na, b, nbb, npw, half, nhalf, sym, S, ld, s);
}


namespace {
cudaError_t overlap_impl(const double2* a, int na, const double2* b, int nbb, int npw, const int* half, int nhalf,
                         bool sym, double* S, int ld, cudaStream_t s) {
  if (na < 1 || nbb < 1) return cudaSuccess;
  const int64_t RS = 2 * (int64_t)npw;                        // the real view of a row
  const int64_t K = half != nullptr ? 2 * (int64_t)nhalf : RS;  // terms of the sum
  const int TB = (na <= 32 && nbb <= 32) ? 32 : 64;
  const int ti = (na + TB - 1) / TB, tj = (nbb + TB - 1) / TB;
  const int tiles = sym ? tj * (tj + 1) / 2 : ti * tj;
  // chunks of the sum: at least two CTAs per SM (152 SMs) and among up to
  // four times that many the count whose CTAs fill their last wave over the
  // SMs best (the FP64 pipe is the bound, so an SM with one CTA more than the
  // others sets the time); each chunk at least 4 k-blocks, and at most two
  // CTAs per SM add into one entry (a few hundred FP64 atomics an entry, at
  // the end of each CTA's chunk, cost microseconds against its sum)
  constexpr int kSMs = 152;
  int64_t max_splits = (K + 4 * kOvK - 1) / (4 * kOvK);
  if (max_splits > 2 * kSMs) max_splits = 2 * kSMs;
  int s0 = (2 * kSMs + tiles - 1) / tiles;
  if (s0 > max_splits) s0 = (int)max_splits;
  if (s0 < 1) s0 = 1;
  int splits = s0;
  double best = -1.0;
  for (int c = s0; c <= 4 * s0 && c <= max_splits; ++c) {
    const int64_t ctas = (int64_t)tiles * c;
    const double fill = (double)ctas / (double)(((ctas + kSMs - 1) / kSMs) * kSMs);
    if (fill > best + 1e-9) {
      best = fill;
      splits = c;
    }
  }
  int64_t kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + kOvK - 1) / kOvK * kOvK;
  splits = (int)((K + kchunk - 1) / kchunk);
  const int64_t entries = (int64_t)na * nbb;
  k_overlap_zero<<<(int)((entries + 255) / 256 < 1216 ? (entries + 255) / 256 : 1216), 256, 0, s>>>(S, na, nbb,
                                                                                                sym ? 1 : 0, ld);
  const double* A = reinterpret_cast<const double*>(a);
  const double* B = reinterpret_cast<const double*>(b);
  if (TB == 32)
    k_overlap<32><<<dim3(tiles, splits), kOvThreads, 0, s>>>(A, na, B, nbb, K, RS, half, sym ? 1 : 0, tj, kchunk,
                                                            S, ld);
  else
    k_overlap<64><<<dim3(tiles, splits), kOvThreads, 0, s>>>(A, na, B, nbb, K, RS, half, sym ? 1 : 0, tj, kchunk,
                                                            S, ld);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_energy_reduce(const int2* pairs, int npairs, const double* occ,
                                 const double* epair, const double* dpair, double scale,
                                 double* out, cudaStream_t s) {
  k_energy<<<1, 1024, 0, s>>>(pairs, npairs, occ, epair, dpair, scale, out);
  return cudaGetLastError();
}

}  // namespace fockx
