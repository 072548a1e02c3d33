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

cudaError_t launch_energy_reduce(const int2* pairs, int npairs, const double* occ,
                                 const double* epair, const double* dpair, double scale,
                                 double* out, cudaStream_t s) {
  k_energy<<<1, 1024, 0, s>>>(pairs, npairs, occ, epair, dpair, scale, out);
  return cudaGetLastError();
}

}  // namespace fockx
