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

cudaError_t launch_energy_reduce(const int2* pairs, int npairs, const double* occ,
                                 const double* epair, const double* dpair, double scale,
                                 double* out, cudaStream_t s) {
  k_energy<<<1, 1024, 0, s>>>(pairs, npairs, occ, epair, dpair, scale, out);
  return cudaGetLastError();
}

}  // namespace fockx
