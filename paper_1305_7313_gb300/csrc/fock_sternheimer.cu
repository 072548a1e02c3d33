// fock_sternheimer.cu — kernels of the Sternheimer CG (§3.1): the local
// potential in real space, per-band inner products on the plane-wave sphere,
// the occupied-manifold projector, the CG vector updates and the regrouping
// gathers.  All in FP64 on complex128 kets [m][npw] (Gamma-point real
// functions, so every inner product <a|b> = sum_G conj(a(G)) b(G) is real).
// The transforms of the kets to real space and back are the plan's own.
#include "fock_internal.h"

namespace fockx {
namespace {

constexpr int kThreads = 256;

// Sum of one double over the CTA; the result is valid in thread 0.
__device__ double block_sum(double v) {
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
  return s;
}

// w[n][r] = v[r] psi[n][r] for the first m bands (grid-stride over all points).
__global__ void k_vmul(const double* __restrict__ v, const double* __restrict__ psi, double* __restrict__ w,
                       int m, int64_t ntot) {
  const int64_t total = (int64_t)m * ntot;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = v[i % ntot] * psi[i];
}

// out[n] = Re sum_G conj(a_n(G)) b_n(G), one CTA per band.
__global__ void k_dots(const double2* __restrict__ a, const double2* __restrict__ b, int npw, double* __restrict__ out) {
  const double2* an = a + (int64_t)blockIdx.x * npw;
  const double2* bn = b + (int64_t)blockIdx.x * npw;
  double s = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) s += an[g].x * bn[g].x + an[g].y * bn[g].y;
  s = block_sum(s);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// c[n * nocc + i] = Re sum_G conj(u_i(G)) x_n(G); CTA (i, n).
__global__ void k_proj_coef(const double2* __restrict__ u, int nocc, const double2* __restrict__ x, int npw,
                            double* __restrict__ c) {
  const int i = blockIdx.x, n = blockIdx.y;
  const double2* ui = u + (int64_t)i * npw;
  const double2* xn = x + (int64_t)n * npw;
  double s = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) s += ui[g].x * xn[g].x + ui[g].y * xn[g].y;
  s = block_sum(s);
  if (threadIdx.x == 0) c[n * nocc + i] = s;
}

// b_n = -(w_n - sum_i c_ni u_i) = -Q w_n.
__global__ void k_rhs(const double2* __restrict__ w, const double2* __restrict__ u, const double* __restrict__ c,
                      int nocc, int m, int npw, double2* __restrict__ b) {
  const int64_t total = (int64_t)m * npw;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(k / npw), g = (int)(k - (int64_t)n * npw);
    double2 s = w[k];
    for (int i = 0; i < nocc; ++i) {
      const double ci = c[n * nocc + i];
      const double2 ui = u[(int64_t)i * npw + g];
      s.x -= ci * ui.x;
      s.y -= ci * ui.y;
    }
    b[k] = make_double2(-s.x, -s.y);
  }
}

// ap_n = ap_n + (|G|^2/2 - eps_n) p_n + alpha sum_i c_ni u_i, where ap holds
// the local-potential part of H p on entry: ap = (H - eps_n + alpha P) p.
__global__ void k_finish(double2* __restrict__ ap, const double2* __restrict__ p, const double* __restrict__ kin,
                         const double* __restrict__ eps, const double2* __restrict__ u, const double* __restrict__ c,
                         int nocc, double alpha, int m, int npw) {
  const int64_t total = (int64_t)m * npw;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(k / npw), g = (int)(k - (int64_t)n * npw);
    const double d = kin[g] - eps[n];
    double2 s = ap[k];
    const double2 pk = p[k];
    s.x += d * pk.x;
    s.y += d * pk.y;
    for (int i = 0; i < nocc; ++i) {
      const double ci = alpha * c[n * nocc + i];
      const double2 ui = u[(int64_t)i * npw + g];
      s.x += ci * ui.x;
      s.y += ci * ui.y;
    }
    ap[k] = s;
  }
}

// x_n += a_n p_n, r_n -= a_n ap_n with a_n = rr_n / pap_n.
__global__ void k_step(double2* __restrict__ x, double2* __restrict__ r, const double2* __restrict__ p,
                       const double2* __restrict__ ap, const double* __restrict__ rr, const double* __restrict__ pap,
                       int m, int npw) {
  const int64_t total = (int64_t)m * npw;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(k / npw);
    const double a = rr[n] / pap[n];
    const double2 pk = p[k], ak = ap[k];
    x[k].x += a * pk.x;
    x[k].y += a * pk.y;
    r[k].x -= a * ak.x;
    r[k].y -= a * ak.y;
  }
}

// p_n = r_n + (rr_new_n / rr_n) p_n.
__global__ void k_dir(double2* __restrict__ p, const double2* __restrict__ r, const double* __restrict__ rr_new,
                      const double* __restrict__ rr, int m, int npw) {
  const int64_t total = (int64_t)m * npw;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(k / npw);
    const double beta = rr_new[n] / rr[n];
    const double2 rk = r[k], pk = p[k];
    p[k] = make_double2(rk.x + beta * pk.x, rk.y + beta * pk.y);
  }
}

// dst[k] = src[perm[k]] for ket arrays (rows of npw) and for per-band scalars.
__global__ void k_gather_rows(const double2* __restrict__ src, double2* __restrict__ dst, const int* __restrict__ perm,
                              int m, int npw) {
  const int64_t total = (int64_t)m * npw;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(k / npw), g = (int)(k - (int64_t)n * npw);
    dst[k] = src[(int64_t)perm[n] * npw + g];
  }
}
__global__ void k_gather_scalars(const double* __restrict__ src, double* __restrict__ dst,
                                 const int* __restrict__ perm, int m) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < m; n += gridDim.x * blockDim.x) dst[n] = src[perm[n]];
}

int grid_for(int64_t total) {
  const int64_t b = (total + kThreads - 1) / kThreads;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

cudaError_t st_vmul(const double* v, const double* psi, double* w, int m, int64_t ntot, cudaStream_t s) {
  k_vmul<<<grid_for((int64_t)m * ntot), kThreads, 0, s>>>(v, psi, w, m, ntot);
  return cudaGetLastError();
}
cudaError_t st_dots(const double2* a, const double2* b, int m, int npw, double* out, cudaStream_t s) {
  k_dots<<<m, kThreads, 0, s>>>(a, b, npw, out);
  return cudaGetLastError();
}
cudaError_t st_proj_coef(const double2* u, int nocc, const double2* x, int m, int npw, double* c, cudaStream_t s) {
  k_proj_coef<<<dim3(nocc, m), kThreads, 0, s>>>(u, nocc, x, npw, c);
  return cudaGetLastError();
}
cudaError_t st_rhs(const double2* w, const double2* u, const double* c, int nocc, int m, int npw, double2* b,
                   cudaStream_t s) {
  k_rhs<<<grid_for((int64_t)m * npw), kThreads, 0, s>>>(w, u, c, nocc, m, npw, b);
  return cudaGetLastError();
}
cudaError_t st_finish(double2* ap, const double2* p, const double* kin, const double* eps, const double2* u,
                      const double* c, int nocc, double alpha, int m, int npw, cudaStream_t s) {
  k_finish<<<grid_for((int64_t)m * npw), kThreads, 0, s>>>(ap, p, kin, eps, u, c, nocc, alpha, m, npw);
  return cudaGetLastError();
}
cudaError_t st_step(double2* x, double2* r, const double2* p, const double2* ap, const double* rr, const double* pap,
                    int m, int npw, cudaStream_t s) {
  k_step<<<grid_for((int64_t)m * npw), kThreads, 0, s>>>(x, r, p, ap, rr, pap, m, npw);
  return cudaGetLastError();
}
cudaError_t st_dir(double2* p, const double2* r, const double* rr_new, const double* rr, int m, int npw,
                   cudaStream_t s) {
  k_dir<<<grid_for((int64_t)m * npw), kThreads, 0, s>>>(p, r, rr_new, rr, m, npw);
  return cudaGetLastError();
}
cudaError_t st_gather_rows(const double2* src, double2* dst, const int* perm, int m, int npw, cudaStream_t s) {
  k_gather_rows<<<grid_for((int64_t)m * npw), kThreads, 0, s>>>(src, dst, perm, m, npw);
  return cudaGetLastError();
}
cudaError_t st_gather_scalars(const double* src, double* dst, const int* perm, int m, cudaStream_t s) {
  k_gather_scalars<<<1, kThreads, 0, s>>>(src, dst, perm, m);
  return cudaGetLastError();
}

}  // namespace fockx
