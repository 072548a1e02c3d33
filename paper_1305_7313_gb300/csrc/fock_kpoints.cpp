// fock_kpoints.cpp — host side of the Brillouin-zone-sampled apply
// (fock_kplan_* in include/fock.h): per-k plane-wave spheres, the table of
// v(G + q) for every distinct q = k_b - k_a, the pair schedule over states
// (k, n), and the orchestration of the complex pass kernels.
//
// Built with -ffp-contract=off (see fock_lattice.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fock.h"
#include "fock_internal.h"
#include "fock_lattice.h"

using fockx::Chain;
using fockx::DevPlan;

namespace {

constexpr int kBandBlock = 16;
constexpr size_t kBufferBytes = size_t(120) << 20;
thread_local std::string g_kcreate_error;

}  // namespace

struct fock_kplan {
  int device = 0;
  int n = 0;
  double cell[9];
  double recip[9];
  double vol = 0.0;
  double ecut = 0.0;
  fock_kernel kind = FOCK_KERNEL_SPENCER_ALAVI;
  double omega = 0.0;
  fock_precision prec = FOCK_PREC_FP64;
  int nk = 0;
  std::vector<double> kfrac, wk;
  std::vector<std::vector<int32_t>> miller;
  std::vector<int> npw;
  std::vector<int*> d_gidx;
  int nq = 0;
  std::vector<int> qidx;  // [ka * nk + kb] -> distinct q = k_b - k_a
  void* d_vq = nullptr;
  double* d_vq64 = nullptr;
  float* d_qfrac = nullptr;  // [nq][3] q in reduced coordinates (mixed form)
  // mixed form: FP64 overlaps of the states of each k point (q = 0 pairs' G = 0)
  double* d_kovl = nullptr;  // [2][nk][nb][nb]: real parts, then imaginary parts
  int64_t kovl_cap = 0;
  const double2** d_krows = nullptr;  // [nk] the orbital arrays of an apply
  int* d_knpw = nullptr;              // [nk] sphere sizes
  int npw_max = 0;
  void* d_tw = nullptr;
  const fockx::KernelOps* ops = nullptr;
  const fockx::KOps* kops = nullptr;
  DevPlan dp{};
  int chain_batch = 1;
  // workspace
  int ns_cap = 0;
  void* d_u = nullptr;
  void* d_w = nullptr;
  void* d_h = nullptr;
  int npair_cap = 0;
  double* d_epair = nullptr;
  int2* d_pairs = nullptr;
  Chain* d_chains = nullptr;
  double* d_occw = nullptr;
  void* d_occwT = nullptr;
  double* d_result = nullptr;
  double* h_result = nullptr;
  int sched_ns = -1;
  int sched_nb = -1;
  std::vector<int2> pairs;
  std::vector<Chain> chains;
  std::string err;
};

namespace {

fock_status kfail(fock_kplan* p, fock_status s, const std::string& msg) {
  if (p) p->err = msg;
  else g_kcreate_error = msg;
  return s;
}

fock_status kcuda(fock_kplan* p, cudaError_t e, const char* what) {
  cudaGetLastError();
  return kfail(p, e == cudaErrorMemoryAllocation ? FOCK_ERR_OOM : FOCK_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define FOCK_KCUDA(p, call)                             \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return kcuda(p, e_, #call);  \
  } while (0)

size_t csz(const fock_kplan* p) { return 2 * (size_t)p->ops->real_bytes; }

void kfree_ws(fock_kplan* p) {
  cudaFree(p->d_u);
  cudaFree(p->d_w);
  cudaFree(p->d_h);
  cudaFree(p->d_epair);
  cudaFree(p->d_pairs);
  cudaFree(p->d_chains);
  cudaFree(p->d_occw);
  cudaFree(p->d_occwT);
  p->d_u = p->d_w = p->d_h = p->d_occwT = nullptr;
  p->d_epair = p->d_occw = nullptr;
  p->d_pairs = nullptr;
  p->d_chains = nullptr;
  p->ns_cap = p->npair_cap = 0;
}

fock_status kensure(fock_kplan* p, int ns, int npairs) {
  const size_t grid_bytes = (size_t)p->dp.ntot * csz(p);
  if (ns > p->ns_cap) {
    cudaFree(p->d_u);
    cudaFree(p->d_w);
    cudaFree(p->d_occw);
    cudaFree(p->d_occwT);
    p->d_u = p->d_w = p->d_occwT = nullptr;
    p->d_occw = nullptr;
    p->ns_cap = 0;
    FOCK_KCUDA(p, cudaMalloc(&p->d_u, grid_bytes * ns));
    FOCK_KCUDA(p, cudaMalloc(&p->d_w, grid_bytes * ns));
    FOCK_KCUDA(p, cudaMalloc((void**)&p->d_occw, sizeof(double) * ns));
    FOCK_KCUDA(p, cudaMalloc(&p->d_occwT, (size_t)p->ops->real_bytes * ns));
    p->ns_cap = ns;
  }
  if (!p->d_h) FOCK_KCUDA(p, cudaMalloc(&p->d_h, grid_bytes * p->chain_batch));
  if (npairs > p->npair_cap) {
    cudaFree(p->d_epair);
    cudaFree(p->d_pairs);
    cudaFree(p->d_chains);
    p->d_epair = nullptr;
    p->d_pairs = nullptr;
    p->d_chains = nullptr;
    p->npair_cap = 0;
    p->sched_ns = -1;
    FOCK_KCUDA(p, cudaMalloc((void**)&p->d_epair, sizeof(double) * npairs));
    FOCK_KCUDA(p, cudaMalloc((void**)&p->d_pairs, sizeof(int2) * npairs));
    FOCK_KCUDA(p, cudaMalloc((void**)&p->d_chains, sizeof(Chain) * npairs));
    p->npair_cap = npairs;
  }
  return FOCK_OK;
}

}  // namespace

extern "C" {

fock_status fock_kplan_create(fock_kplan_t* out, const int grid[3], const double cell[9], double ecut_ha,
                              int nk, const double* kpts, const double* wk, fock_kernel kind,
                              const double* kparams, int nkparams, fock_precision prec) {
  g_kcreate_error.clear();
  if (!out) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !cell || !kpts || !wk || nk < 1 || nk > 4096)
    return kfail(nullptr, FOCK_ERR_INVALID_ARG, "NULL argument or nk out of range");
  if (prec != FOCK_PREC_FP64 && prec != FOCK_PREC_MIXED32)
    return kfail(nullptr, FOCK_ERR_INVALID_ARG, "k-point plans run the FP64 and mixed forms only");
  if (kind != FOCK_KERNEL_SPENCER_ALAVI && kind != FOCK_KERNEL_ERFC)
    return kfail(nullptr, FOCK_ERR_INVALID_ARG, "unknown kernel kind");
  if (!(ecut_ha > 0.0) || !std::isfinite(ecut_ha)) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "bad ecut");
  double omega = 0.0;
  if (kind == FOCK_KERNEL_ERFC) {
    if (!kparams || nkparams < 1 || !(kparams[0] > 0.0) || !std::isfinite(kparams[0]))
      return kfail(nullptr, FOCK_ERR_INVALID_ARG, "erfc kernel needs kparams = {omega > 0}");
    omega = kparams[0];
  }
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(cell[i])) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "cell is not finite");
  for (int i = 0; i < 3 * nk; ++i)
    if (!std::isfinite(kpts[i])) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "k points are not finite");
  for (int i = 0; i < nk; ++i)
    if (!std::isfinite(wk[i])) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "weights are not finite");
  if (grid[0] != grid[1] || grid[1] != grid[2])
    return kfail(nullptr, FOCK_ERR_UNSUPPORTED_SIZE, "the FFT grid must be cubic (N1 = N2 = N3)");
  const int n = grid[0];
  const fockx::KernelOps* ops = fockx::find_kernel_ops(prec == FOCK_PREC_FP64 ? 0 : 1, n);
  const fockx::KOps* kops = fockx::find_kops(prec == FOCK_PREC_FP64 ? 0 : 1, n);
  if (!ops || !kops) return kfail(nullptr, FOCK_ERR_UNSUPPORTED_SIZE, "no kernels compiled for this N");

  fock_kplan* p = new (std::nothrow) fock_kplan();
  if (!p) return kfail(nullptr, FOCK_ERR_OOM, "host allocation failed");
  auto bail = [&](fock_status st) {
    g_kcreate_error = p->err;
    fock_kplan_destroy(p);
    return st;
  };
  std::memcpy(p->cell, cell, sizeof(p->cell));
  p->n = n;
  p->ecut = ecut_ha;
  p->kind = kind;
  p->omega = omega;
  p->prec = prec;
  p->ops = ops;
  p->kops = kops;
  p->nk = nk;
  p->kfrac.assign(kpts, kpts + 3 * nk);
  p->wk.assign(wk, wk + nk);
  const double vs = fockx::lattice::reciprocal(cell, p->recip);
  if (!(std::fabs(vs) > 0.0)) return bail(kfail(p, FOCK_ERR_INVALID_ARG, "the cell is degenerate"));
  p->vol = std::fabs(vs);

  // one sphere per k point (host only: a grid is refused before any CUDA call)
  const int64_t ntot = (int64_t)n * n * n;
  auto off = [n](int m1, int m2, int m3) {
    return ((((m1 % n) + n) % n) * n + (((m2 % n) + n) % n)) * n + (((m3 % n) + n) % n);
  };
  std::vector<fockx::lattice::GEntry> sph;
  std::vector<int> mlo((size_t)3 * nk), mhi((size_t)3 * nk);
  for (int k = 0; k < nk; ++k) {
    if (!fockx::lattice::build_sphere(cell, p->recip, ecut_ha, n, sph, &p->kfrac[3 * k]))
      return bail(kfail(p, FOCK_ERR_GRID_TOO_SMALL, "a G-sphere does not fit on the grid"));
    std::vector<int32_t> mill(3 * sph.size());
    for (int a = 0; a < 3; ++a) {
      mlo[3 * k + a] = 0;
      mhi[3 * k + a] = 0;
    }
    for (size_t g = 0; g < sph.size(); ++g) {
      for (int a = 0; a < 3; ++a) {
        mill[3 * g + a] = sph[g].m[a];
        mlo[3 * k + a] = std::min(mlo[3 * k + a], sph[g].m[a]);
        mhi[3 * k + a] = std::max(mhi[3 * k + a], sph[g].m[a]);
      }
    }
    p->miller.push_back(mill);
    p->npw.push_back((int)sph.size());
  }
  // The pair kernels evaluate each unique pair of states once and take the
  // reverse pair's potential as the complex conjugate.  That equals the plain
  // sum over ordered pairs exactly when no pair density u_a* u_b has a
  // component on a Nyquist plane (frequency -N/2 of an even axis): there the
  // partner frequency +N/2 is the same grid point, so the reverse pair would
  // see the kernel at another |G + q|.  The frequencies of u_a* u_b are the
  // differences m_b - m_a of the two spheres, so every pair of k points
  // (k = k' included) must keep max m_b - min m_a below N/2 on every axis.
  if (n % 2 == 0)
    for (int ka = 0; ka < nk; ++ka)
      for (int kb = 0; kb < nk; ++kb)
        for (int a = 0; a < 3; ++a)
          if (2 * (mhi[3 * kb + a] - mlo[3 * ka + a]) >= n)
            return bail(kfail(p, FOCK_ERR_GRID_TOO_SMALL,
                              "the pair densities reach the Nyquist frequency -N/2 of the grid "
                              "(need N > 2 (max m - min m') over every pair of spheres)"));
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) return bail(kcuda(p, e, "cudaGetDevice"));
  for (int k = 0; k < nk; ++k) {
    const std::vector<int32_t>& mill = p->miller[k];
    std::vector<int> gidx(mill.size() / 3);
    for (size_t g = 0; g < gidx.size(); ++g) gidx[g] = off(mill[3 * g], mill[3 * g + 1], mill[3 * g + 2]);
    int* d = nullptr;
    if ((e = cudaMalloc((void**)&d, sizeof(int) * std::max<size_t>(1, gidx.size()))) != cudaSuccess)
      return bail(kcuda(p, e, "cudaMalloc"));
    p->d_gidx.push_back(d);
    if ((e = cudaMemcpy(d, gidx.data(), sizeof(int) * gidx.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(kcuda(p, e, "cudaMemcpy"));
  }

  // distinct q = k_b - k_a and their kernel tables on the full grid
  std::vector<double> qs;
  p->qidx.assign((size_t)nk * nk, 0);
  for (int ka = 0; ka < nk; ++ka)
    for (int kb = 0; kb < nk; ++kb) {
      double q[3];
      for (int a = 0; a < 3; ++a) q[a] = p->kfrac[3 * kb + a] - p->kfrac[3 * ka + a];
      int found = -1;
      for (size_t j = 0; j * 3 < qs.size(); ++j)
        if (qs[3 * j] == q[0] && qs[3 * j + 1] == q[1] && qs[3 * j + 2] == q[2]) found = (int)j;
      if (found < 0) {
        found = (int)(qs.size() / 3);
        qs.insert(qs.end(), q, q + 3);
      }
      p->qidx[(size_t)ka * nk + kb] = found;
    }
  p->nq = (int)(qs.size() / 3);
  const bool fp64 = ops->real_bytes == 8;
  std::vector<double> v64((size_t)p->nq * ntot);
  for (int j = 0; j < p->nq; ++j)
    for (int k1 = 0; k1 < n; ++k1)
      for (int k2 = 0; k2 < n; ++k2)
        for (int k3 = 0; k3 < n; ++k3) {
          const double g2 = fockx::lattice::g2_of(p->recip, fockx::lattice::freq_of(k1, n),
                                                  fockx::lattice::freq_of(k2, n), fockx::lattice::freq_of(k3, n),
                                                  &qs[3 * j]);
          double v, dv;
          fockx::lattice::kernel_value(kind, p->vol, omega, g2, &v, &dv);
          v64[(size_t)j * ntot + ((size_t)k1 * n + k2) * n + k3] = v;
        }
  if ((e = cudaMalloc((void**)&p->d_vq64, sizeof(double) * v64.size())) != cudaSuccess ||
      (e = cudaMemcpy(p->d_vq64, v64.data(), sizeof(double) * v64.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(kcuda(p, e, "uploading the kernel tables"));
  std::vector<double> tw(2 * n);
  for (int t = 0; t < n; ++t) {
    const long double ang = 2.0L * 3.141592653589793238462643383279502884L * t / n;
    tw[2 * t] = (double)std::cos(ang);
    tw[2 * t + 1] = -(double)std::sin(ang);
  }
  if (fp64) {
    for (double& x : v64) x /= (double)ntot;
    if ((e = cudaMalloc(&p->d_vq, sizeof(double) * v64.size())) != cudaSuccess ||
        (e = cudaMemcpy(p->d_vq, v64.data(), sizeof(double) * v64.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_tw, sizeof(double) * tw.size())) != cudaSuccess ||
        (e = cudaMemcpy(p->d_tw, tw.data(), sizeof(double) * tw.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(kcuda(p, e, "uploading tables"));
  } else {
    std::vector<float> v32(v64.size()), tw32(tw.size());
    for (size_t i = 0; i < v64.size(); ++i) v32[i] = (float)(v64[i] / (double)ntot);
    for (size_t i = 0; i < tw.size(); ++i) tw32[i] = (float)tw[i];
    if ((e = cudaMalloc(&p->d_vq, sizeof(float) * v32.size())) != cudaSuccess ||
        (e = cudaMemcpy(p->d_vq, v32.data(), sizeof(float) * v32.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_tw, sizeof(float) * tw32.size())) != cudaSuccess ||
        (e = cudaMemcpy(p->d_tw, tw32.data(), sizeof(float) * tw32.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(kcuda(p, e, "uploading tables"));
  }
  if ((e = cudaMalloc((void**)&p->d_result, 4 * sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost((void**)&p->h_result, 4 * sizeof(double))) != cudaSuccess)
    return bail(kcuda(p, e, "allocating results"));

  DevPlan& d = p->dp;
  d.n = n;
  d.k3h = n / 2 + 1;
  d.ntot = ntot;
  d.hsize = ntot;
  d.tw = p->d_tw;
  d.inv_ntot = 1.0 / (double)ntot;
  d.psi_scale = 1.0 / std::sqrt(p->vol);
  d.out_scale = std::sqrt(p->vol) / (double)ntot;
  d.msmall2 = -1;
  d.vtabq = p->d_vq;
  d.vtabq64 = p->d_vq64;
  d.q0 = -1;
  for (int j = 0; j < p->nq; ++j)
    if (qs[3 * j] == 0.0 && qs[3 * j + 1] == 0.0 && qs[3 * j + 2] == 0.0) d.q0 = j;
  if (!fp64) {
    // the mixed form's FP64 terms: |m + q|^2 <= 3 (reduced coordinates)
    std::vector<float> qf(qs.begin(), qs.end());
    if ((e = cudaMalloc((void**)&p->d_qfrac, sizeof(float) * qf.size())) != cudaSuccess ||
        (e = cudaMemcpy(p->d_qfrac, qf.data(), sizeof(float) * qf.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(kcuda(p, e, "uploading q"));
    d.qfrac = p->d_qfrac;
    d.msmall2 = 3;
    p->npw_max = *std::max_element(p->npw.begin(), p->npw.end());
    if ((e = cudaMalloc((void**)&p->d_krows, sizeof(double2*) * nk)) != cudaSuccess ||
        (e = cudaMalloc((void**)&p->d_knpw, sizeof(int) * nk)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_knpw, p->npw.data(), sizeof(int) * nk, cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(kcuda(p, e, "uploading the sphere sizes"));
    d.ovl_scale = (double)ntot / p->vol;
  }
  p->chain_batch = (int)std::max<size_t>(1, kBufferBytes / ((size_t)ntot * csz(p)));

  int optin = 0;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device)) != cudaSuccess)
    return bail(kcuda(p, e, "cudaDeviceGetAttribute"));
  if (ops->smem > (size_t)optin)
    return bail(kfail(p, FOCK_ERR_UNSUPPORTED_SIZE, "the grid needs more shared memory than a CTA has"));
  if ((e = ops->configure(d)) != cudaSuccess || (e = kops->configure()) != cudaSuccess)
    return bail(kcuda(p, e, "configuring kernels"));
  *out = p;
  return FOCK_OK;
}

fock_status fock_gsphere_k(const int grid[3], const double cell[9], double ecut_ha, const double* kpt,
                           int64_t* npw, int32_t* miller, int64_t capacity) {
  g_kcreate_error.clear();
  if (!grid || !cell || !kpt || !npw) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "NULL argument");
  if (!(ecut_ha > 0.0) || !std::isfinite(ecut_ha)) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "bad ecut");
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(cell[i])) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "cell is not finite");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(kpt[i])) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "k point is not finite");
  double recip[9];
  if (!(std::fabs(fockx::lattice::reciprocal(cell, recip)) > 0.0))
    return kfail(nullptr, FOCK_ERR_INVALID_ARG, "the cell is degenerate");
  std::vector<fockx::lattice::GEntry> sph;
  const int n = std::min(grid[0], std::min(grid[1], grid[2]));
  if (!fockx::lattice::build_sphere(cell, recip, ecut_ha, n, sph, kpt))
    return kfail(nullptr, FOCK_ERR_GRID_TOO_SMALL, "the G-sphere does not fit on the grid");
  *npw = (int64_t)sph.size();
  if (miller) {
    if (capacity < (int64_t)sph.size()) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "miller buffer too small");
    for (size_t g = 0; g < sph.size(); ++g)
      for (int a = 0; a < 3; ++a) miller[3 * g + a] = sph[g].m[a];
  }
  return FOCK_OK;
}

fock_status fock_kplan_nk(fock_kplan_t p, int* nk) {
  if (!p || !nk) return kfail(p, FOCK_ERR_INVALID_ARG, "bad argument");
  *nk = p->nk;
  return FOCK_OK;
}

fock_status fock_kplan_npw(fock_kplan_t p, int k, int64_t* npw) {
  if (!p || !npw || k < 0 || k >= p->nk) return kfail(p, FOCK_ERR_INVALID_ARG, "bad argument");
  *npw = p->npw[k];
  return FOCK_OK;
}

fock_status fock_kplan_gvectors(fock_kplan_t p, int k, int32_t* miller) {
  if (!p || !miller || k < 0 || k >= p->nk) return kfail(p, FOCK_ERR_INVALID_ARG, "bad argument");
  std::memcpy(miller, p->miller[k].data(), sizeof(int32_t) * p->miller[k].size());
  return FOCK_OK;
}

fock_status fock_kplan_set_batch(fock_kplan_t p, int chain_batch) {
  if (!p || chain_batch < 1 || chain_batch > 4096) return kfail(p, FOCK_ERR_INVALID_ARG, "bad chain_batch");
  if (chain_batch != p->chain_batch) {
    cudaFree(p->d_h);
    p->d_h = nullptr;
    p->chain_batch = chain_batch;
  }
  return FOCK_OK;
}

fock_status fock_kplan_apply(fock_kplan_t p, const void* const* psi_G, int nb, const double* occ,
                             void* const* vpsi_G, double* ex, fock_stream_t stream) {
  if (!p) return kfail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (!psi_G || !vpsi_G || !occ || nb < 1) return kfail(p, FOCK_ERR_INVALID_ARG, "NULL argument or nb < 1");
  const int nk = p->nk;
  for (int k = 0; k < nk; ++k) {
    if (!psi_G[k] || !vpsi_G[k]) return kfail(p, FOCK_ERR_INVALID_ARG, "NULL orbital array");
    const size_t bytes = (size_t)nb * (size_t)p->npw[k] * 16;
    const char* a = static_cast<const char*>(psi_G[k]);
    const char* b = static_cast<const char*>(vpsi_G[k]);
    if (a < b + bytes && b < a + bytes) return kfail(p, FOCK_ERR_INVALID_ARG, "psi_G and vpsi_G overlap");
  }
  for (int i = 0; i < nk * nb; ++i)
    if (!std::isfinite(occ[i])) return kfail(p, FOCK_ERR_INVALID_ARG, "occupations must be finite");
  if ((int64_t)nk * nb > (1 << 15)) return kfail(p, FOCK_ERR_INVALID_ARG, "too many states");
  int dev = -1;
  FOCK_KCUDA(p, cudaGetDevice(&dev));
  if (dev != p->device) return kfail(p, FOCK_ERR_INVALID_ARG, "the plan belongs to another device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ns = nk * nb;
  const int npairs = ns * (ns + 1) / 2;
  fock_status st = kensure(p, ns, npairs);
  if (st != FOCK_OK) return st;
  if (p->sched_ns != ns || p->sched_nb != nb) {
    p->pairs.clear();
    p->chains.clear();
    const int nblk = (ns + kBandBlock - 1) / kBandBlock;
    for (int bi = 0; bi < nblk; ++bi)
      for (int bj = bi; bj < nblk; ++bj)
        for (int a = bi * kBandBlock; a < std::min(ns, (bi + 1) * kBandBlock); ++a)
          for (int b = std::max(a, bj * kBandBlock); b < std::min(ns, (bj + 1) * kBandBlock); ++b) {
            Chain c{};
            c.ai = a;
            c.aj = b;
            c.bi = c.bj = -1;
            c.pa = (int)p->pairs.size();
            c.pb = -1;
            c.pad1 = p->qidx[(size_t)(a / nb) * nk + (b / nb)];
            p->pairs.push_back(make_int2(a, b));
            p->chains.push_back(c);
          }
    FOCK_KCUDA(p, cudaMemcpyAsync(p->d_pairs, p->pairs.data(), sizeof(int2) * npairs, cudaMemcpyHostToDevice, s));
    FOCK_KCUDA(p, cudaMemcpyAsync(p->d_chains, p->chains.data(), sizeof(Chain) * npairs, cudaMemcpyHostToDevice, s));
    FOCK_KCUDA(p, cudaStreamSynchronize(s));
    p->sched_ns = ns;
    p->sched_nb = nb;
  }
  // occupation times k weight, per state
  std::vector<double> ow(ns);
  for (int k = 0; k < nk; ++k)
    for (int b = 0; b < nb; ++b) ow[(size_t)k * nb + b] = p->wk[k] * occ[(size_t)k * nb + b];
  FOCK_KCUDA(p, cudaMemcpyAsync(p->d_occw, ow.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
  if (p->ops->real_bytes == 8) {
    FOCK_KCUDA(p, cudaMemcpyAsync(p->d_occwT, ow.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
  } else {
    std::vector<float> f(ow.begin(), ow.end());
    FOCK_KCUDA(p, cudaMemcpyAsync(p->d_occwT, f.data(), sizeof(float) * ns, cudaMemcpyHostToDevice, s));
  }
  FOCK_KCUDA(p, cudaStreamSynchronize(s));  // the host vectors above are locals
  const size_t grid_bytes = (size_t)p->dp.ntot * csz(p);
  FOCK_KCUDA(p, cudaMemsetAsync(p->d_w, 0, grid_bytes * ns, s));
  FOCK_KCUDA(p, cudaMemsetAsync(p->d_epair, 0, sizeof(double) * npairs, s));
  const int nbat = p->chain_batch;  // bands per O(nb) launch: the transform buffer holds chain_batch grids
  for (int k = 0; k < nk; ++k)
    for (int b0 = 0; b0 < nb; b0 += nbat) {
      const int cnt = std::min(nbat, nb - b0);
      const double2* src = static_cast<const double2*>(psi_G[k]) + (size_t)b0 * p->npw[k];
      FOCK_KCUDA(p, p->kops->to_real(p->dp, src, p->npw[k], p->d_gidx[k], k * nb + b0, cnt, p->d_h, p->d_u, s));
    }
  DevPlan dp = p->dp;
  if (p->ops->real_bytes == 4 && dp.q0 >= 0) {
    // FP64 overlaps of each k point's states for the G = 0 terms of its q = 0 pairs
    const int64_t per = (int64_t)nb * nb;
    if (2 * nk * per > p->kovl_cap) {
      cudaFree(p->d_kovl);
      p->d_kovl = nullptr;
      p->kovl_cap = 0;
      FOCK_KCUDA(p, cudaMalloc((void**)&p->d_kovl, sizeof(double) * (size_t)(2 * nk * per)));
      p->kovl_cap = 2 * nk * per;
    }
    double* re = p->d_kovl;
    double* im = p->d_kovl + nk * per;
    std::vector<const double2*> rows(nk);
    for (int k = 0; k < nk; ++k) rows[k] = static_cast<const double2*>(psi_G[k]);
    FOCK_KCUDA(p, cudaMemcpyAsync(p->d_krows, rows.data(), sizeof(double2*) * nk, cudaMemcpyHostToDevice, s));
    // (a copy from pageable memory returns once the source has been staged,
    // so the local vector may go)
    FOCK_KCUDA(p, fockx::launch_overlap_sets(p->d_krows, p->d_knpw, p->npw_max, nk, nb, re, im, s));
    dp.kovl_re = re;
    dp.kovl_im = im;
    dp.kovl_nb = nb;
  }
  for (int c = 0; c < npairs; c += p->chain_batch) {
    const int cnt = std::min(p->chain_batch, npairs - c);
    const Chain* ch = p->d_chains + c;
    FOCK_KCUDA(p, p->kops->pair_fwd(dp, p->d_u, ch, cnt, p->d_h, s));
    FOCK_KCUDA(p, p->kops->pair_col(dp, p->d_h, ch, cnt, p->d_epair, s));
    FOCK_KCUDA(p, p->kops->pair_inv(dp, p->d_u, p->d_w, p->d_occwT, ch, cnt, p->d_h, s));
  }
  for (int k = 0; k < nk; ++k)
    for (int b0 = 0; b0 < nb; b0 += nbat) {
      const int cnt = std::min(nbat, nb - b0);
      double2* dst = static_cast<double2*>(vpsi_G[k]) + (size_t)b0 * p->npw[k];
      FOCK_KCUDA(p, p->kops->to_sphere(p->dp, p->d_w, k * nb + b0, cnt, p->npw[k], p->d_gidx[k], p->d_h, dst, s));
    }
  const double scale = -0.5 * p->vol / ((double)p->dp.ntot * (double)p->dp.ntot);
  FOCK_KCUDA(p, fockx::launch_energy_reduce(p->d_pairs, npairs, p->d_occw, p->d_epair, nullptr, scale,
                                            p->d_result, s));
  if (ex) {
    FOCK_KCUDA(p, cudaMemcpyAsync(p->h_result, p->d_result, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    FOCK_KCUDA(p, cudaStreamSynchronize(s));
    *ex = p->h_result[0];
  }
  return FOCK_OK;
}

const char* fock_kplan_last_error(fock_kplan_t p) { return p ? p->err.c_str() : g_kcreate_error.c_str(); }

fock_status fock_kplan_destroy(fock_kplan_t p) {
  if (!p) return FOCK_OK;
  kfree_ws(p);
  for (int* d : p->d_gidx) cudaFree(d);
  cudaFree(p->d_vq);
  cudaFree(p->d_vq64);
  cudaFree(p->d_qfrac);
  cudaFree(p->d_kovl);
  cudaFree(p->d_krows);
  cudaFree(p->d_knpw);
  cudaFree(p->d_tw);
  cudaFree(p->d_result);
  if (p->h_result) cudaFreeHost(p->h_result);
  delete p;
  return FOCK_OK;
}

}  // extern "C"
