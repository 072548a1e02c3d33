// fock_plan.cpp — host side of the C ABI declared in include/fock.h: cell and
// plane-wave sphere, Coulomb-kernel tables, twiddles, pair schedule, workspace
// and the orchestration of the kernel passes.
//
// Built with -ffp-contract=off: the sphere's order is defined by a fixed
// sequence of IEEE operations (no fused multiply-add), so every machine builds
// the same list.
#include "fock.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fock_internal.h"
#include "fock_lattice.h"

using fockx::Chain;
using fockx::DevPlan;
using fockx::KernelOps;

namespace {

constexpr int kBandBlock = 16;                  // default bands per block of the pair schedule
constexpr size_t kChainBufferBytes = 320u << 20;  // budget of the default pair-transform buffer
constexpr int kMsmall2 = 3;                     // |m|^2 of the kernel terms kept in FP64 (mixed)

// d as the double-float pair (hi, lo): hi = float(d), lo = float(d - hi).
void split_df64(double d, float* out) {
  const float hi = (float)d;
  out[0] = hi;
  out[1] = (float)(d - (double)hi);
}

thread_local std::string g_create_error;

using fockx::lattice::GEntry;
using fockx::lattice::build_sphere;
using fockx::lattice::freq_of;
using fockx::lattice::g2_of;
using fockx::lattice::kPi;

struct Workspace {
  int nb_cap = 0;
  size_t psi_bytes = 0;
  void* psi = nullptr;
  void* w = nullptr;
  void* h = nullptr;
  void* hx[3] = {nullptr, nullptr, nullptr};  // transform buffers of the other pair-loop streams
  size_t h_bytes = 0;
  int npair_cap = 0;
  double* epair = nullptr;
  double* dpair = nullptr;
  int2* pairs = nullptr;
  Chain* chains = nullptr;
  double* occ = nullptr;
  void* occT = nullptr;
};

}  // namespace

struct fock_plan {
  int device = 0;
  int n = 0;
  double cell[9];
  double recip[9];
  double vol = 0.0;
  double ecut = 0.0;
  fock_kernel kind = FOCK_KERNEL_SPENCER_ALAVI;
  double omega = 0.0;
  fock_precision prec = FOCK_PREC_FP64;
  std::vector<int32_t> miller;
  int npw = 0;
  const KernelOps* ops = nullptr;
  DevPlan dp{};
  int chain_batch = 1;
  int band_block = kBandBlock;
  // device tables
  int* d_gidx = nullptr;
  int* d_gidxneg = nullptr;
  void* d_tw = nullptr;
  void* d_vtab = nullptr;
  void* d_dvtab = nullptr;
  double* d_vtab64 = nullptr;
  double* d_dvtab64 = nullptr;
  int* d_ncol = nullptr;
  int* d_colmap = nullptr;
  int* d_kept = nullptr;
  // deterministic accumulation (fock_plan_set_deterministic)
  bool det = false;
  double vnorm = 0.0;          // ||v||_2 over the whole grid
  double* d_stats = nullptr;   // [2 * det_nb_cap] per-band max |psi| and sum psi^2
  double* d_scale = nullptr;   // [2] fixed-point scale 2^s and 2^-s
  double* d_epart = nullptr;   // [det_npair_cap * ncta_col] per-CTA energy partials
  double* d_dpart = nullptr;
  int det_nb_cap = 0;
  int det_npair_cap = 0;
  // mixed form: FP64 pair overlaps for the G = 0 terms (DevPlan::ovl) and the
  // occupied coefficients of fock_set_occupied (for the fixed operator's)
  double* d_ovl = nullptr;
  int64_t ovl_cap = 0;
  int* d_half = nullptr;  // G = 0, then one of each pair G, -G of the sphere (positions)
  int nhalf_g = 0;
  // FP64: the kernel table scaled by -f0 (DevPlan::vtab_f)
  void* d_vtab_f = nullptr;
  double vtab_f_f0 = 0.0;
  double2* d_cocc = nullptr;
  int64_t cocc_cap = 0;
  int64_t kept_columns = 0;  // lines of the column map (both pairs)
  double* d_result = nullptr;
  double* h_result = nullptr;  // pinned
  int64_t table_bytes = 0;
  Workspace ws;
  // pair schedule of the last band count uploaded
  int sched_nb = -1;
  std::vector<int2> pairs;
  std::vector<Chain> chains;
  std::vector<double> occ_host;
  // fixed operator (fock_set_occupied): the first fixed_nb bands of the
  // real-space workspace hold the occupied orbitals that define V_x
  int fixed_nb = 0;
  int fixed_sched_nt = -1;
  int fixed_sched_bb = 0;
  // pair-loop launches rotate over the caller's stream and streams - 1
  // plan-owned ones, each with its own transform buffer
  int streams = 1;
  cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
  // launch accounting and optional per-launch event timing
  fock_stats stats{};
  bool timing = false;
  std::vector<cudaEvent_t> events;  // pool, two per timed launch
  std::vector<int> event_phase;     // phase of each timed launch
  size_t nev = 0;                   // timed launches recorded in the current call
  std::string err;
};

namespace {

fock_status fail(fock_plan* p, fock_status s, const std::string& msg) {
  if (p) p->err = msg;
  else g_create_error = msg;
  return s;
}

fock_status cuda_fail(fock_plan* p, cudaError_t e, const char* what) {
  const fock_status s = (e == cudaErrorMemoryAllocation) ? FOCK_ERR_OOM : FOCK_ERR_CUDA;
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a sticky launch error of this thread's last call
  return fail(p, s, msg);
}

#define FOCK_CUDA(p, call)                              \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(p, e_, #call); \
  } while (0)

template <class Ptr>
cudaError_t dev_alloc(Ptr** ptr, size_t bytes) {
  return cudaMalloc(reinterpret_cast<void**>(ptr), bytes == 0 ? 16 : bytes);
}

void free_ws(Workspace& w) {
  cudaFree(w.psi);
  cudaFree(w.w);
  cudaFree(w.h);
  for (void* x : w.hx) cudaFree(x);
  cudaFree(w.epair);
  cudaFree(w.dpair);
  cudaFree(w.pairs);
  cudaFree(w.chains);
  cudaFree(w.occ);
  cudaFree(w.occT);
  w = Workspace{};
}

void reciprocal(const double* cell, double* recip, double* vol_signed) {
  *vol_signed = fockx::lattice::reciprocal(cell, recip);
}

void kernel_value(const fock_plan* p, double g2, double* v, double* dv) {
  fockx::lattice::kernel_value(p->kind, p->vol, p->omega, g2, v, dv);
}

// Unique pairs i <= j in band blocks of kBandBlock (block rows outer), i outer and j
// inner inside a block, so consecutive pairs share psi_i and a batch of chains
// touches a few blocks of orbitals.  Chain k holds pairs 2k and 2k+1.
void schedule_pairs(int nb, int bb, std::vector<int2>& pairs) {
  pairs.clear();
  pairs.reserve((size_t)nb * (nb + 1) / 2);
  const int nblk = (nb + bb - 1) / bb;
  for (int bi = 0; bi < nblk; ++bi) {
    for (int bj = bi; bj < nblk; ++bj) {
      const int i0 = bi * bb, i1 = std::min(nb, i0 + bb);
      const int j0 = bj * bb, j1 = std::min(nb, j0 + bb);
      for (int i = i0; i < i1; ++i)
        for (int j = std::max(i, j0); j < j1; ++j) pairs.push_back(make_int2(i, j));
    }
  }
}

void build_schedule(fock_plan* p, int nb) { schedule_pairs(nb, p->band_block, p->pairs); }

// Chains [c0, c1) of shard `shard` of `nshards` over nch chains.
void shard_range(int nch, int shard, int nshards, int* c0, int* c1) {
  *c0 = (int)((int64_t)nch * shard / nshards);
  *c1 = (int)((int64_t)nch * (shard + 1) / nshards);
}

void chains_from_pairs(const std::vector<int2>& pairs, std::vector<Chain>& chains) {
  chains.clear();
  const int np = (int)pairs.size();
  chains.reserve((np + 1) / 2);
  for (int k = 0; 2 * k < np; ++k) {
    Chain c{};
    c.ai = pairs[2 * k].x;
    c.aj = pairs[2 * k].y;
    c.pa = 2 * k;
    if (2 * k + 1 < np) {
      c.bi = pairs[2 * k + 1].x;
      c.bj = pairs[2 * k + 1].y;
      c.pb = 2 * k + 1;
    } else {
      c.bi = c.bj = -1;
      c.pb = -1;
    }
    chains.push_back(c);
  }
}

void stats_reset(fock_plan* p) {
  const int cb = p->stats.chain_batch, bb = p->stats.band_batch;
  p->stats = fock_stats{};
  p->stats.chain_batch = cb;
  p->stats.band_batch = bb;
  p->nev = 0;
  p->event_phase.clear();
}

// Brackets one pass (`launches` kernels) of phase `ph`: events are recorded on
// the stream around it when timing is on.
struct PhaseScope {
  fock_plan* p;
  int ph;
  cudaStream_t s;
  size_t idx;
  PhaseScope(fock_plan* p_, int ph_, int launches, cudaStream_t s_) : p(p_), ph(ph_), s(s_), idx(0) {
    p->stats.launches += launches;
    p->stats.phase_launches[ph] += launches;
    if (p->timing) {
      idx = p->nev++;
      while (p->events.size() < 2 * p->nev) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) break;
        p->events.push_back(e);
      }
      if (p->events.size() >= 2 * p->nev) {
        cudaEventRecord(p->events[2 * idx], s);
        p->event_phase.push_back(ph);
      } else {
        p->nev--;
        p->timing = false;
      }
    }
  }
  ~PhaseScope() {
    if (p->timing && idx < p->nev) cudaEventRecord(p->events[2 * idx + 1], s);
  }
};

fock_status collect_timing(fock_plan* p, cudaStream_t s) {
  if (!p->timing || p->nev == 0) return FOCK_OK;
  FOCK_CUDA(p, cudaStreamSynchronize(s));
  for (size_t k = 0; k < p->nev; ++k) {
    float ms = 0.f;
    FOCK_CUDA(p, cudaEventElapsedTime(&ms, p->events[2 * k], p->events[2 * k + 1]));
    p->stats.phase_ms[p->event_phase[k]] += ms;
  }
  return FOCK_OK;
}

fock_status check_device(fock_plan* p) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaGetDevice");
  if (dev != p->device) return fail(p, FOCK_ERR_INVALID_ARG, "the plan belongs to another device");
  return FOCK_OK;
}

fock_status ensure_workspace(fock_plan* p, int nb, int npairs) {
  Workspace& w = p->ws;
  const size_t rb = (size_t)p->ops->real_bytes;
  if (nb > w.nb_cap) {
    cudaFree(w.psi);
    cudaFree(w.w);
    cudaFree(w.occ);
    cudaFree(w.occT);
    w.psi = w.w = w.occT = nullptr;
    w.occ = nullptr;
    w.nb_cap = 0;
    w.psi_bytes = (size_t)nb * (size_t)p->dp.ntot * rb;
    FOCK_CUDA(p, dev_alloc(&w.psi, w.psi_bytes));
    FOCK_CUDA(p, dev_alloc(&w.w, w.psi_bytes));
    FOCK_CUDA(p, dev_alloc(&w.occ, sizeof(double) * nb));
    FOCK_CUDA(p, dev_alloc(&w.occT, rb * nb));
    w.nb_cap = nb;
  }
  if (w.h == nullptr) {
    const size_t chain_bytes = (size_t)p->dp.hsize * 2 * rb;
    w.h_bytes = chain_bytes * (size_t)p->chain_batch;
    FOCK_CUDA(p, dev_alloc(&w.h, w.h_bytes));
  }
  if (npairs > w.npair_cap) {
    cudaFree(w.epair);
    cudaFree(w.dpair);
    cudaFree(w.pairs);
    cudaFree(w.chains);
    w.epair = w.dpair = nullptr;
    w.pairs = nullptr;
    w.chains = nullptr;
    w.npair_cap = 0;
    p->sched_nb = -1;
    p->fixed_sched_nt = -1;
    FOCK_CUDA(p, dev_alloc(&w.epair, sizeof(double) * npairs));
    FOCK_CUDA(p, dev_alloc(&w.dpair, sizeof(double) * npairs));
    FOCK_CUDA(p, dev_alloc(&w.pairs, sizeof(int2) * npairs));
    FOCK_CUDA(p, dev_alloc(&w.chains, sizeof(Chain) * ((npairs + 1) / 2)));
    w.npair_cap = npairs;
  }
  return FOCK_OK;
}

// Grow the real-space workspace to `nb` bands, keeping the first `keep` bands
// of the orbitals (the fixed occupied set).
fock_status grow_keeping(fock_plan* p, int nb, int keep) {
  Workspace& w = p->ws;
  if (nb <= w.nb_cap) return FOCK_OK;
  const size_t rb = (size_t)p->ops->real_bytes;
  const size_t bytes = (size_t)nb * (size_t)p->dp.ntot * rb;
  void *psi = nullptr, *wacc = nullptr, *occT = nullptr;
  double* occ = nullptr;
  cudaError_t e;
  if ((e = dev_alloc(&psi, bytes)) != cudaSuccess || (e = dev_alloc(&wacc, bytes)) != cudaSuccess ||
      (e = dev_alloc(&occ, sizeof(double) * nb)) != cudaSuccess || (e = dev_alloc(&occT, rb * nb)) != cudaSuccess) {
    cudaFree(psi);
    cudaFree(wacc);
    cudaFree(occ);
    cudaFree(occT);
    return cuda_fail(p, e, "growing the workspace");
  }
  if (keep > 0 && w.psi) {
    e = cudaMemcpy(psi, w.psi, (size_t)keep * (size_t)p->dp.ntot * rb, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(occ, w.occ, sizeof(double) * keep, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(occT, w.occT, rb * keep, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
      cudaFree(psi);
      cudaFree(wacc);
      cudaFree(occ);
      cudaFree(occT);
      return cuda_fail(p, e, "copying the occupied orbitals");
    }
  }
  cudaFree(w.psi);
  cudaFree(w.w);
  cudaFree(w.occ);
  cudaFree(w.occT);
  w.psi = psi;
  w.w = wacc;
  w.occ = occ;
  w.occT = occT;
  w.psi_bytes = bytes;
  w.nb_cap = nb;
  return FOCK_OK;
}

fock_status upload_occ(fock_plan* p, const double* occ, int nb, cudaStream_t s) {
  p->occ_host.assign(occ, occ + nb);
  FOCK_CUDA(p, cudaMemcpyAsync(p->ws.occ, occ, sizeof(double) * nb, cudaMemcpyHostToDevice, s));
  if (p->prec == FOCK_PREC_FP64) {
    FOCK_CUDA(p, cudaMemcpyAsync(p->ws.occT, occ, sizeof(double) * nb, cudaMemcpyHostToDevice, s));
  } else if (p->prec == FOCK_PREC_DF64) {
    std::vector<float> f(2 * (size_t)nb);
    for (int k = 0; k < nb; ++k) split_df64(occ[k], &f[2 * k]);
    FOCK_CUDA(p, cudaMemcpyAsync(p->ws.occT, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice, s));
    FOCK_CUDA(p, cudaStreamSynchronize(s));  // f is a local buffer
  } else {
    std::vector<float> f(occ, occ + nb);
    FOCK_CUDA(p, cudaMemcpyAsync(p->ws.occT, f.data(), sizeof(float) * nb, cudaMemcpyHostToDevice, s));
    FOCK_CUDA(p, cudaStreamSynchronize(s));  // f is a local buffer
  }
  return FOCK_OK;
}

// The FP64 overlaps of the mixed form's G = 0 terms: S(i, j) = Re sum_G
// conj(a_i) b_j for the pairs of an apply, into the plan's buffer, and the
// DevPlan fields that point the column pass at them (ld columns, column j at
// j - j0).  Other precisions leave dp.ovl NULL.
fock_status prepare_overlaps(fock_plan* p, const void* a, int na, const void* b, int nbb, bool sym, int j0,
                             DevPlan* dp, cudaStream_t s) {
  dp->ovl = nullptr;
  if (p->ops->prec != 1 || na < 1 || nbb < 1) return FOCK_OK;
  const int64_t need = (int64_t)na * nbb;
  if (need > p->ovl_cap) {
    cudaFree(p->d_ovl);
    p->d_ovl = nullptr;
    p->ovl_cap = 0;
    FOCK_CUDA(p, dev_alloc(&p->d_ovl, sizeof(double) * (size_t)need));
    p->ovl_cap = need;
  }
  FOCK_CUDA(p, fockx::launch_overlap(static_cast<const double2*>(a), na, static_cast<const double2*>(b), nbb,
                                     p->npw, p->d_half, p->nhalf_g, sym, p->d_ovl, nbb, s));
  dp->ovl = p->d_ovl;
  dp->ovl_ld = nbb;
  dp->ovl_j0 = j0;
  dp->ovl_scale = (double)p->dp.ntot / p->vol;
  return FOCK_OK;
}

// FP64: when every band of an apply has the same nonzero occupation f0,
// point the DevPlan at the kernel table scaled by -f0 (built on the device,
// kept while f0 stays the same).  (In double-float the same change measured
// 2% slower and is not made.)
fock_status prepare_prescaled(fock_plan* p, const double* occ, int nb, DevPlan* dp, cudaStream_t s) {
  dp->vtab_f = nullptr;
  if (p->ops->prec != 0 || nb < 1 || occ[0] == 0.0) return FOCK_OK;
  for (int i = 1; i < nb; ++i)
    if (occ[i] != occ[0]) return FOCK_OK;
  const double f0 = occ[0];
  const int64_t nhalf = (int64_t)p->dp.n * p->dp.n * p->dp.k3h;
  if (p->d_vtab_f == nullptr) {
    FOCK_CUDA(p, dev_alloc(&p->d_vtab_f, (size_t)nhalf * sizeof(double)));
    p->vtab_f_f0 = 0.0;
  }
  if (p->vtab_f_f0 != f0) {
    FOCK_CUDA(p, fockx::launch_scaled_table(p->d_vtab64, nhalf, -f0 / (double)p->dp.ntot,
                                            static_cast<double*>(p->d_vtab_f), s));
    p->vtab_f_f0 = f0;
    p->stats.launches += 1;
  }
  dp->vtab = p->d_vtab_f;
  dp->vtab_f = p->d_vtab_f;
  dp->vtab_f_factor = -f0;
  return FOCK_OK;
}

int bands_per_grid_batch(const fock_plan* p) {
  const size_t grid_bytes = (size_t)p->dp.ntot * 2 * (size_t)p->ops->real_bytes;
  const int q = (int)std::max<size_t>(1, p->ws.h_bytes / grid_bytes);
  return 2 * q;
}

fock_status orbitals_to_real(fock_plan* p, const void* psiG, int nb, cudaStream_t s) {
  const int nbat = bands_per_grid_batch(p);
  p->stats.band_batch = nbat;
  for (int b0 = 0; b0 < nb; b0 += nbat) {
    const int cnt = std::min(nbat, nb - b0);
    PhaseScope ps(p, FOCK_PHASE_TO_REAL, 3, s);
    FOCK_CUDA(p, p->ops->to_real(p->dp, static_cast<const double2*>(psiG), nb, b0, cnt, p->ws.h,
                                 p->ws.psi, s));
  }
  return FOCK_OK;
}

fock_status validate_apply(fock_plan* p, const void* psiG, int nb, const void* out) {
  if (!p) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (!psiG || !out) return fail(p, FOCK_ERR_INVALID_ARG, "psi_G or the output is NULL");
  if (nb < 1) return fail(p, FOCK_ERR_INVALID_ARG, "nb must be >= 1");
  if (nb > (1 << 15)) return fail(p, FOCK_ERR_INVALID_ARG, "nb is larger than 32768");
  return check_device(p);
}

// Deterministic mode: buffers for nbands real-space bands and npairs pairs.
fock_status det_buffers(fock_plan* p, int nbands, int npairs) {
  if (nbands > p->det_nb_cap) {
    cudaFree(p->d_stats);
    p->d_stats = nullptr;
    p->det_nb_cap = 0;
    FOCK_CUDA(p, dev_alloc(&p->d_stats, sizeof(double) * 2 * nbands));
    p->det_nb_cap = nbands;
  }
  if (!p->d_scale) FOCK_CUDA(p, dev_alloc(&p->d_scale, sizeof(double) * 2));
  if (npairs > p->det_npair_cap) {
    cudaFree(p->d_epart);
    cudaFree(p->d_dpart);
    p->d_epart = p->d_dpart = nullptr;
    p->det_npair_cap = 0;
    const size_t n = (size_t)npairs * (size_t)p->dp.ncta_col;
    FOCK_CUDA(p, dev_alloc(&p->d_epart, sizeof(double) * n));
    FOCK_CUDA(p, dev_alloc(&p->d_dpart, sizeof(double) * n));
    p->det_npair_cap = npairs;
  }
  return FOCK_OK;
}

// Deterministic mode: the fixed-point scale of this call from the real-space
// bands [0, nbands) (sources: the first nsrc, occupations in ws.occ).
fock_status det_prepare(fock_plan* p, int nbands, int nsrc, DevPlan* dp, cudaStream_t s) {
  FOCK_CUDA(p, fockx::launch_orbital_stats(p->ops->prec, p->ws.psi, nbands, p->dp.ntot, p->d_stats, s));
  FOCK_CUDA(p, fockx::launch_det_scale(p->d_stats, nbands, p->ws.occ, nsrc, p->vnorm, p->dp.ntot, p->d_scale, s));
  dp->det = 1;
  dp->det_scale = p->d_scale;
  return FOCK_OK;
}

// The plan-owned streams of the pair loop, their fork/join events and
// transform buffers.
fock_status pipeline_resources(fock_plan* p) {
  if (!p->ev_fork) FOCK_CUDA(p, cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  for (int k = 0; k + 1 < p->streams; ++k) {
    if (!p->aux[k]) FOCK_CUDA(p, cudaStreamCreateWithFlags(&p->aux[k], cudaStreamNonBlocking));
    if (!p->ev_join[k]) FOCK_CUDA(p, cudaEventCreateWithFlags(&p->ev_join[k], cudaEventDisableTiming));
    if (!p->ws.hx[k]) FOCK_CUDA(p, dev_alloc(&p->ws.hx[k], p->ws.h_bytes));
  }
  return FOCK_OK;
}

fock_status apply_impl(fock_plan* p, const void* psiG, int nb, const double* occ, int shard,
                       int nshards, void* vpsiG, double* ex, double* dex, fock_stream_t stream) {
  fock_status st = validate_apply(p, psiG, nb, vpsiG);
  if (st != FOCK_OK) return st;
  if (!occ) return fail(p, FOCK_ERR_INVALID_ARG, "occ is NULL");
  if (nshards < 1 || shard < 0 || shard >= nshards)
    return fail(p, FOCK_ERR_INVALID_ARG, "shard must satisfy 0 <= shard < nshards");
  for (int i = 0; i < nb; ++i)
    if (!std::isfinite(occ[i])) return fail(p, FOCK_ERR_INVALID_ARG, "occupations must be finite");
  const size_t bytes = (size_t)nb * (size_t)p->npw * 16;
  const char* a = static_cast<const char*>(psiG);
  const char* b = static_cast<const char*>(vpsiG);
  if (a < b + bytes && b < a + bytes) return fail(p, FOCK_ERR_INVALID_ARG, "psi_G and vpsi_G overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  stats_reset(p);
  p->fixed_nb = 0;  // the real-space workspace is about to be overwritten
  const int npairs = nb * (nb + 1) / 2;
  st = ensure_workspace(p, nb, npairs);
  if (st != FOCK_OK) return st;
  if (p->sched_nb != nb) {
    build_schedule(p, nb);
    chains_from_pairs(p->pairs, p->chains);
    p->fixed_sched_nt = -1;
    FOCK_CUDA(p, cudaMemcpyAsync(p->ws.pairs, p->pairs.data(), sizeof(int2) * npairs,
                                 cudaMemcpyHostToDevice, s));
    FOCK_CUDA(p, cudaMemcpyAsync(p->ws.chains, p->chains.data(), sizeof(Chain) * p->chains.size(),
                                 cudaMemcpyHostToDevice, s));
    FOCK_CUDA(p, cudaStreamSynchronize(s));  // the host vectors may change on the next call
    p->sched_nb = nb;
  }
  st = upload_occ(p, occ, nb, s);
  if (st != FOCK_OK) return st;
  const size_t rb = (size_t)p->ops->real_bytes;
  FOCK_CUDA(p, cudaMemsetAsync(p->ws.w, 0, (size_t)nb * (size_t)p->dp.ntot * rb, s));
  FOCK_CUDA(p, cudaMemsetAsync(p->ws.epair, 0, sizeof(double) * npairs, s));
  FOCK_CUDA(p, cudaMemsetAsync(p->ws.dpair, 0, sizeof(double) * npairs, s));
  st = orbitals_to_real(p, psiG, nb, s);
  if (st != FOCK_OK) return st;

  DevPlan dp = p->dp;
  if (!dex) dp.dvtab64 = nullptr;  // skip the dE/domega partials nobody asked for
  if (p->ops->prec == 1) {  // FP64 overlaps for the G = 0 terms (two launches)
    PhaseScope ps(p, FOCK_PHASE_TO_REAL, 2, s);
    st = prepare_overlaps(p, psiG, nb, psiG, nb, true, 0, &dp, s);
    if (st != FOCK_OK) return st;
  }
  st = prepare_prescaled(p, occ, nb, &dp, s);
  if (st != FOCK_OK) return st;
  double* ep = p->ws.epair;
  double* dpp = p->ws.dpair;
  if (p->det) {
    st = det_buffers(p, nb, npairs);
    if (st != FOCK_OK) return st;
    st = det_prepare(p, nb, nb, &dp, s);
    if (st != FOCK_OK) return st;
    ep = p->d_epart;
    dpp = p->d_dpart;
  }
  const int nch = (int)p->chains.size();
  int c0 = 0, c1 = 0;
  shard_range(nch, shard, nshards, &c0, &c1);
  p->stats.chain_batch = p->chain_batch;
  p->stats.chains = c1 - c0;
  p->stats.pairs = std::min(npairs, 2 * c1) - std::min(npairs, 2 * c0);
  // several streams: launch k runs on stream k mod S (stream 0 = the call's)
  // with that stream's transform buffer, so neighbouring launches' kernels
  // share the GPU; W and the pair energies take atomic (or exact integer)
  // updates, which commute
  const int nst = std::max(1, std::min(p->streams, (c1 - c0 + p->chain_batch - 1) / p->chain_batch));
  if (nst > 1) {
    st = pipeline_resources(p);
    if (st != FOCK_OK) return st;
    FOCK_CUDA(p, cudaEventRecord(p->ev_fork, s));
    for (int k = 0; k + 1 < nst; ++k) FOCK_CUDA(p, cudaStreamWaitEvent(p->aux[k], p->ev_fork, 0));
  }
  for (int c = c0, k = 0; c < c1; c += p->chain_batch, ++k) {
    const int cnt = std::min(p->chain_batch, c1 - c);
    const Chain* ch = p->ws.chains + c;
    const int j = k % nst;
    cudaStream_t sk = j == 0 ? s : p->aux[j - 1];
    void* hk = j == 0 ? p->ws.h : p->ws.hx[j - 1];
    {
      PhaseScope ps(p, FOCK_PHASE_PAIR_FWD, 1, sk);
      FOCK_CUDA(p, p->ops->pair_fwd(dp, p->ws.psi, ch, cnt, hk, sk));
    }
    {
      PhaseScope ps(p, FOCK_PHASE_PAIR_COL, 1, sk);
      FOCK_CUDA(p, p->ops->pair_col(dp, hk, ch, cnt, ep, dpp, sk));
    }
    {
      PhaseScope ps(p, FOCK_PHASE_PAIR_INV, 1, sk);
      FOCK_CUDA(p, p->ops->pair_inv(dp, p->ws.psi, p->ws.w, p->ws.occT, ch, cnt, hk, sk));
    }
  }
  for (int k = 0; k + 1 < nst; ++k) {
    FOCK_CUDA(p, cudaEventRecord(p->ev_join[k], p->aux[k]));
    FOCK_CUDA(p, cudaStreamWaitEvent(s, p->ev_join[k], 0));
  }
  const int p0 = std::min(npairs, 2 * c0), p1 = std::min(npairs, 2 * c1);
  if (p->det) {
    FOCK_CUDA(p, fockx::launch_det_to_double(p->ws.w, (int64_t)nb * p->dp.ntot, p->d_scale, s));
    const int nc = p->dp.ncta_col;
    FOCK_CUDA(p, fockx::launch_det_pair_sums(p->d_epart + (size_t)p0 * nc, p1 - p0, nc, p->ws.epair + p0, s));
    if (dp.dvtab64)
      FOCK_CUDA(p, fockx::launch_det_pair_sums(p->d_dpart + (size_t)p0 * nc, p1 - p0, nc, p->ws.dpair + p0, s));
  }

  const int nbat = bands_per_grid_batch(p);
  for (int b0 = 0; b0 < nb; b0 += nbat) {
    const int cnt = std::min(nbat, nb - b0);
    PhaseScope ps(p, FOCK_PHASE_TO_SPHERE, 3, s);
    FOCK_CUDA(p, p->ops->to_sphere(p->dp, p->ws.w, nb, b0, cnt, p->ws.h,
                                   static_cast<double2*>(vpsiG), s));
  }

  const double scale = -0.5 * p->vol / ((double)p->dp.ntot * (double)p->dp.ntot);
  {
    PhaseScope ps(p, FOCK_PHASE_ENERGY, 1, s);
    FOCK_CUDA(p, fockx::launch_energy_reduce(p->ws.pairs + p0, p1 - p0, p->ws.occ,
                                             p->ws.epair + p0,
                                             dp.dvtab64 ? p->ws.dpair + p0 : nullptr, scale,
                                             p->d_result, s));
  }
  st = collect_timing(p, s);
  if (st != FOCK_OK) return st;
  if (ex || dex) {
    FOCK_CUDA(p, cudaMemcpyAsync(p->h_result, p->d_result, 2 * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
    FOCK_CUDA(p, cudaStreamSynchronize(s));
    if (ex) *ex = p->h_result[0];
    if (dex) *dex = p->h_result[1];
  }
  return FOCK_OK;
}

bool supported_n(int n) {
  int m = n;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1 && n >= 2;
}

}  // namespace

namespace fockx {

bool plan_view(fock_plan* plan, PlanView* out) {
  if (!plan || !out) return false;
  out->device = plan->device;
  out->ops = plan->ops;
  out->dp = plan->dp;
  return true;
}

void plan_set_error(fock_plan* plan, const char* msg) {
  if (plan) plan->err = msg;
}

}  // namespace fockx

namespace {

// Device buffers of one Sternheimer solve, freed on every exit path.
struct StBuffers {
  std::vector<void*> ptrs;
  ~StBuffers() {
    for (void* q : ptrs) cudaFree(q);
  }
  template <class P>
  cudaError_t alloc(P** out, size_t bytes) {
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
    if (e == cudaSuccess) ptrs.push_back(q);
    *out = static_cast<P*>(q);
    return e;
  }
};

}  // namespace

extern "C" {

const char* fock_status_string(fock_status s) {
  switch (s) {
    case FOCK_OK: return "ok";
    case FOCK_ERR_INVALID_ARG: return "invalid argument";
    case FOCK_ERR_UNSUPPORTED_SIZE: return "unsupported grid size";
    case FOCK_ERR_GRID_TOO_SMALL: return "the plane-wave sphere does not fit on the grid";
    case FOCK_ERR_OOM: return "out of device memory";
    case FOCK_ERR_CUDA: return "CUDA error";
    case FOCK_ERR_TIMEOUT: return "a bounded device wait timed out";
  }
  return "unknown status";
}

const char* fock_last_error(fock_plan_t plan) {
  return plan ? plan->err.c_str() : g_create_error.c_str();
}

fock_status fock_plan_create(fock_plan_t* out, const int grid[3], const double cell[9],
                             double ecut_ha, fock_kernel kind, const double* kparams,
                             int nkparams, fock_precision prec, unsigned flags) {
  g_create_error.clear();
  if (!out) return fail(nullptr, FOCK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !cell) return fail(nullptr, FOCK_ERR_INVALID_ARG, "grid or cell is NULL");
  if (!(flags & FOCK_GAMMA_REAL))
    return fail(nullptr, FOCK_ERR_INVALID_ARG, "FOCK_GAMMA_REAL is required");
  if (flags & ~FOCK_GAMMA_REAL) return fail(nullptr, FOCK_ERR_INVALID_ARG, "unknown flag bits");
  if (prec != FOCK_PREC_FP64 && prec != FOCK_PREC_MIXED32 && prec != FOCK_PREC_DF64)
    return fail(nullptr, FOCK_ERR_INVALID_ARG, "unknown precision");
  if (kind != FOCK_KERNEL_SPENCER_ALAVI && kind != FOCK_KERNEL_ERFC)
    return fail(nullptr, FOCK_ERR_INVALID_ARG, "unknown kernel kind");
  if (!(ecut_ha > 0.0) || !std::isfinite(ecut_ha))
    return fail(nullptr, FOCK_ERR_INVALID_ARG, "ecut must be positive and finite");
  double omega = 0.0;
  if (kind == FOCK_KERNEL_ERFC) {
    if (!kparams || nkparams < 1 || !(kparams[0] > 0.0) || !std::isfinite(kparams[0]))
      return fail(nullptr, FOCK_ERR_INVALID_ARG, "erfc kernel needs kparams = {omega > 0}");
    omega = kparams[0];
  }
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(cell[i])) return fail(nullptr, FOCK_ERR_INVALID_ARG, "cell is not finite");
  if (grid[0] != grid[1] || grid[1] != grid[2])
    return fail(nullptr, FOCK_ERR_UNSUPPORTED_SIZE, "the FFT grid must be cubic (N1 = N2 = N3)");
  const int n = grid[0];
  if (n < 2 || !supported_n(n)) return fail(nullptr, FOCK_ERR_UNSUPPORTED_SIZE, "N must be 2^a 3^b");
  const KernelOps* ops = fockx::find_kernel_ops((int)prec, n);
  if (!ops) {
    return fail(nullptr, FOCK_ERR_UNSUPPORTED_SIZE,
                "no kernels compiled for N = " + std::to_string(n));
  }

  fock_plan* p = new (std::nothrow) fock_plan();
  if (!p) return fail(nullptr, FOCK_ERR_OOM, "host allocation failed");
  std::memcpy(p->cell, cell, sizeof(p->cell));
  p->n = n;
  p->ecut = ecut_ha;
  p->kind = kind;
  p->omega = omega;
  p->prec = prec;
  p->ops = ops;

  // cell volume and reciprocal lattice, b_i = (2 pi / Omega) (a_j x a_k)
  reciprocal(cell, p->recip, &p->vol);
  if (!(std::fabs(p->vol) > 0.0)) {
    delete p;
    return fail(nullptr, FOCK_ERR_INVALID_ARG, "the cell is degenerate");
  }
  p->vol = std::fabs(p->vol);

  // the sphere |G|^2 <= 2 Ecut in canonical order
  std::vector<GEntry> sph;
  if (!build_sphere(cell, p->recip, ecut_ha, n, sph)) {
    delete p;
    return fail(nullptr, FOCK_ERR_GRID_TOO_SMALL, "the G-sphere does not fit on the grid");
  }
  p->npw = (int)sph.size();
  p->miller.resize(3 * sph.size());
  std::vector<int> gidx(sph.size()), gneg(sph.size());
  auto off = [n](int m1, int m2, int m3) {
    const int i1 = ((m1 % n) + n) % n, i2 = ((m2 % n) + n) % n, i3 = ((m3 % n) + n) % n;
    return (i1 * n + i2) * n + i3;
  };
  // half of the sphere for the Gamma-point overlaps: G = 0 first, then the G
  // whose first nonzero Miller index is positive
  std::vector<int> half;
  half.reserve(sph.size() / 2 + 1);
  for (size_t k = 0; k < sph.size(); ++k) {
    for (int a = 0; a < 3; ++a) p->miller[3 * k + a] = sph[k].m[a];
    gidx[k] = off(sph[k].m[0], sph[k].m[1], sph[k].m[2]);
    gneg[k] = off(-sph[k].m[0], -sph[k].m[1], -sph[k].m[2]);
    const int* m = sph[k].m;
    const int lead = m[0] != 0 ? m[0] : (m[1] != 0 ? m[1] : m[2]);
    if (lead == 0) half.insert(half.begin(), (int)k);
    else if (lead > 0) half.push_back((int)k);
  }
  p->nhalf_g = (int)half.size();  // (npw + 1) / 2: the sphere is closed under G -> -G

  // kernel tables on the stored half of the grid: [k1][k2][k3 <= N/2]
  const int kh = n / 2 + 1;
  const int64_t nhalf = (int64_t)n * n * kh;
  const int64_t ntot = (int64_t)n * n * n;
  std::vector<double> v64(nhalf), dv64(nhalf);
  for (int k1 = 0; k1 < n; ++k1)
    for (int k2 = 0; k2 < n; ++k2)
      for (int k3 = 0; k3 < kh; ++k3) {
        const double g2 = g2_of(p->recip, freq_of(k1, n), freq_of(k2, n), freq_of(k3, n));
        const int64_t i = ((int64_t)k1 * n + k2) * kh + k3;
        kernel_value(p, g2, &v64[i], &dv64[i]);
      }
  {
    double s2 = 0.0;  // ||v||_2^2 over the full grid from the stored half
    for (int k1 = 0; k1 < n; ++k1)
      for (int k2 = 0; k2 < n; ++k2)
        for (int k3 = 0; k3 < kh; ++k3) {
          const double v = v64[((int64_t)k1 * n + k2) * kh + k3];
          s2 += (k3 == 0 || 2 * k3 == n ? 1.0 : 2.0) * v * v;
        }
    p->vnorm = std::sqrt(s2);
  }
  // Columns (k2, k3 <= N/2) of the half spectrum a pair density can reach.
  // The product of two sphere orbitals has components only at |G| <= 2 Gmax,
  // so the columns that the ball |G|^2 <= 8 Ecut hits (indices modulo N, so a
  // grid that aliases the pair densities keeps what the aliases reach) are
  // kept; the others hold rounding noise only and are never stored,
  // transformed or read.  Row k2 keeps the prefix k3 < ncol[k2].
  std::vector<int> ncol(n, 0);
  {
    const double r2 = 8.0 * ecut_ha * (1.0 + 1e-9);
    int mb[3];
    for (int a = 0; a < 3; ++a) {
      const double len = std::sqrt(cell[3 * a] * cell[3 * a] + cell[3 * a + 1] * cell[3 * a + 1] +
                                   cell[3 * a + 2] * cell[3 * a + 2]);
      mb[a] = (int)std::floor(std::sqrt(r2) * len / (2.0 * kPi)) + 1;
    }
    std::vector<unsigned char> mark((size_t)n * n, 0);
    for (int m1 = -mb[0]; m1 <= mb[0]; ++m1)
      for (int m2 = -mb[1]; m2 <= mb[1]; ++m2)
        for (int m3 = -mb[2]; m3 <= mb[2]; ++m3)
          if (g2_of(p->recip, m1, m2, m3) <= r2)
            mark[(size_t)(((m2 % n) + n) % n) * n + (((m3 % n) + n) % n)] = 1;
    for (int k2 = 0; k2 < n; ++k2)
      for (int k3 = 0; k3 < kh; ++k3)
        if (mark[(size_t)k2 * n + k3]) ncol[k2] = k3 + 1;
  }
  std::vector<int> colmap, kept;
  for (int k2 = 0; k2 < n; ++k2)
    for (int s = 0; s < 2; ++s)
      for (int k3 = 0; k3 < ncol[k2]; ++k3) colmap.push_back((k2 << 16) | (s << 15) | k3);
  for (int k2 = 0; k2 < n; ++k2)
    for (int k3 = 0; k3 < ncol[k2]; ++k3) kept.push_back((k2 << 16) | k3);
  const int nlines = ops->col_lines;
  p->kept_columns = (int64_t)colmap.size();
  const int ncta_col = std::max(1, (int)((colmap.size() + nlines - 1) / nlines));
  colmap.resize((size_t)ncta_col * nlines, -1);

  const bool fp64 = prec == FOCK_PREC_FP64;
  // twiddles w[t] = exp(-2 pi i t / N)
  std::vector<double> tw64(2 * n);
  for (int t = 0; t < n; ++t) {
    const long double ang = 2.0L * 3.141592653589793238462643383279502884L * t / n;
    tw64[2 * t] = (double)std::cos(ang);
    tw64[2 * t + 1] = -(double)std::sin(ang);
  }

  fock_status st = FOCK_OK;
  auto upload = [&](void** dst, const void* src, size_t bytes) -> bool {
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      st = cuda_fail(nullptr, e, "uploading plan tables");
      return false;
    }
    p->table_bytes += (int64_t)bytes;
    return true;
  };
  cudaError_t ge = cudaGetDevice(&p->device);
  if (ge != cudaSuccess) {
    delete p;
    return cuda_fail(nullptr, ge, "cudaGetDevice");
  }
  bool ok = upload((void**)&p->d_gidx, gidx.data(), sizeof(int) * gidx.size()) &&
            upload((void**)&p->d_gidxneg, gneg.data(), sizeof(int) * gneg.size()) &&
            upload((void**)&p->d_half, half.data(), sizeof(int) * half.size()) &&
            upload((void**)&p->d_vtab64, v64.data(), sizeof(double) * nhalf);
  if (ok && kind == FOCK_KERNEL_ERFC) ok = upload((void**)&p->d_dvtab64, dv64.data(), sizeof(double) * nhalf);
  if (ok)
    ok = upload((void**)&p->d_ncol, ncol.data(), sizeof(int) * ncol.size()) &&
         upload((void**)&p->d_colmap, colmap.data(), sizeof(int) * colmap.size()) &&
         upload((void**)&p->d_kept, kept.data(), sizeof(int) * kept.size());
  if (ok) {
    if (fp64) {
      std::vector<double> vs(nhalf);
      for (int64_t i = 0; i < nhalf; ++i) vs[i] = v64[i] / (double)ntot;
      ok = upload(&p->d_vtab, vs.data(), sizeof(double) * nhalf) &&
           upload(&p->d_tw, tw64.data(), sizeof(double) * tw64.size());
    } else if (prec == FOCK_PREC_DF64) {
      // (hi, lo) float pairs: v / Ntot, dv/domega and the twiddles
      std::vector<float> vs(2 * nhalf), tw2(4 * n);
      for (int64_t i = 0; i < nhalf; ++i) split_df64(v64[i] / (double)ntot, &vs[2 * i]);
      for (int t = 0; t < 2 * n; ++t) split_df64(tw64[t], &tw2[2 * t]);
      ok = upload(&p->d_vtab, vs.data(), sizeof(float) * vs.size()) &&
           upload(&p->d_tw, tw2.data(), sizeof(float) * tw2.size());
      if (ok && kind == FOCK_KERNEL_ERFC) {
        std::vector<float> dvs(2 * nhalf);
        for (int64_t i = 0; i < nhalf; ++i) split_df64(dv64[i], &dvs[2 * i]);
        ok = upload(&p->d_dvtab, dvs.data(), sizeof(float) * dvs.size());
      }
    } else {
      std::vector<float> vs(nhalf), tw32(2 * n);
      for (int64_t i = 0; i < nhalf; ++i) vs[i] = (float)(v64[i] / (double)ntot);
      for (int t = 0; t < 2 * n; ++t) tw32[t] = (float)tw64[t];
      ok = upload(&p->d_vtab, vs.data(), sizeof(float) * nhalf) &&
           upload(&p->d_tw, tw32.data(), sizeof(float) * tw32.size());
      if (ok && kind == FOCK_KERNEL_ERFC) {
        std::vector<float> dvs(dv64.begin(), dv64.end());
        ok = upload(&p->d_dvtab, dvs.data(), sizeof(float) * nhalf);
      }
    }
  }
  if (ok) ok = upload((void**)&p->d_result, std::vector<double>(4, 0.0).data(), 4 * sizeof(double));
  if (ok) {
    cudaError_t e = cudaMallocHost((void**)&p->h_result, 4 * sizeof(double));
    if (e != cudaSuccess) {
      st = cuda_fail(nullptr, e, "cudaMallocHost");
      ok = false;
    }
  }
  if (!ok) {
    fock_destroy(p);
    return st;
  }

  DevPlan& d = p->dp;
  d.n = n;
  d.k3h = kh;
  d.ntot = ntot;
  d.hsize = (int64_t)n * n * 2 * kh;
  d.npw = p->npw;
  d.gidx = p->d_gidx;
  d.gidxneg = p->d_gidxneg;
  d.tw = p->d_tw;
  d.vtab = p->d_vtab;
  d.vtab64 = p->d_vtab64;
  d.dvtab64 = p->d_dvtab64;
  d.dvtab = fp64 ? (const void*)p->d_dvtab64 : (const void*)p->d_dvtab;
  d.inv_ntot = 1.0 / (double)ntot;
  d.psi_scale = 1.0 / std::sqrt(p->vol);
  d.out_scale = std::sqrt(p->vol) / (double)ntot;
  d.msmall2 = prec == FOCK_PREC_MIXED32 ? kMsmall2 : -1;
  d.ncol = p->d_ncol;
  d.colmap = p->d_colmap;
  d.ncta_col = ncta_col;
  d.kept = p->d_kept;
  d.nkept = (int)kept.size();
  {
    // kept rows as two runs [0, lo) and [n - hi, n); any other pattern keeps all rows
    int lo = 0, hi = 0, cmax = 0;
    while (lo < n && ncol[lo] > 0) ++lo;
    while (hi < n - lo && ncol[n - 1 - hi] > 0) ++hi;
    bool runs = true;
    for (int k2 = lo; k2 < n - hi; ++k2) runs = runs && ncol[k2] == 0;
    if (!runs) {
      lo = n;
      hi = 0;
    }
    for (int k2 = 0; k2 < n; ++k2) cmax = std::max(cmax, ncol[k2]);
    d.row_lo = lo;
    d.row_hi = hi;
    d.col_max = std::max(1, cmax);
  }
  d.det = 0;  // set per call on a copy when the plan is deterministic
  d.tile[0] = d.tile[1] = d.tile[2] = 0;
  d.det_scale = nullptr;

  int optin = 0, sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) {
    fock_destroy(p);
    return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
  }
  // Default chains per launch: a multiple of c0 = SMs / gcd(N, SMs), so the N
  // CTAs per chain of the plane passes fill whole waves (19 on a 152-SM GPU for
  // every compiled N), as many multiples as the buffer budget holds.
  const size_t chain_bytes = (size_t)d.hsize * 2 * (size_t)ops->real_bytes;
  {
    int a = n, b = std::max(1, sms);
    while (b != 0) {
      const int t = a % b;
      a = b;
      b = t;
    }
    const size_t c0 = (size_t)std::max(1, sms) / (size_t)a;
    const size_t fit = kChainBufferBytes / chain_bytes;
    p->chain_batch = (int)(fit >= c0 ? c0 * (fit / c0) : std::max<size_t>(1, fit));
  }
  if (ops->smem > (size_t)optin) {
    fock_destroy(p);
    return fail(nullptr, FOCK_ERR_UNSUPPORTED_SIZE, "the grid needs more shared memory than a CTA has");
  }
  e = ops->configure(d);
  if (e != cudaSuccess) {
    fock_destroy(p);
    return cuda_fail(nullptr, e, "configuring kernels");
  }
  *out = p;
  return FOCK_OK;
}

fock_status fock_gsphere(const int grid[3], const double cell[9], double ecut_ha, int64_t* npw,
                         int32_t* miller, int64_t capacity) {
  g_create_error.clear();
  if (!grid || !cell || !npw) return fail(nullptr, FOCK_ERR_INVALID_ARG, "NULL argument");
  if (!(ecut_ha > 0.0) || !std::isfinite(ecut_ha))
    return fail(nullptr, FOCK_ERR_INVALID_ARG, "ecut must be positive and finite");
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(cell[i])) return fail(nullptr, FOCK_ERR_INVALID_ARG, "cell is not finite");
  double recip[9], vol;
  reciprocal(cell, recip, &vol);
  if (!(std::fabs(vol) > 0.0)) return fail(nullptr, FOCK_ERR_INVALID_ARG, "the cell is degenerate");
  const int n = std::min(grid[0], std::min(grid[1], grid[2]));
  std::vector<GEntry> sph;
  if (!build_sphere(cell, recip, ecut_ha, n, sph))
    return fail(nullptr, FOCK_ERR_GRID_TOO_SMALL, "the G-sphere does not fit on the grid");
  *npw = (int64_t)sph.size();
  if (miller) {
    if (capacity < (int64_t)sph.size())
      return fail(nullptr, FOCK_ERR_INVALID_ARG, "miller buffer too small");
    for (size_t k = 0; k < sph.size(); ++k)
      for (int a = 0; a < 3; ++a) miller[3 * k + a] = sph[k].m[a];
  }
  return FOCK_OK;
}

fock_status fock_schedule(int nb, int band_block, int shard, int nshards, int32_t* pairs,
                          int64_t capacity, int64_t* npairs) {
  g_create_error.clear();
  if (!npairs) return fail(nullptr, FOCK_ERR_INVALID_ARG, "npairs is NULL");
  if (nb < 1 || nb > (1 << 15)) return fail(nullptr, FOCK_ERR_INVALID_ARG, "nb out of range");
  if (band_block == 0) band_block = kBandBlock;
  if (band_block < 1) return fail(nullptr, FOCK_ERR_INVALID_ARG, "band_block must be >= 1");
  if (nshards < 1 || shard < 0 || shard >= nshards)
    return fail(nullptr, FOCK_ERR_INVALID_ARG, "shard must satisfy 0 <= shard < nshards");
  std::vector<int2> all;
  schedule_pairs(nb, band_block, all);
  const int np = (int)all.size();
  const int nch = (np + 1) / 2;
  int c0 = 0, c1 = 0;
  shard_range(nch, shard, nshards, &c0, &c1);
  const int p0 = std::min(np, 2 * c0), p1 = std::min(np, 2 * c1);
  *npairs = p1 - p0;
  if (pairs) {
    if (capacity < p1 - p0) return fail(nullptr, FOCK_ERR_INVALID_ARG, "pairs buffer too small");
    for (int k = p0; k < p1; ++k) {
      pairs[2 * (k - p0)] = all[k].x;
      pairs[2 * (k - p0) + 1] = all[k].y;
    }
  }
  return FOCK_OK;
}

fock_status fock_plan_set_band_block(fock_plan_t plan, int band_block) {
  if (!plan) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (band_block < 1 || band_block > (1 << 15))
    return fail(plan, FOCK_ERR_INVALID_ARG, "band_block must be in [1, 32768]");
  if (band_block != plan->band_block) {
    plan->band_block = band_block;
    plan->sched_nb = -1;  // rebuilt at the next call
  }
  return FOCK_OK;
}

fock_status fock_plan_tiling_info(fock_plan_t plan, int pass, int tile, int* radices, int* nstages,
                                  int* threads_per_line, int* threads, int* ntiles) {
  if (!plan) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (!radices || !nstages || !threads_per_line || !threads || !ntiles)
    return fail(plan, FOCK_ERR_INVALID_ARG, "NULL output");
  if (pass < 0 || pass > 2 || tile < 0 || tile > 1) return fail(plan, FOCK_ERR_INVALID_ARG, "pass or tile out of range");
  int r[8], nst = 0, tl = 0, thr = 0;
  const int nt = plan->ops->tile_plan(pass, tile, r, &nst, &tl, &thr);
  if (tile >= nt) return fail(plan, FOCK_ERR_INVALID_ARG, "this plan has one tiling for that pass");
  for (int k = 0; k < nst; ++k) radices[k] = r[k];
  *nstages = nst;
  *threads_per_line = tl;
  *threads = thr;
  *ntiles = nt;
  return FOCK_OK;
}

fock_status fock_plan_set_tiling(fock_plan_t plan, const int tiles[3]) {
  if (!plan) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (!tiles) return fail(plan, FOCK_ERR_INVALID_ARG, "tiles is NULL");
  for (int pass = 0; pass < 3; ++pass) {
    int r[8], nst = 0, tl = 0, thr = 0;
    const int nt = plan->ops->tile_plan(pass, 0, r, &nst, &tl, &thr);
    if (tiles[pass] < 0 || tiles[pass] >= nt)
      return fail(plan, FOCK_ERR_INVALID_ARG, "a tile index is not below the pass's number of tilings");
  }
  for (int pass = 0; pass < 3; ++pass) plan->dp.tile[pass] = tiles[pass];
  return FOCK_OK;
}

fock_status fock_sternheimer_solve(fock_plan_t p, const double* vloc, const void* u_G, int nocc,
                                   const double* eps, const void* w_G, int nrhs, double alpha, double tol,
                                   int maxiter, void* g_G, int* iters, double* resid, fock_stream_t stream) {
  if (!p) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (p->prec != FOCK_PREC_FP64) return fail(p, FOCK_ERR_INVALID_ARG, "the Sternheimer solve needs an FP64 plan");
  if (!vloc || !u_G || !eps || !w_G || !g_G) return fail(p, FOCK_ERR_INVALID_ARG, "NULL argument");
  if (nocc < 1 || nrhs < 1 || nocc > (1 << 15) || nrhs > (1 << 15) || maxiter < 1)
    return fail(p, FOCK_ERR_INVALID_ARG, "nocc, nrhs and maxiter must be >= 1 (nocc, nrhs <= 32768)");
  if (!std::isfinite(alpha) || !(tol > 0.0) || !std::isfinite(tol))
    return fail(p, FOCK_ERR_INVALID_ARG, "alpha must be finite and tol positive");
  for (int n = 0; n < nrhs; ++n)
    if (!std::isfinite(eps[n])) return fail(p, FOCK_ERR_INVALID_ARG, "eps must be finite");
  const size_t npw = (size_t)p->npw;
  const size_t kb = npw * nrhs * sizeof(double2);
  {
    const char* g = static_cast<const char*>(g_G);
    const char* w = static_cast<const char*>(w_G);
    const char* u = static_cast<const char*>(u_G);
    const size_t ub = npw * nocc * sizeof(double2);
    if ((g < w + kb && w < g + kb) || (g < u + ub && u < g + kb))
      return fail(p, FOCK_ERR_INVALID_ARG, "g_G overlaps w_G or u_G");
  }
  fock_status st = check_device(p);
  if (st != FOCK_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = ensure_workspace(p, nrhs, 1);
  if (st != FOCK_OK) return st;
  p->fixed_nb = 0;  // the real-space workspace is overwritten
  const double2* u = static_cast<const double2*>(u_G);
  StBuffers buf;
  double2 *x, *r, *pk, *ap, *tmp;
  double *kin, *d_eps, *c, *rr, *rrn, *pap, *sc;
  int* perm;
  const size_t nb8 = sizeof(double) * nrhs;
  FOCK_CUDA(p, buf.alloc(&x, kb));
  FOCK_CUDA(p, buf.alloc(&r, kb));
  FOCK_CUDA(p, buf.alloc(&pk, kb));
  FOCK_CUDA(p, buf.alloc(&ap, kb));
  FOCK_CUDA(p, buf.alloc(&tmp, kb));
  FOCK_CUDA(p, buf.alloc(&kin, sizeof(double) * npw));
  FOCK_CUDA(p, buf.alloc(&d_eps, nb8));
  FOCK_CUDA(p, buf.alloc(&c, sizeof(double) * nocc * nrhs));
  FOCK_CUDA(p, buf.alloc(&rr, nb8));
  FOCK_CUDA(p, buf.alloc(&rrn, nb8));
  FOCK_CUDA(p, buf.alloc(&pap, nb8));
  FOCK_CUDA(p, buf.alloc(&sc, nb8));
  FOCK_CUDA(p, buf.alloc(&perm, sizeof(int) * nrhs));
  // |G|^2 / 2 on the sphere, in the plan's canonical order
  std::vector<double> kin_h(npw);
  for (size_t g = 0; g < npw; ++g)
    kin_h[g] = 0.5 * fockx::lattice::g2_of(p->recip, p->miller[3 * g], p->miller[3 * g + 1], p->miller[3 * g + 2]);
  std::vector<double> eps_h(eps, eps + nrhs);
  FOCK_CUDA(p, cudaMemcpyAsync(kin, kin_h.data(), sizeof(double) * npw, cudaMemcpyHostToDevice, s));
  FOCK_CUDA(p, cudaMemcpyAsync(d_eps, eps_h.data(), nb8, cudaMemcpyHostToDevice, s));

  const int ip = (int)npw;
  const int nbat = bands_per_grid_batch(p);
  // (H - eps_n + alpha P) on the kets q at positions [0, m) into out
  auto apply_a = [&](const double2* q, int m, double2* out) -> fock_status {
    for (int b0 = 0; b0 < m; b0 += nbat)
      FOCK_CUDA(p, p->ops->to_real(p->dp, q, m, b0, std::min(nbat, m - b0), p->ws.h, p->ws.psi, s));
    FOCK_CUDA(p, fockx::st_vmul(vloc, static_cast<const double*>(p->ws.psi), static_cast<double*>(p->ws.w), m,
                                p->dp.ntot, s));
    for (int b0 = 0; b0 < m; b0 += nbat)
      FOCK_CUDA(p, p->ops->to_sphere(p->dp, p->ws.w, m, b0, std::min(nbat, m - b0), p->ws.h, out, s));
    FOCK_CUDA(p, fockx::st_proj_coef(u, nocc, q, m, ip, c, s));
    FOCK_CUDA(p, fockx::st_finish(out, q, kin, d_eps, u, c, nocc, alpha, m, ip, s));
    return FOCK_OK;
  };

  // b = -Q w into r; x = 0; p = r; rr = <r|r>
  FOCK_CUDA(p, fockx::st_proj_coef(u, nocc, static_cast<const double2*>(w_G), nrhs, ip, c, s));
  FOCK_CUDA(p, fockx::st_rhs(static_cast<const double2*>(w_G), u, c, nocc, nrhs, ip, r, s));
  FOCK_CUDA(p, cudaMemsetAsync(x, 0, kb, s));
  FOCK_CUDA(p, cudaMemcpyAsync(pk, r, kb, cudaMemcpyDeviceToDevice, s));
  FOCK_CUDA(p, fockx::st_dots(r, r, nrhs, ip, rr, s));

  // order[k]: the band at position k; positions [0, m) are not converged
  std::vector<int> order(nrhs), it_h(nrhs, 0), keep;
  for (int n = 0; n < nrhs; ++n) order[n] = n;
  std::vector<double> rr_h(nrhs);
  int m = nrhs;
  for (int it = 0; it < maxiter && m > 0; ++it) {
    st = apply_a(pk, m, ap);
    if (st != FOCK_OK) return st;
    FOCK_CUDA(p, fockx::st_dots(pk, ap, m, ip, pap, s));
    FOCK_CUDA(p, fockx::st_step(x, r, pk, ap, rr, pap, m, ip, s));
    FOCK_CUDA(p, fockx::st_dots(r, r, m, ip, rrn, s));
    FOCK_CUDA(p, fockx::st_dir(pk, r, rrn, rr, m, ip, s));
    FOCK_CUDA(p, cudaMemcpyAsync(rr, rrn, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    FOCK_CUDA(p, cudaMemcpyAsync(rr_h.data(), rrn, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    FOCK_CUDA(p, cudaStreamSynchronize(s));
    for (int k = 0; k < m; ++k) ++it_h[order[k]];
    // regroup: not converged first, then converged, each in their order
    keep.clear();
    for (int k = 0; k < m; ++k)
      if (!(std::sqrt(rr_h[k]) < tol)) keep.push_back(k);
    const int m_new = (int)keep.size();
    for (int k = 0; k < m; ++k)
      if (std::sqrt(rr_h[k]) < tol) keep.push_back(k);
    bool moved = false;
    for (int k = 0; k < m; ++k) moved = moved || keep[k] != k;
    if (moved) {
      FOCK_CUDA(p, cudaMemcpyAsync(perm, keep.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
      double2* rows[3] = {x, r, pk};
      for (double2* a : rows) {
        FOCK_CUDA(p, fockx::st_gather_rows(a, tmp, perm, m, ip, s));
        FOCK_CUDA(p, cudaMemcpyAsync(a, tmp, npw * m * sizeof(double2), cudaMemcpyDeviceToDevice, s));
      }
      double* scal[2] = {rr, d_eps};
      for (double* a : scal) {
        FOCK_CUDA(p, fockx::st_gather_scalars(a, sc, perm, m, s));
        FOCK_CUDA(p, cudaMemcpyAsync(a, sc, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
      }
      std::vector<int> o2(order);
      std::vector<double> r2(rr_h);
      for (int k = 0; k < m; ++k) {
        o2[k] = order[keep[k]];
        r2[k] = rr_h[keep[k]];
      }
      order.swap(o2);
      rr_h.swap(r2);
    }
    m = m_new;
  }
  // back to the original band order: g[order[k]] = x[k]
  std::vector<int> inv(nrhs);
  for (int k = 0; k < nrhs; ++k) inv[order[k]] = k;
  FOCK_CUDA(p, cudaMemcpyAsync(perm, inv.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
  FOCK_CUDA(p, fockx::st_gather_rows(x, static_cast<double2*>(g_G), perm, nrhs, ip, s));
  FOCK_CUDA(p, cudaMemcpyAsync(rr_h.data(), rr, nb8, cudaMemcpyDeviceToHost, s));
  FOCK_CUDA(p, cudaStreamSynchronize(s));
  for (int k = 0; k < nrhs; ++k) {
    if (iters) iters[order[k]] = it_h[order[k]];
    if (resid) resid[order[k]] = std::sqrt(rr_h[k]);
  }
  return FOCK_OK;
}

fock_status fock_plan_set_batch(fock_plan_t plan, int chain_batch) {
  if (!plan) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (chain_batch < 1 || chain_batch > 4096)
    return fail(plan, FOCK_ERR_INVALID_ARG, "chain_batch must be in [1, 4096]");
  if (chain_batch != plan->chain_batch) {
    cudaFree(plan->ws.h);  // stream-ordered work using it has been queued by earlier calls;
    plan->ws.h = nullptr;  // cudaFree waits for the device to finish with it
    for (void*& x : plan->ws.hx) {
      cudaFree(x);
      x = nullptr;
    }
    plan->ws.h_bytes = 0;
    plan->chain_batch = chain_batch;
  }
  return FOCK_OK;
}

fock_status fock_plan_set_streams(fock_plan_t plan, int streams) {
  if (!plan) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (streams < 1 || streams > 4) return fail(plan, FOCK_ERR_INVALID_ARG, "streams must be 1 to 4");
  plan->streams = streams;
  return FOCK_OK;
}

fock_status fock_plan_set_timing(fock_plan_t plan, int enable) {
  if (!plan) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  plan->timing = enable != 0;
  return FOCK_OK;
}

fock_status fock_plan_stats(fock_plan_t plan, fock_stats* stats) {
  if (!plan || !stats) return fail(plan, FOCK_ERR_INVALID_ARG, "NULL argument");
  *stats = plan->stats;
  return FOCK_OK;
}

fock_status fock_plan_npw(fock_plan_t plan, int64_t* npw) {
  if (!plan || !npw) return fail(plan, FOCK_ERR_INVALID_ARG, "NULL argument");
  *npw = plan->npw;
  return FOCK_OK;
}

fock_status fock_plan_gvectors(fock_plan_t plan, int32_t* miller) {
  if (!plan || !miller) return fail(plan, FOCK_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(miller, plan->miller.data(), sizeof(int32_t) * plan->miller.size());
  return FOCK_OK;
}

fock_status fock_plan_reserve(fock_plan_t plan, int nb_max) {
  if (!plan) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (nb_max < 1 || nb_max > (1 << 15)) return fail(plan, FOCK_ERR_INVALID_ARG, "nb_max out of range");
  fock_status st = check_device(plan);
  if (st != FOCK_OK) return st;
  return ensure_workspace(plan, nb_max, nb_max * (nb_max + 1) / 2);
}

fock_status fock_plan_set_deterministic(fock_plan_t plan, int enable) {
  if (!plan) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (enable && plan->prec == FOCK_PREC_MIXED32)
    return fail(plan, FOCK_ERR_INVALID_ARG, "deterministic accumulation is offered for FP64 and double-float plans");
  plan->det = enable != 0;
  return FOCK_OK;
}

fock_status fock_plan_columns(fock_plan_t plan, int64_t* kept, int64_t* total) {
  if (!plan) return fail(nullptr, FOCK_ERR_INVALID_ARG, "plan is NULL");
  if (kept) *kept = plan->kept_columns;
  if (total) *total = (int64_t)plan->n * 2 * (plan->n / 2 + 1);
  return FOCK_OK;
}

fock_status fock_plan_device_bytes(fock_plan_t plan, int64_t* bytes) {
  if (!plan || !bytes) return fail(plan, FOCK_ERR_INVALID_ARG, "NULL argument");
  const Workspace& w = plan->ws;
  int64_t b = plan->table_bytes + 2 * (int64_t)w.psi_bytes + (int64_t)w.h_bytes;
  b += (int64_t)w.npair_cap * (2 * sizeof(double) + sizeof(int2)) +
       (int64_t)((w.npair_cap + 1) / 2) * sizeof(Chain);
  b += (int64_t)w.nb_cap * (sizeof(double) + plan->ops->real_bytes);
  *bytes = b;
  return FOCK_OK;
}

fock_status fock_apply(fock_plan_t plan, const void* psi_G, int nb, const double* occ,
                       void* vpsi_G, double* ex, double* dex, fock_stream_t stream) {
  return apply_impl(plan, psi_G, nb, occ, 0, 1, vpsi_G, ex, dex, stream);
}

fock_status fock_apply_shard(fock_plan_t plan, const void* psi_G, int nb, const double* occ,
                             int shard, int nshards, void* vpsi_G, double* ex, double* dex,
                             fock_stream_t stream) {
  return apply_impl(plan, psi_G, nb, occ, shard, nshards, vpsi_G, ex, dex, stream);
}

fock_status fock_set_occupied(fock_plan_t plan, const void* psi_G, int nb, const double* occ,
                              fock_stream_t stream) {
  fock_status st = validate_apply(plan, psi_G, nb, psi_G);
  if (st != FOCK_OK) return st;
  if (!occ) return fail(plan, FOCK_ERR_INVALID_ARG, "occ is NULL");
  for (int i = 0; i < nb; ++i)
    if (!std::isfinite(occ[i])) return fail(plan, FOCK_ERR_INVALID_ARG, "occupations must be finite");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  stats_reset(plan);
  plan->fixed_nb = 0;
  st = ensure_workspace(plan, nb, 1);
  if (st != FOCK_OK) return st;
  st = upload_occ(plan, occ, nb, s);
  if (st != FOCK_OK) return st;
  st = orbitals_to_real(plan, psi_G, nb, s);
  if (st != FOCK_OK) return st;
  if (plan->ops->prec == 1) {
    // the coefficients of the occupied set, for the FP64 overlaps of the
    // fixed operator's G = 0 terms
    const int64_t need = (int64_t)nb * plan->npw;
    if (need > plan->cocc_cap) {
      cudaFree(plan->d_cocc);
      plan->d_cocc = nullptr;
      plan->cocc_cap = 0;
      FOCK_CUDA(plan, dev_alloc(&plan->d_cocc, sizeof(double2) * (size_t)need));
      plan->cocc_cap = need;
    }
    FOCK_CUDA(plan, cudaMemcpyAsync(plan->d_cocc, psi_G, sizeof(double2) * (size_t)need, cudaMemcpyDeviceToDevice, s));
  }
  plan->fixed_nb = nb;
  plan->fixed_sched_nt = -1;
  return FOCK_OK;
}

fock_status fock_apply_fixed(fock_plan_t plan, const void* phi_G, int nt, void* vphi_G,
                             fock_stream_t stream) {
  fock_plan* p = plan;
  fock_status st = validate_apply(p, phi_G, nt, vphi_G);
  if (st != FOCK_OK) return st;
  if (p->fixed_nb < 1) return fail(p, FOCK_ERR_INVALID_ARG, "no occupied set: call fock_set_occupied first");
  const size_t bytes = (size_t)nt * (size_t)p->npw * 16;
  const char* a = static_cast<const char*>(phi_G);
  const char* b = static_cast<const char*>(vphi_G);
  if (a < b + bytes && b < a + bytes) return fail(p, FOCK_ERR_INVALID_ARG, "phi_G and vphi_G overlap");
  const int nb = p->fixed_nb;
  if ((int64_t)nb * nt > (int64_t)1 << 30) return fail(p, FOCK_ERR_INVALID_ARG, "too many pairs");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  stats_reset(p);
  st = grow_keeping(p, nb + nt, nb);
  if (st != FOCK_OK) return st;
  const int npairs = nb * nt;
  st = ensure_workspace(p, nb + nt, npairs);
  if (st != FOCK_OK) return st;
  if (p->fixed_sched_nt != nt || p->fixed_sched_bb != p->band_block) {
    // pairs (occupied i, trial a) in band_block x band_block blocks, one-sided
    std::vector<int2> pairs;
    pairs.reserve(npairs);
    const int bb = p->band_block;
    for (int i0 = 0; i0 < nb; i0 += bb)
      for (int a0 = 0; a0 < nt; a0 += bb)
        for (int i = i0; i < std::min(nb, i0 + bb); ++i)
          for (int t = a0; t < std::min(nt, a0 + bb); ++t) pairs.push_back(make_int2(i, nb + t));
    chains_from_pairs(pairs, p->chains);
    for (Chain& c : p->chains) {
      c.flags = fockx::kChainOneSidedA | fockx::kChainOneSidedB;
      c.pa = c.pb = -1;
    }
    FOCK_CUDA(p, cudaMemcpyAsync(p->ws.chains, p->chains.data(), sizeof(Chain) * p->chains.size(),
                                 cudaMemcpyHostToDevice, s));
    FOCK_CUDA(p, cudaStreamSynchronize(s));
    p->sched_nb = -1;  // the symmetric schedule on the device is gone
    p->fixed_sched_nt = nt;
    p->fixed_sched_bb = p->band_block;
  }
  const size_t rb = (size_t)p->ops->real_bytes;
  const size_t off = (size_t)nb * (size_t)p->dp.ntot * rb;
  char* psi_trial = static_cast<char*>(p->ws.psi) + off;
  char* w_trial = static_cast<char*>(p->ws.w) + off;
  FOCK_CUDA(p, cudaMemsetAsync(w_trial, 0, (size_t)nt * (size_t)p->dp.ntot * rb, s));
  const int nbat = bands_per_grid_batch(p);
  p->stats.band_batch = nbat;
  for (int b0 = 0; b0 < nt; b0 += nbat) {
    PhaseScope ps(p, FOCK_PHASE_TO_REAL, 3, s);
    FOCK_CUDA(p, p->ops->to_real(p->dp, static_cast<const double2*>(phi_G), nt, b0, std::min(nbat, nt - b0),
                                 p->ws.h, psi_trial, s));
  }
  DevPlan dp = p->dp;
  dp.dvtab64 = nullptr;
  if (p->det) {
    st = det_buffers(p, nb + nt, 1);
    if (st != FOCK_OK) return st;
    st = det_prepare(p, nb + nt, nb, &dp, s);
    if (st != FOCK_OK) return st;
  }
  if (p->ops->prec == 1 && p->d_cocc != nullptr) {
    // FP64 overlaps of the pairs (occupied i, trial nb + t) for the G = 0 terms
    PhaseScope ps(p, FOCK_PHASE_TO_REAL, 2, s);
    st = prepare_overlaps(p, p->d_cocc, nb, phi_G, nt, false, nb, &dp, s);
    if (st != FOCK_OK) return st;
  }
  st = prepare_prescaled(p, p->occ_host.data(), nb, &dp, s);  // the occupied set's occupations
  if (st != FOCK_OK) return st;
  const int nch = (int)p->chains.size();
  p->stats.chain_batch = p->chain_batch;
  p->stats.chains = nch;
  p->stats.pairs = npairs;
  for (int c = 0; c < nch; c += p->chain_batch) {
    const int cnt = std::min(p->chain_batch, nch - c);
    const Chain* ch = p->ws.chains + c;
    {
      PhaseScope ps(p, FOCK_PHASE_PAIR_FWD, 1, s);
      FOCK_CUDA(p, p->ops->pair_fwd(dp, p->ws.psi, ch, cnt, p->ws.h, s));
    }
    {
      PhaseScope ps(p, FOCK_PHASE_PAIR_COL, 1, s);
      FOCK_CUDA(p, p->ops->pair_col(dp, p->ws.h, ch, cnt, p->ws.epair, p->ws.dpair, s));
    }
    {
      PhaseScope ps(p, FOCK_PHASE_PAIR_INV, 1, s);
      FOCK_CUDA(p, p->ops->pair_inv(dp, p->ws.psi, p->ws.w, p->ws.occT, ch, cnt, p->ws.h, s));
    }
  }
  if (p->det) FOCK_CUDA(p, fockx::launch_det_to_double(w_trial, (int64_t)nt * p->dp.ntot, p->d_scale, s));
  for (int b0 = 0; b0 < nt; b0 += nbat) {
    PhaseScope ps(p, FOCK_PHASE_TO_SPHERE, 3, s);
    FOCK_CUDA(p, p->ops->to_sphere(p->dp, w_trial, nt, b0, std::min(nbat, nt - b0), p->ws.h,
                                   static_cast<double2*>(vphi_G), s));
  }
  return collect_timing(p, s);
}

fock_status fock_pair_energies(fock_plan_t plan, const void* psi_G, int nb, const int32_t* pairs,
                               int npairs, double* e, double* d, fock_stream_t stream) {
  fock_status st = validate_apply(plan, psi_G, nb, e);
  if (st != FOCK_OK) return st;
  if (!pairs || npairs < 1) return fail(plan, FOCK_ERR_INVALID_ARG, "pairs is empty");
  std::vector<int2> list(npairs);
  for (int k = 0; k < npairs; ++k) {
    const int i = pairs[2 * k], j = pairs[2 * k + 1];
    if (i < 0 || j < 0 || i >= nb || j >= nb)
      return fail(plan, FOCK_ERR_INVALID_ARG, "a band index is out of range");
    list[k] = make_int2(i, j);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = ensure_workspace(plan, nb, npairs);
  if (st != FOCK_OK) return st;
  std::vector<Chain> chains;
  chains_from_pairs(list, chains);
  plan->sched_nb = -1;  // the device chain list is overwritten below
  plan->fixed_nb = 0;   // and the real-space workspace
  plan->fixed_sched_nt = -1;
  stats_reset(plan);
  FOCK_CUDA(plan, cudaMemcpyAsync(plan->ws.chains, chains.data(), sizeof(Chain) * chains.size(),
                                  cudaMemcpyHostToDevice, s));
  FOCK_CUDA(plan, cudaMemsetAsync(plan->ws.epair, 0, sizeof(double) * npairs, s));
  FOCK_CUDA(plan, cudaMemsetAsync(plan->ws.dpair, 0, sizeof(double) * npairs, s));
  st = orbitals_to_real(plan, psi_G, nb, s);
  if (st != FOCK_OK) return st;
  const int nch = (int)chains.size();
  for (int c = 0; c < nch; c += plan->chain_batch) {
    const int cnt = std::min(plan->chain_batch, nch - c);
    const Chain* ch = plan->ws.chains + c;
    {
      PhaseScope ps(plan, FOCK_PHASE_PAIR_FWD, 1, s);
      FOCK_CUDA(plan, plan->ops->pair_fwd(plan->dp, plan->ws.psi, ch, cnt, plan->ws.h, s));
    }
    {
      PhaseScope ps(plan, FOCK_PHASE_PAIR_COL, 1, s);
      FOCK_CUDA(plan, plan->ops->pair_col(plan->dp, plan->ws.h, ch, cnt, plan->ws.epair,
                                          plan->ws.dpair, s));
    }
  }
  plan->stats.chains = nch;
  plan->stats.pairs = npairs;
  plan->stats.chain_batch = plan->chain_batch;
  st = collect_timing(plan, s);
  if (st != FOCK_OK) return st;
  std::vector<double> he(npairs), hd(npairs);
  FOCK_CUDA(plan, cudaMemcpyAsync(he.data(), plan->ws.epair, sizeof(double) * npairs,
                                  cudaMemcpyDeviceToHost, s));
  FOCK_CUDA(plan, cudaMemcpyAsync(hd.data(), plan->ws.dpair, sizeof(double) * npairs,
                                  cudaMemcpyDeviceToHost, s));
  FOCK_CUDA(plan, cudaStreamSynchronize(s));
  const double inv2 = 1.0 / ((double)plan->dp.ntot * (double)plan->dp.ntot);
  for (int k = 0; k < npairs; ++k) {
    e[k] = he[k] * inv2;
    if (d) d[k] = plan->dp.dvtab64 ? hd[k] * inv2 : 0.0;
  }
  return FOCK_OK;
}

fock_status fock_destroy(fock_plan_t plan) {
  if (!plan) return FOCK_OK;
  for (cudaEvent_t e : plan->events) cudaEventDestroy(e);
  if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
  for (int k = 0; k < 3; ++k) {
    if (plan->ev_join[k]) cudaEventDestroy(plan->ev_join[k]);
    if (plan->aux[k]) cudaStreamDestroy(plan->aux[k]);
  }
  free_ws(plan->ws);
  cudaFree(plan->d_gidx);
  cudaFree(plan->d_gidxneg);
  cudaFree(plan->d_tw);
  cudaFree(plan->d_vtab);
  cudaFree(plan->d_vtab64);
  cudaFree(plan->d_dvtab);
  cudaFree(plan->d_dvtab64);
  cudaFree(plan->d_ncol);
  cudaFree(plan->d_colmap);
  cudaFree(plan->d_kept);
  cudaFree(plan->d_stats);
  cudaFree(plan->d_scale);
  cudaFree(plan->d_epart);
  cudaFree(plan->d_dpart);
  cudaFree(plan->d_ovl);
  cudaFree(plan->d_half);
  cudaFree(plan->d_cocc);
  cudaFree(plan->d_vtab_f);
  cudaFree(plan->d_result);
  if (plan->h_result) cudaFreeHost(plan->h_result);
  delete plan;
  return FOCK_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct fock_batch {
  int nsys = 0;
  int device = 0;
  int prec = 0;
  std::vector<fock_plan*> plans;
  std::vector<int> nb;
  std::vector<const void*> psi;
  std::vector<void*> vpsi;
  fock_batch_options opt{};
  const fockx::PersistOps* pops = nullptr;
  fockx::SysDesc* d_sys = nullptr;
  fockx::Segment* d_seg = nullptr;
  unsigned* d_counters = nullptr;
  unsigned char* d_ring = nullptr;
  double* d_result = nullptr;
  double* h_result = nullptr;  // pinned [2 nsys]
  unsigned* h_err = nullptr;   // pinned
  std::vector<fockx::Segment> segs;
  int ntasks = 0;
  int grid = 0;
  size_t slot_bytes = 0;
  int64_t launches = 0;
  cudaStream_t cap_stream = nullptr;
  std::vector<cudaStream_t> branch;          // per-system streams (non-persistent mode)
  std::vector<cudaEvent_t> branch_ev;        // fork / join events of the branches
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the pair passes
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string err;
};

namespace {

fock_status bfail(fock_batch* b, fock_status s, const std::string& msg) {
  if (b) b->err = msg;
  else g_create_error = msg;
  return s;
}

fock_status bcuda(fock_batch* b, cudaError_t e, const char* what) {
  cudaGetLastError();
  const fock_status s = (e == cudaErrorMemoryAllocation) ? FOCK_ERR_OOM : FOCK_ERR_CUDA;
  return bfail(b, s, std::string(what) + ": " + cudaGetErrorString(e));
}

#define FOCK_BCUDA(b, call)                              \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call);   \
  } while (0)

void batch_free(fock_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  for (cudaStream_t st : b->branch) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->branch_ev) cudaEventDestroy(ev);
  cudaFree(b->d_sys);
  cudaFree(b->d_seg);
  cudaFree(b->d_counters);
  cudaFree(b->d_ring);
  cudaFree(b->d_result);
  if (b->h_result) cudaFreeHost(b->h_result);
  if (b->h_err) cudaFreeHost(b->h_err);
}

// Queue the whole batched apply on stream s (also used under graph capture).
fock_status batch_enqueue(fock_batch* b, cudaStream_t s) {
  const int nseg = (int)b->segs.size();
  b->launches = 0;
  FOCK_BCUDA(b, cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned) * (2 + nseg), s));
  for (int k = 0; k < b->nsys; ++k) {
    fock_plan* p = b->plans[k];
    const int nb = b->nb[k];
    const int npairs = nb * (nb + 1) / 2;
    const size_t rb = (size_t)p->ops->real_bytes;
    FOCK_BCUDA(b, cudaMemsetAsync(p->ws.w, 0, (size_t)nb * (size_t)p->dp.ntot * rb, s));
    FOCK_BCUDA(b, cudaMemsetAsync(p->ws.epair, 0, sizeof(double) * npairs, s));
    FOCK_BCUDA(b, cudaMemsetAsync(p->ws.dpair, 0, sizeof(double) * npairs, s));
    const int nbat = bands_per_grid_batch(p);
    for (int b0 = 0; b0 < nb; b0 += nbat) {
      FOCK_BCUDA(b, p->ops->to_real(p->dp, static_cast<const double2*>(b->psi[k]), nb, b0,
                                    std::min(nbat, nb - b0), p->ws.h, p->ws.psi, s));
      b->launches += 3;
    }
    if (p->ops->prec == 1) {
      FOCK_BCUDA(b, fockx::launch_overlap(static_cast<const double2*>(b->psi[k]), nb,
                                          static_cast<const double2*>(b->psi[k]), nb, p->npw, p->d_half, p->nhalf_g,
                                          true, p->d_ovl, nb, s));
      b->launches += 2;
    }
  }
  const unsigned long long limit_ns = (unsigned long long)(b->opt.wait_limit_s * 1e9);
  // external event nodes when captured, so the elapsed time is readable after a replay
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  FOCK_BCUDA(b, cudaStreamIsCapturing(s, &cap));
  const unsigned ev_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
  FOCK_BCUDA(b, cudaEventRecordWithFlags(b->ev0, s, ev_flags));
  if (b->opt.persistent == 2) {
    FOCK_BCUDA(b, b->pops->launch_dataflow(b->d_sys, b->d_seg, nseg, b->ntasks, b->d_counters, b->d_ring,
                                           b->slot_bytes, limit_ns, s));
    b->launches += 1;
  } else if (b->opt.persistent) {
    FOCK_BCUDA(b, b->pops->launch(b->grid, b->d_sys, b->d_seg, nseg, b->ntasks, b->d_counters,
                                  b->d_ring, b->slot_bytes, limit_ns, s));
    b->launches += 1;
  } else {
    // fork one branch per system, each running its size-specialised pair passes
    // over its own transform buffer, and join them back into s
    FOCK_BCUDA(b, cudaEventRecord(b->branch_ev[0], s));
    for (int k = 0; k < b->nsys; ++k) {
      fock_plan* p = b->plans[k];
      cudaStream_t bs = b->branch[k];
      FOCK_BCUDA(b, cudaStreamWaitEvent(bs, b->branch_ev[0], 0));
      fockx::DevPlan dp = p->dp;
      if (!b->opt.want_dex) dp.dvtab64 = nullptr;
      if (p->ops->prec == 1) {
        dp.ovl = p->d_ovl;
        dp.ovl_ld = b->nb[k];
        dp.ovl_j0 = 0;
        dp.ovl_scale = (double)p->dp.ntot / p->vol;
      }
      const int nch = (int)p->chains.size();
      for (int c = 0; c < nch; c += p->chain_batch) {
        const int cnt = std::min(p->chain_batch, nch - c);
        const Chain* ch = p->ws.chains + c;
        FOCK_BCUDA(b, p->ops->pair_fwd(dp, p->ws.psi, ch, cnt, p->ws.h, bs));
        FOCK_BCUDA(b, p->ops->pair_col(dp, p->ws.h, ch, cnt, p->ws.epair, p->ws.dpair, bs));
        FOCK_BCUDA(b, p->ops->pair_inv(dp, p->ws.psi, p->ws.w, p->ws.occT, ch, cnt, p->ws.h, bs));
        b->launches += 3;
      }
      FOCK_BCUDA(b, cudaEventRecord(b->branch_ev[1 + k], bs));
      FOCK_BCUDA(b, cudaStreamWaitEvent(s, b->branch_ev[1 + k], 0));
    }
  }
  FOCK_BCUDA(b, cudaEventRecordWithFlags(b->ev1, s, ev_flags));
  for (int k = 0; k < b->nsys; ++k) {
    fock_plan* p = b->plans[k];
    const int nb = b->nb[k];
    const int npairs = nb * (nb + 1) / 2;
    const int nbat = bands_per_grid_batch(p);
    for (int b0 = 0; b0 < nb; b0 += nbat) {
      FOCK_BCUDA(b, p->ops->to_sphere(p->dp, p->ws.w, nb, b0, std::min(nbat, nb - b0), p->ws.h,
                                      static_cast<double2*>(b->vpsi[k]), s));
      b->launches += 3;
    }
    const double scale = -0.5 * p->vol / ((double)p->dp.ntot * (double)p->dp.ntot);
    FOCK_BCUDA(b, fockx::launch_energy_reduce(p->ws.pairs, npairs, p->ws.occ, p->ws.epair,
                                              b->opt.want_dex && p->dp.dvtab64 ? p->ws.dpair : nullptr,
                                              scale, b->d_result + 2 * k, s));
    b->launches += 1;
  }
  FOCK_BCUDA(b, cudaMemcpyAsync(b->h_result, b->d_result, sizeof(double) * 2 * b->nsys,
                                cudaMemcpyDeviceToHost, s));
  FOCK_BCUDA(b, cudaMemcpyAsync(b->h_err, b->d_counters + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  return FOCK_OK;
}

}  // namespace

extern "C" {

fock_status fock_batch_default_options(fock_batch_options* opt) {
  if (!opt) return bfail(nullptr, FOCK_ERR_INVALID_ARG, "opt is NULL");
  opt->slot_chains = 8;
  opt->ring = 3;
  opt->ctas_per_sm = 0;
  opt->use_graph = 1;
  opt->want_dex = 0;
  opt->wait_limit_s = 10.0;
  opt->stall_segment = -1;
  opt->persistent = 1;
  return FOCK_OK;
}

fock_status fock_batch_create(fock_batch_t* out, int nsys, const fock_plan_t* plans, const int* nb,
                              const void* const* psi_G, const double* const* occ,
                              void* const* vpsi_G, const fock_batch_options* opt) {
  g_create_error.clear();
  if (!out) return bfail(nullptr, FOCK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nsys < 1 || !plans || !nb || !psi_G || !occ || !vpsi_G)
    return bfail(nullptr, FOCK_ERR_INVALID_ARG, "empty batch or NULL array");
  fock_batch_options o;
  fock_batch_default_options(&o);
  if (opt) o = *opt;
  if (o.slot_chains < 1 || o.ring < 3 || o.ctas_per_sm < 0 || !(o.wait_limit_s > 0.0) || o.persistent < 0 ||
      o.persistent > 2)
    return bfail(nullptr, FOCK_ERR_INVALID_ARG, "bad batch options");
  int dev = -1;
  cudaError_t ge = cudaGetDevice(&dev);
  if (ge != cudaSuccess) return bcuda(nullptr, ge, "cudaGetDevice");
  for (int k = 0; k < nsys; ++k) {
    if (!plans[k] || !psi_G[k] || !vpsi_G[k] || !occ[k] || nb[k] < 1 || nb[k] > (1 << 15))
      return bfail(nullptr, FOCK_ERR_INVALID_ARG, "system " + std::to_string(k) + ": bad argument");
    for (int m = 0; m < k; ++m)
      if (plans[m] == plans[k]) return bfail(nullptr, FOCK_ERR_INVALID_ARG, "a plan appears twice");
    if (plans[k]->device != dev) return bfail(nullptr, FOCK_ERR_INVALID_ARG, "plans on another device");
    if (plans[k]->prec != plans[0]->prec)
      return bfail(nullptr, FOCK_ERR_INVALID_ARG, "plans of different precision");
    if (!fockx::persist_supports(plans[k]->n))
      return bfail(nullptr, FOCK_ERR_UNSUPPORTED_SIZE, "batched grids must be 24, 32, 48, 64, 72 or 96");
  }
  if (plans[0]->prec == FOCK_PREC_DF64)
    return bfail(nullptr, FOCK_ERR_INVALID_ARG, "batches run the FP64 and mixed forms only");
  fock_batch* b = new (std::nothrow) fock_batch();
  if (!b) return bfail(nullptr, FOCK_ERR_OOM, "host allocation failed");
  b->nsys = nsys;
  b->device = dev;
  b->prec = plans[0]->prec == FOCK_PREC_FP64 ? 0 : 1;
  b->opt = o;
  b->plans.assign(plans, plans + nsys);
  b->nb.assign(nb, nb + nsys);
  b->psi.assign(psi_G, psi_G + nsys);
  b->vpsi.assign(vpsi_G, vpsi_G + nsys);
  auto fail_create = [&](fock_status st) {
    g_create_error = b->err;
    batch_free(b);
    delete b;
    return st;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail_create(bcuda(b, e, "cudaStreamCreate"));
  if ((e = cudaEventCreate(&b->ev0)) != cudaSuccess || (e = cudaEventCreate(&b->ev1)) != cudaSuccess)
    return fail_create(bcuda(b, e, "cudaEventCreate"));
  if (!o.persistent) {
    for (int k = 0; k < nsys; ++k) {
      cudaStream_t st = nullptr;
      if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
        return fail_create(bcuda(b, e, "cudaStreamCreate"));
      b->branch.push_back(st);
    }
    for (int k = 0; k < nsys + 1; ++k) {
      cudaEvent_t ev = nullptr;
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return fail_create(bcuda(b, e, "cudaEventCreate"));
      b->branch_ev.push_back(ev);
    }
  }
  b->pops = fockx::find_persist_ops(b->prec);
  if ((e = b->pops->configure()) != cudaSuccess) return fail_create(bcuda(b, e, "configuring the persistent kernel"));

  // per-system workspaces, schedules and occupations
  int nmax = 0;
  for (int k = 0; k < nsys; ++k) {
    fock_plan* p = b->plans[k];
    const int npairs = nb[k] * (nb[k] + 1) / 2;
    fock_status st = ensure_workspace(p, nb[k], npairs);
    if (st != FOCK_OK) return fail_create(bfail(b, st, p->err));
    build_schedule(p, nb[k]);
    chains_from_pairs(p->pairs, p->chains);
    if ((e = cudaMemcpyAsync(p->ws.pairs, p->pairs.data(), sizeof(int2) * npairs, cudaMemcpyHostToDevice,
                             b->cap_stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(p->ws.chains, p->chains.data(), sizeof(Chain) * p->chains.size(),
                             cudaMemcpyHostToDevice, b->cap_stream)) != cudaSuccess)
      return fail_create(bcuda(b, e, "uploading a schedule"));
    p->sched_nb = nb[k];
    st = upload_occ(p, occ[k], nb[k], b->cap_stream);
    if (st != FOCK_OK) return fail_create(bfail(b, st, p->err));
    if ((e = cudaStreamSynchronize(b->cap_stream)) != cudaSuccess) return fail_create(bcuda(b, e, "sync"));
    nmax = std::max(nmax, p->n);
  }

  // runs of chains, one transform-buffer slot each, and the segment list
  const size_t csz = 2 * (size_t)b->plans[0]->ops->real_bytes;
  const size_t hmax = (size_t)nmax * nmax * 2 * (nmax / 2 + 1);
  b->slot_bytes = (size_t)o.slot_chains * hmax * csz;
  struct Run {
    int sys, chain0, nch;
  };
  std::vector<Run> runs;
  for (int k = 0; k < nsys; ++k) {
    fock_plan* p = b->plans[k];
    const int nch = (int)p->chains.size();
    const int per = (int)std::max<size_t>(1, b->slot_bytes / ((size_t)p->dp.hsize * csz));
    for (int c0 = 0; c0 < nch; c0 += per) runs.push_back(Run{k, c0, std::min(per, nch - c0)});
  }
  const int R = (int)runs.size(), D = o.ring;
  std::vector<int> ifwd(R, -1), icol(R, -1), iinv(R, -1);
  auto emit = [&](int kind, int t, int dep, int dep2) {
    fockx::Segment sg{};
    sg.kind = kind;
    sg.sys = runs[t].sys;
    sg.chain0 = runs[t].chain0;
    sg.nch = runs[t].nch;
    sg.slot = t % D;
    sg.dep = dep;
    sg.dep2 = dep2;
    sg.ntasks = (sg.kind == 1 ? b->plans[sg.sys]->dp.ncta_col : b->plans[sg.sys]->n) * sg.nch;
    b->segs.push_back(sg);
    return (int)b->segs.size() - 1;
  };
  for (int t = 0; t < R + 2; ++t) {
    if (t < R) ifwd[t] = emit(0, t, -1, t >= D ? iinv[t - D] : -1);
    if (t - 1 >= 0 && t - 1 < R) icol[t - 1] = emit(1, t - 1, ifwd[t - 1], -1);
    if (t - 2 >= 0 && t - 2 < R) iinv[t - 2] = emit(2, t - 2, icol[t - 2], -1);
  }
  int acc = 0;
  for (auto& sg : b->segs) {
    sg.task0 = acc;
    acc += sg.ntasks;
  }
  b->ntasks = acc;
  const int nseg = (int)b->segs.size();
  if (o.stall_segment >= 0 && o.stall_segment < nseg) b->segs[o.stall_segment].dep = o.stall_segment;

  std::vector<fockx::SysDesc> sd(nsys);
  for (int k = 0; k < nsys; ++k) {
    fock_plan* p = b->plans[k];
    sd[k].g = p->dp;
    if (!o.want_dex) sd[k].g.dvtab64 = nullptr;
    if (p->ops->prec == 1) {
      // the FP64 overlaps of the system's pairs (G = 0 terms), filled by each run
      const int64_t need = (int64_t)nb[k] * nb[k];
      if (need > p->ovl_cap) {
        cudaFree(p->d_ovl);
        p->d_ovl = nullptr;
        p->ovl_cap = 0;
        if ((e = cudaMalloc((void**)&p->d_ovl, sizeof(double) * (size_t)need)) != cudaSuccess)
          return fail_create(bcuda(b, e, "allocating the overlaps"));
        p->ovl_cap = need;
      }
      sd[k].g.ovl = p->d_ovl;
      sd[k].g.ovl_ld = nb[k];
      sd[k].g.ovl_j0 = 0;
      sd[k].g.ovl_scale = (double)p->dp.ntot / p->vol;
    }
    sd[k].psi = p->ws.psi;
    sd[k].W = p->ws.w;
    sd[k].occT = p->ws.occT;
    sd[k].chains = p->ws.chains;
    sd[k].epair = p->ws.epair;
    sd[k].dpair = p->ws.dpair;
  }
  if ((e = cudaMalloc((void**)&b->d_sys, sizeof(fockx::SysDesc) * nsys)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_seg, sizeof(fockx::Segment) * nseg)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_counters, sizeof(unsigned) * (2 + nseg))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_ring, b->slot_bytes * D)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_result, sizeof(double) * 2 * nsys)) != cudaSuccess ||
      (e = cudaMallocHost((void**)&b->h_result, sizeof(double) * 2 * nsys)) != cudaSuccess ||
      (e = cudaMallocHost((void**)&b->h_err, sizeof(unsigned))) != cudaSuccess)
    return fail_create(bcuda(b, e, "allocating the batch"));
  if ((e = cudaMemcpy(b->d_sys, sd.data(), sizeof(fockx::SysDesc) * nsys, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_seg, b->segs.data(), sizeof(fockx::Segment) * nseg, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail_create(bcuda(b, e, "uploading the batch"));

  int per_sm = 0, nsm = 0;
  if ((e = b->pops->occupancy(&per_sm)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return fail_create(bcuda(b, e, "occupancy query"));
  if (per_sm < 1) return fail_create(bfail(b, FOCK_ERR_UNSUPPORTED_SIZE, "the persistent kernel does not fit an SM"));
  if (o.ctas_per_sm > 0) per_sm = std::min(per_sm, o.ctas_per_sm);
  // every CTA of the grid must be resident at once: the waits rely on it
  b->grid = std::min(b->ntasks, per_sm * nsm);
  if (o.persistent == 2) b->grid = b->ntasks;  // the dataflow launch: one CTA per task

  if (o.use_graph) {
    if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return fail_create(bcuda(b, e, "cudaStreamBeginCapture"));
    fock_status st = batch_enqueue(b, b->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (st != FOCK_OK) {
      if (g) cudaGraphDestroy(g);
      return fail_create(st);
    }
    if (e != cudaSuccess) return fail_create(bcuda(b, e, "cudaStreamEndCapture"));
    b->graph = g;
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
      return fail_create(bcuda(b, e, "cudaGraphInstantiate"));
  }
  *out = b;
  return FOCK_OK;
}

fock_status fock_batch_run(fock_batch_t b, double* ex, double* dex, fock_stream_t stream) {
  if (!b) return bfail(nullptr, FOCK_ERR_INVALID_ARG, "batch is NULL");
  int dev = -1;
  FOCK_BCUDA(b, cudaGetDevice(&dev));
  if (dev != b->device) return bfail(b, FOCK_ERR_INVALID_ARG, "the batch belongs to another device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (b->exec) {
    FOCK_BCUDA(b, cudaGraphLaunch(b->exec, s));
  } else {
    fock_status st = batch_enqueue(b, s);
    if (st != FOCK_OK) return st;
  }
  FOCK_BCUDA(b, cudaStreamSynchronize(s));
  if (*b->h_err != 0u) {
    return bfail(b, FOCK_ERR_TIMEOUT,
                 "a dependency wait of segment " + std::to_string(*b->h_err - 1) + " gave up");
  }
  for (int k = 0; k < b->nsys; ++k) {
    if (ex) ex[k] = b->h_result[2 * k];
    if (dex) dex[k] = b->h_result[2 * k + 1];
  }
  return FOCK_OK;
}

fock_status fock_batch_info(fock_batch_t b, int64_t* launches, int64_t* tasks, int* grid, int* segments,
                            double* persist_ms) {
  if (!b) return bfail(nullptr, FOCK_ERR_INVALID_ARG, "batch is NULL");
  if (persist_ms) {
    float ms = 0.f;
    *persist_ms = cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess ? (double)ms : -1.0;
    cudaGetLastError();
  }
  if (launches) *launches = b->launches;
  if (tasks) *tasks = b->ntasks;
  if (grid) *grid = b->grid;
  if (segments) *segments = (int)b->segs.size();
  return FOCK_OK;
}

const char* fock_batch_last_error(fock_batch_t b) { return b ? b->err.c_str() : g_create_error.c_str(); }

fock_status fock_batch_destroy(fock_batch_t b) {
  if (!b) return FOCK_OK;
  batch_free(b);
  delete b;
  return FOCK_OK;
}

}  // extern "C"
