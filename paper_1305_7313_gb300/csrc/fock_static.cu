// fock_static.cu — fock_pair_energies_static: the pair energies of
// fock_pair_energies for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the pair
// energies: code under a framework that owns every device allocation (a
// caching allocator, a fixed memory budget that the library may not grow),
// or a loop that cannot take an allocation's latency or the device-wide
// synchronisation cudaMalloc and cudaFree may imply.  This entry point takes
// the working memory the pair passes need (real-space orbitals, the
// half-spectrum transform buffer, the chain list and the per-pair partial
// sums) from one file-scope device array of kStaticScratchBytes instead of the
// plan's workspace.  It calls no cudaMalloc, cudaFree or other allocating
// routine.
//
// It is still a synchronising call: it copies the caller's host pair list to
// the device, waits for its stream, and scales the energies on the host.  It
// must not be issued on a stream that is being captured into a CUDA graph.
//
// The array exists once per device for the lifetime of the process that
// loaded the library.  Host code must not use its name as a device address:
// at set-up, the first call in each CUDA context of a device (with that device
// current) asks the runtime for the array's device address
// (cudaGetSymbolAddress) and keeps it for that context; a new context on the
// device (after cudaDeviceReset, say) is looked up again.
//
// Every call uses the same array and leaves its contents behind; the call
// clears what must start at zero.  Two calls whose work overlaps on the GPU
// (different streams, or host threads without ordering) race on the array.
#include <algorithm>
#include <mutex>
#include <vector>

#include <cuda.h>  // driver types for the context query; the entry points come through the runtime

#include "fock.h"
#include "fock_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_address[kMaxDevices];         // device address of g_static_scratch, per device
unsigned long long g_scratch_ctx[kMaxDevices];  // id of the context that address belongs to (0: none)

__global__ void k_chains_from_pairs(const int2* __restrict__ pairs, int npairs,
                                    fockx::Chain* __restrict__ chains) {
  const int nch = (npairs + 1) / 2;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nch; k += gridDim.x * blockDim.x) {
    fockx::Chain c;
    const int2 a = pairs[2 * k];
    c.ai = a.x;
    c.aj = a.y;
    c.pa = 2 * k;
    if (2 * k + 1 < npairs) {
      const int2 b = pairs[2 * k + 1];
      c.bi = b.x;
      c.bj = b.y;
      c.pb = 2 * k + 1;
    } else {
      c.bi = c.bj = -1;
      c.pb = -1;
    }
    c.flags = c.pad1 = 0;
    chains[k] = c;
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

fock_status fail(fock_plan_t plan, fock_status s, const char* msg) {
  fockx::plan_set_error(plan, msg);
  return s;
}

fock_status cuda_fail(fock_plan_t plan, cudaError_t e) {
  cudaGetLastError();
  fockx::plan_set_error(plan, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FOCK_ERR_OOM : FOCK_ERR_CUDA;
}

// Id of the current CUDA context (unique for the life of the process), or 0
// when the driver cannot tell; the driver entry points are fetched through
// the runtime, so the library does not link the driver library itself.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    resolved = true;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on `device` (which must be current),
// looked up once per context of the device.  When the context cannot be
// identified the address is looked up on every call.
cudaError_t scratch_address(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  const unsigned long long ctx = current_context_id();
  if (ctx == 0 || g_scratch_ctx[device] != ctx || g_scratch_address[device] == nullptr) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_address[device] = ptr;
    g_scratch_ctx[device] = ctx;
  }
  *out = static_cast<unsigned char*>(g_scratch_address[device]);
  return cudaSuccess;
}

}  // namespace

extern "C" fock_status fock_pair_energies_static(fock_plan_t plan, const void* psi_G, int nb,
                                                 const int32_t* pairs, int npairs, double* e,
                                                 double* d, fock_stream_t stream) {
  fockx::PlanView v;
  if (!fockx::plan_view(plan, &v)) return FOCK_ERR_INVALID_ARG;
  if (!psi_G || !e || !pairs) return fail(plan, FOCK_ERR_INVALID_ARG, "NULL argument");
  if (nb < 1 || npairs < 1) return fail(plan, FOCK_ERR_INVALID_ARG, "nb and npairs must be >= 1");
  for (int k = 0; k < 2 * npairs; ++k)
    if (pairs[k] < 0 || pairs[k] >= nb) return fail(plan, FOCK_ERR_INVALID_ARG, "a band index is out of range");
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return cuda_fail(plan, err);
  if (dev != v.device) return fail(plan, FOCK_ERR_INVALID_ARG, "the plan belongs to another device");
  if (dev < 0 || dev >= kMaxDevices) return fail(plan, FOCK_ERR_INVALID_ARG, "device ordinal too large");

  // layout of the scratch array
  const size_t rb = (size_t)v.ops->real_bytes;
  const size_t chain_bytes = (size_t)v.dp.hsize * 2 * rb;
  const int nch = (npairs + 1) / 2;
  const size_t off_psi = 0;
  const size_t off_pairs = align256(off_psi + (size_t)nb * (size_t)v.dp.ntot * rb);
  const size_t off_chains = align256(off_pairs + sizeof(int2) * (size_t)npairs);
  const size_t off_e = align256(off_chains + sizeof(fockx::Chain) * (size_t)nch);
  const size_t off_d = align256(off_e + sizeof(double) * (size_t)npairs);
  const size_t off_h = align256(off_d + sizeof(double) * (size_t)npairs);
  if (off_h + chain_bytes > kStaticScratchBytes) {
    return fail(plan, FOCK_ERR_INVALID_ARG,
                "the request needs more than the 32 MiB static scratch "
                "(real-space orbitals nb*N^3 reals + one N^2(N+2) complex transform buffer)");
  }
  const int cb = (int)std::min<size_t>((size_t)nch, (kStaticScratchBytes - off_h) / chain_bytes);

  unsigned char* base = nullptr;
  err = scratch_address(dev, &base);
  if (err != cudaSuccess) return cuda_fail(plan, err);
  void* psi = base + off_psi;
  int2* dpairs = reinterpret_cast<int2*>(base + off_pairs);
  fockx::Chain* chains = reinterpret_cast<fockx::Chain*>(base + off_chains);
  double* ep = reinterpret_cast<double*>(base + off_e);
  double* dp = reinterpret_cast<double*>(base + off_d);
  void* hbuf = base + off_h;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fockx::DevPlan g = v.dp;
  if (!d) g.dvtab64 = nullptr;
  if ((err = cudaMemcpyAsync(dpairs, pairs, sizeof(int2) * (size_t)npairs, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(plan, err);
  k_chains_from_pairs<<<(nch + 255) / 256, 256, 0, s>>>(dpairs, npairs, chains);
  if ((err = cudaGetLastError()) != cudaSuccess) return cuda_fail(plan, err);
  if ((err = cudaMemsetAsync(ep, 0, sizeof(double) * (size_t)npairs, s)) != cudaSuccess) return cuda_fail(plan, err);
  if ((err = cudaMemsetAsync(dp, 0, sizeof(double) * (size_t)npairs, s)) != cudaSuccess) return cuda_fail(plan, err);
  // orbitals to real space one band pair at a time (one grid of the transform buffer)
  for (int b0 = 0; b0 < nb; b0 += 2) {
    err = v.ops->to_real(g, static_cast<const double2*>(psi_G), nb, b0, std::min(2, nb - b0), hbuf, psi, s);
    if (err != cudaSuccess) return cuda_fail(plan, err);
  }
  for (int c = 0; c < nch; c += cb) {
    const int cnt = std::min(cb, nch - c);
    if ((err = v.ops->pair_fwd(g, psi, chains + c, cnt, hbuf, s)) != cudaSuccess) return cuda_fail(plan, err);
    if ((err = v.ops->pair_col(g, hbuf, chains + c, cnt, ep, dp, s)) != cudaSuccess) return cuda_fail(plan, err);
  }
  if ((err = cudaMemcpyAsync(e, ep, sizeof(double) * (size_t)npairs, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(plan, err);
  if (d && (err = cudaMemcpyAsync(d, dp, sizeof(double) * (size_t)npairs, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(plan, err);
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(plan, err);
  const double inv2 = 1.0 / ((double)v.dp.ntot * (double)v.dp.ntot);
  for (int k = 0; k < npairs; ++k) {
    e[k] *= inv2;
    if (d) d[k] = g.dvtab64 ? d[k] * inv2 : 0.0;
  }
  return FOCK_OK;
}
