// fock_persist.cuh — the pair passes of many systems in one persistent launch.
//
// The work of a batch of systems (uneven grids and band counts) is cut into
// segments: a segment is one pass kind (forward plane pass, column pass,
// inverse plane pass) over a run of consecutive chains of one system, i.e.
// N * nch (planes) or ncta_col * nch (column-map CTAs) tasks of one CTA each.  A resident
// grid of CTAs takes tasks in ticket order from a global counter.  Segments are
// listed in an order in which every dependency points backwards:
//
//   iteration t:  fwd(t), col(t-1), inv(t-2)       (t over all chain runs of all systems)
//
// col(t) needs fwd(t) complete, inv(t) needs col(t) complete, and fwd(t)
// reuses the transform-buffer slot of run t - D (a ring of D >= 3 slots), so it
// needs inv(t - D) complete.  A CTA waits only for tasks with smaller tickets,
// which resident CTAs hold, so the lowest unfinished ticket can always run: no
// deadlock.  Every wait is still bounded (wall-clock limit and spin count);
// when one gives up, the kernel records the segment in an error word, every
// CTA stops at its next ticket or wait, and the host reports FOCK_ERR_TIMEOUT.
//
// Producers publish a finished task with __threadfence + atomicAdd on the
// segment's counter; consumers acquire the counter and read the transform
// buffer through L2 (__ldcg in the task functions), so no stale L1 line is
// ever used.
#pragma once

#include "fock_kernels.cuh"

namespace fockx {

// CTA size: enough for the 96^3 column pass (4 threads per line in FP32, 8 in FP64)
template <class T> constexpr int kPersistMaxT = sizeof(T) == 8 ? 800 : 416;

template <class T>
struct PersistGeo {
  // largest dynamic shared memory over the grid sizes the persistent kernel runs
  static constexpr size_t smem_of(size_t a, size_t b) { return a > b ? a : b; }
  static constexpr size_t SMEM = smem_of(
      smem_of(smem_of(Geo<T, 96, kPersistMaxT<T>>::SMEM_PLANE, Geo<T, 96, kPersistMaxT<T>>::SMEM_COLH),
              smem_of(Geo<T, 72, kPersistMaxT<T>>::SMEM_PLANE, Geo<T, 72, kPersistMaxT<T>>::SMEM_COLH)),
      smem_of(Geo<T, 96, kPersistMaxT<T>>::SMEM_INV, Geo<T, 72, kPersistMaxT<T>>::SMEM_INV));
  static constexpr int MIN_CTAS = sizeof(T) == 4 ? 2 : 1;  // shared memory allows 2 in FP32
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait until *p >= target; false when the error word is set or the limit passes.
__device__ inline bool bounded_wait(const unsigned* p, unsigned target, const unsigned* err,
                                    unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (unsigned spin = 0; spin < (1u << 28); ++spin) {
    if (ld_acquire(p) >= target) return true;
    if (ld_acquire(err) != 0u) return false;
    if (global_ns() - t0 > limit_ns) return false;
    __nanosleep(256);
  }
  return false;
}

// One task body per (pass kind, N), each compiled as its own function so that
// it gets the register allocation of a stand-alone kernel.
template <class T, int N, int KIND>
__device__ __noinline__ void persist_task(const SysDesc* __restrict__ sys, int sysi, int chain, int idx,
                                          cplx<T>* Hc) {
  // the dynamic shared array by name (not through a pointer argument), so its
  // accesses stay shared-memory accesses with 32-bit addresses
  extern __shared__ __align__(16) unsigned char smem[];
  const SysDesc& sd = sys[sysi];
  const Chain ch = sd.chains[chain];
  if constexpr (KIND == 0) {
    pair_fwd_task<T, N, kPersistMaxT<T>>(sd.g, static_cast<const T*>(sd.psi), ch, Hc, idx, smem);
  } else if constexpr (KIND == 1) {
    pair_col_task<T, N, kPersistMaxT<T>>(sd.g, Hc, ch, idx, sd.epair, sd.dpair, smem);
  } else {
    pair_inv_task<T, N, kPersistMaxT<T>>(sd.g, static_cast<const T*>(sd.psi), static_cast<T*>(sd.W),
                                      static_cast<const T*>(sd.occT), ch, Hc, idx, smem);
  }
}

template <class T, int N>
__device__ __forceinline__ void run_task(const SysDesc* sys, const Segment& sg, int local, cplx<T>* hslot,
                                         int64_t hsize) {
  // tasks per chain: N planes, or the column-map CTAs of the column pass
  const int per = sg.kind == 1 ? sys[sg.sys].g.ncta_col : N;
  const int c = local / per, idx = local - c * per;
  cplx<T>* Hc = hslot + (int64_t)c * hsize;
  if (sg.kind == 0) persist_task<T, N, 0>(sys, sg.sys, sg.chain0 + c, idx, Hc);
  else if (sg.kind == 1) persist_task<T, N, 1>(sys, sg.sys, sg.chain0 + c, idx, Hc);
  else persist_task<T, N, 2>(sys, sg.sys, sg.chain0 + c, idx, Hc);
}

// counters[0]: next ticket; counters[1]: error word (segment + 1 of the wait that
// gave up); counters[2 + s]: finished tasks of segment s.
template <class T>
__global__ void __launch_bounds__(kPersistMaxT<T>, PersistGeo<T>::MIN_CTAS)
    k_pair_persistent(const SysDesc* __restrict__ sys, const Segment* __restrict__ seg, int nseg,
                      int ntasks, unsigned* counters, unsigned char* hring, size_t slot_bytes,
                      unsigned long long limit_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ticket;
  __shared__ int s_ok;
  unsigned* err = counters + 1;
  unsigned* done = counters + 2;
  int cur = 0;  // tickets of one CTA only increase, so the segment search moves forward
  for (;;) {
    __syncthreads();  // the previous task is done with shared memory
    if (threadIdx.x == 0) {
      s_ticket = ld_acquire(err) != 0u ? ntasks : (int)atomicAdd(counters, 1u);
    }
    __syncthreads();
    const int t = s_ticket;
    if (t >= ntasks) break;
    while (t >= seg[cur].task0 + seg[cur].ntasks) ++cur;
    const Segment sg = seg[cur];
    if (threadIdx.x == 0) {
      bool ok = true;
      if (sg.dep >= 0) ok = bounded_wait(done + sg.dep, (unsigned)seg[sg.dep].ntasks, err, limit_ns);
      if (ok && sg.dep2 >= 0)
        ok = bounded_wait(done + sg.dep2, (unsigned)seg[sg.dep2].ntasks, err, limit_ns);
      if (!ok) atomicCAS(err, 0u, (unsigned)cur + 1u);
      s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) break;
    cplx<T>* hslot = reinterpret_cast<cplx<T>*>(hring + (size_t)sg.slot * slot_bytes);
    const int local = t - sg.task0;
    const int n = sys[sg.sys].g.n;
    const int64_t hsize = sys[sg.sys].g.hsize;
    switch (n) {
      case 24: run_task<T, 24>(sys, sg, local, hslot, hsize); break;
      case 32: run_task<T, 32>(sys, sg, local, hslot, hsize); break;
      case 48: run_task<T, 48>(sys, sg, local, hslot, hsize); break;
      case 64: run_task<T, 64>(sys, sg, local, hslot, hsize); break;
      case 72: run_task<T, 72>(sys, sg, local, hslot, hsize); break;
      case 96: run_task<T, 96>(sys, sg, local, hslot, hsize); break;
      default: break;  // the host admits only the sizes above
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + cur, 1u);
    }
  }
}

// ---------------------------------------------------------------- dataflow launch
//
// The same segments and dependencies as the persistent kernel, but one CTA per
// task and no loop: the grid has one CTA per ticket.  A CTA takes its ticket
// from the global counter when it starts (so tickets follow the order in which
// CTAs become resident, whatever the hardware's dispatch order), waits for the
// segments its task depends on (all of smaller tickets, held by CTAs that have
// already started: the lowest unfinished ticket can always run), runs the task
// body inlined (the register allocation of a stand-alone kernel, no call
// boundary) and publishes it.  Waits are bounded as in the persistent kernel.

// The task body, inlined, for grid size N.
template <class T, int N>
__device__ __forceinline__ void dataflow_task(const SysDesc* __restrict__ sys, const Segment& sg, int local,
                                              cplx<T>* hslot, unsigned char* smem) {
  const SysDesc& sd = sys[sg.sys];
  const int per = sg.kind == 1 ? sd.g.ncta_col : N;
  const int c = local / per, idx = local - c * per;
  cplx<T>* Hc = hslot + (int64_t)c * sd.g.hsize;
  const Chain ch = sd.chains[sg.chain0 + c];
  if (sg.kind == 0) {
    pair_fwd_task<T, N, kPersistMaxT<T>>(sd.g, static_cast<const T*>(sd.psi), ch, Hc, idx, smem);
  } else if (sg.kind == 1) {
    pair_col_task<T, N, kPersistMaxT<T>>(sd.g, Hc, ch, idx, sd.epair, sd.dpair, smem);
  } else {
    pair_inv_task<T, N, kPersistMaxT<T>>(sd.g, static_cast<const T*>(sd.psi), static_cast<T*>(sd.W),
                                         static_cast<const T*>(sd.occT), ch, Hc, idx, smem);
  }
}

template <class T>
__global__ void __launch_bounds__(kPersistMaxT<T>, PersistGeo<T>::MIN_CTAS)
    k_pair_dataflow(const SysDesc* __restrict__ sys, const Segment* __restrict__ seg, int nseg, int ntasks,
                    unsigned* counters, unsigned char* hring, size_t slot_bytes, unsigned long long limit_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ticket, s_seg;
  unsigned* err = counters + 1;
  unsigned* done = counters + 2;
  if (threadIdx.x == 0) {
    int t = ntasks, cur = -1;
    if (ld_acquire(err) == 0u) {
      t = (int)atomicAdd(counters, 1u);
      if (t < ntasks) {  // the segment of ticket t: the last with task0 <= t
        int lo = 0, hi = nseg - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) / 2;
          if (seg[mid].task0 <= t) lo = mid;
          else hi = mid - 1;
        }
        cur = lo;
        const Segment& sg = seg[cur];
        bool ok = true;
        if (sg.dep >= 0) ok = bounded_wait(done + sg.dep, (unsigned)seg[sg.dep].ntasks, err, limit_ns);
        if (ok && sg.dep2 >= 0) ok = bounded_wait(done + sg.dep2, (unsigned)seg[sg.dep2].ntasks, err, limit_ns);
        if (!ok) {
          atomicCAS(err, 0u, (unsigned)cur + 1u);
          t = ntasks;
        }
      }
    }
    s_ticket = t;
    s_seg = cur;
  }
  __syncthreads();
  const int t = s_ticket;
  if (t >= ntasks) return;
  const Segment sg = seg[s_seg];
  cplx<T>* hslot = reinterpret_cast<cplx<T>*>(hring + (size_t)sg.slot * slot_bytes);
  const int local = t - sg.task0;
  switch (sys[sg.sys].g.n) {
    case 24: dataflow_task<T, 24>(sys, sg, local, hslot, smem_raw); break;
    case 32: dataflow_task<T, 32>(sys, sg, local, hslot, smem_raw); break;
    case 48: dataflow_task<T, 48>(sys, sg, local, hslot, smem_raw); break;
    case 64: dataflow_task<T, 64>(sys, sg, local, hslot, smem_raw); break;
    case 72: dataflow_task<T, 72>(sys, sg, local, hslot, smem_raw); break;
    case 96: dataflow_task<T, 96>(sys, sg, local, hslot, smem_raw); break;
    default: break;  // the host admits only the sizes above
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(done + s_seg, 1u);
  }
}

template <class T>
struct PersistLaunch {
  static cudaError_t configure() {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_pair_persistent<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PersistGeo<T>::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void*)k_pair_dataflow<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PersistGeo<T>::SMEM);
  }
  static cudaError_t occupancy(int* ctas_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_pair_persistent<T>, kPersistMaxT<T>,
                                                         PersistGeo<T>::SMEM);
  }
  static cudaError_t launch(int grid, const SysDesc* sys, const Segment* seg, int nseg, int ntasks,
                            unsigned* counters, unsigned char* hring, size_t slot_bytes,
                            unsigned long long limit_ns, cudaStream_t s) {
    k_pair_persistent<T><<<grid, kPersistMaxT<T>, PersistGeo<T>::SMEM, s>>>(sys, seg, nseg, ntasks, counters,
                                                                      hring, slot_bytes, limit_ns);
    return cudaGetLastError();
  }
  static cudaError_t launch_dataflow(const SysDesc* sys, const Segment* seg, int nseg, int ntasks,
                                     unsigned* counters, unsigned char* hring, size_t slot_bytes,
                                     unsigned long long limit_ns, cudaStream_t s) {
    k_pair_dataflow<T><<<ntasks, kPersistMaxT<T>, PersistGeo<T>::SMEM, s>>>(sys, seg, nseg, ntasks, counters,
                                                                          hring, slot_bytes, limit_ns);
    return cudaGetLastError();
  }
  static constexpr PersistOps ops() {
    return PersistOps{(int)sizeof(T), PersistGeo<T>::SMEM, configure, occupancy, launch, launch_dataflow};
  }
};

}  // namespace fockx
