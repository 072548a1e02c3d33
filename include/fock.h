/*
 * fock.h — C ABI of the GB300 Fock exact-exchange library (libfockx.so).
 *
 * The library applies the Fock exact-exchange operator of hybrid-functional
 * plane-wave DFT to a set of Gamma-point orbitals and returns the exchange
 * energy (arXiv:1305.7313, §4 "The Exact Exchange (EXX) within the planewave
 * method": the reciprocal-space E_x equation, the V_x|u_i> equation and the
 * paragraph on overlap charge densities computed by FFT):
 *
 *   psi_i(r)        = Omega^-1/2 sum_{G in S} c_i(G) exp(i G.r)
 *   phi_ij(r)       = IFFT[ v(G) FFT(psi_i* psi_j) ](r)
 *   (V_x psi_j)(r)  = - sum_i f_i psi_i(r) phi_ij(r)
 *   (V_x psi_j)(G)  = (sqrt(Omega)/Ntot) FFT(V_x psi_j)(G),   G in S
 *   E_x             = -(Omega/2) sum_{i,j} f_i f_j sum_G v(G) |FFT(psi_i* psi_j)(G)/Ntot|^2
 *                   = 1/2 sum_j f_j <psi_j | V_x psi_j>
 *
 * Units are Hartree atomic units (bohr, Ha).  FFT is the unnormalised forward
 * transform with exp(-i G.r); IFFT carries 1/Ntot; Ntot = N1 N2 N3.
 *
 * Conventions shared by every entry point
 *  - Every call returns a fock_status; nothing is thrown and nothing exits.
 *    fock_last_error(plan) gives a one-line description of the last failure.
 *  - Errors every entry point shares (each entry lists the others it has): a
 *    NULL handle or output pointer, or an argument outside its stated range,
 *    gives FOCK_ERR_INVALID_ARG (the *_destroy calls accept NULL and return
 *    FOCK_OK); a call that queues GPU work can also give FOCK_ERR_CUDA (a
 *    CUDA call failed; the last-error text names it) and, where it grows its
 *    workspace, FOCK_ERR_OOM.
 *  - "device" pointers are CUDA global-memory pointers of the current device;
 *    "host" pointers are ordinary CPU memory.  The caller owns every buffer it
 *    passes; the library never frees or keeps them past the call.
 *  - The plan owns its tables and a workspace that grows on demand (or via
 *    fock_plan_reserve).  One plan must not be used by two calls at the same
 *    time (host threads or overlapping streams): they share the workspace.
 *  - Work is ordered on the given stream (a cudaStream_t passed as void*;
 *    NULL = the legacy default stream).  A call returns after queueing its
 *    kernels unless it must hand a value back in host memory (ex, dex or the
 *    pair energies), in which case it synchronises that stream first.
 *  - Inputs are never modified.
 */
#ifndef FOCK_H
#define FOCK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fock_plan* fock_plan_t;
typedef void* fock_stream_t; /* a cudaStream_t */

typedef enum {
  FOCK_OK = 0,
  FOCK_ERR_INVALID_ARG = 1,      /* a NULL pointer, a non-positive size, a bad enum, ... */
  FOCK_ERR_UNSUPPORTED_SIZE = 2, /* grid not cubic, N not 2^a 3^b, or too large for the kernels */
  FOCK_ERR_GRID_TOO_SMALL = 3,   /* the G-sphere does not fit on the FFT grid (2|m_a| >= N_a) */
  FOCK_ERR_OOM = 4,              /* device allocation failed */
  FOCK_ERR_CUDA = 5,             /* a CUDA runtime call or a kernel launch failed */
  FOCK_ERR_TIMEOUT = 6           /* a bounded device-side wait gave up */
} fock_status;

typedef enum {
  /* Spencer-Alavi spherical truncation: v(G) = 4 pi (1 - cos(|G| Rc)) / |G|^2,
   * v(0) = 2 pi Rc^2, Rc = (3 Omega / 4 pi)^(1/3).  No parameters. */
  FOCK_KERNEL_SPENCER_ALAVI = 0,
  /* erfc screening: v(G) = 4 pi (1 - exp(-|G|^2 / 4 w^2)) / |G|^2, v(0) = pi / w^2.
   * kparams = {w} (bohr^-1, > 0). */
  FOCK_KERNEL_ERFC = 1
} fock_kernel;

typedef enum {
  /* Everything in FP64: transforms, products, accumulators, energies. */
  FOCK_PREC_FP64 = 0,
  /* complex64 transforms and FP32 pair products / V_x psi accumulation; the
   * kernel terms of the smallest |G| (|m|^2 <= 3) and every energy sum in FP64.
   * The G = 0 value of each pair density is taken from the FP64 overlap
   * Re sum_G c_i(G)* c_j(G) of the input coefficients (times N^3 / Omega),
   * computed on the device for every apply (fock_apply, fock_apply_shard,
   * fock_apply_fixed, batches; an nb x nb FP64 buffer in the plan). */
  FOCK_PREC_MIXED32 = 1,
  /* Double-float: every real of the pair passes and the O(nb) transforms is
   * the unevaluated sum of two floats (about 48 significant bits, float's
   * exponent range), computed with error-free float transformations on the
   * FP32 pipe; V_x psi accumulators, energies and the I/O stay FP64.  Same
   * inputs, outputs and tolerance (1e-10 relative) as FOCK_PREC_FP64.  Gamma
   * point only: batches and k-point plans refuse it (INVALID_ARG). */
  FOCK_PREC_DF64 = 2
} fock_precision;

/* Orbitals are Gamma-point real functions: c(-G) = c(G)*.  Required. */
#define FOCK_GAMMA_REAL 1u

/*
 * fock_plan_create — build the plane-wave sphere, the Coulomb-kernel table and
 * the FFT plan for one cell.
 *   out      host; receives the new plan (set to NULL on failure).
 *   grid     host int[3]; FFT grid N1, N2, N3.  Must be cubic (N1 = N2 = N3)
 *            with N one of the compiled sizes 8, 12, 16, 24, 32, 36, 48, 64,
 *            72, 96 (other N: UNSUPPORTED_SIZE).
 *   cell     host double[9]; rows a1, a2, a3 of the cell in bohr (any
 *            non-degenerate lattice).
 *   ecut_ha  plane-wave cutoff in Ha: S = {G : |G|^2 / 2 <= ecut_ha}.
 *   kind, kparams, nkparams   Coulomb kernel and its parameters (see fock_kernel).
 *   prec     arithmetic of the apply (see fock_precision).
 *   flags    must contain FOCK_GAMMA_REAL.
 * The sphere's canonical order: ascending FP64 |G|^2, ties broken
 * lexicographically on the Miller indices (m1, m2, m3); |G|^2 is evaluated as
 * G_x = (m1 b1x + m2 b2x) + m3 b3x (same for y, z), |G|^2 = (Gx^2 + Gy^2) + Gz^2,
 * with b_i = (2 pi / Omega) (a_j x a_k), Omega = a1 . (a2 x a3), no fused
 * multiply-add anywhere.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, GRID_TOO_SMALL, OOM, CUDA.
 */
fock_status fock_plan_create(fock_plan_t* out, const int grid[3], const double cell[9],
                             double ecut_ha, fock_kernel kind, const double* kparams,
                             int nkparams, fock_precision prec, unsigned flags);

/*
 * fock_gsphere — the plane-wave sphere of a cell without creating a plan (host
 * only, no GPU needed): the same list, in the same canonical order, that
 * fock_plan_create builds.
 *   grid, cell, ecut_ha   as in fock_plan_create (the grid is used only for the
 *                         GRID_TOO_SMALL check).
 *   npw      host int64; receives the number of plane waves.
 *   miller   host int32 [capacity][3] or NULL; receives the Miller indices
 *            when capacity >= npw (call once with NULL to size the buffer).
 * Errors: INVALID_ARG, GRID_TOO_SMALL, and INVALID_ARG when miller is not NULL
 * but capacity < npw.
 */
fock_status fock_gsphere(const int grid[3], const double cell[9], double ecut_ha, int64_t* npw,
                         int32_t* miller, int64_t capacity);

/*
 * fock_schedule — the unique pairs (i <= j) that fock_apply_shard(..., shard,
 * nshards, ...) evaluates for nb bands with a plan whose band block is
 * band_block (0: the default of 16), in the library's fixed schedule (host
 * only, no GPU).  The schedule visits blocks of band_block x band_block pairs
 * (block rows outer) so that consecutive pairs share orbitals.  This is the band-group split of §5 (Fig. 3) as the library
 * draws it: the shards are disjoint and together hold every unique pair once.
 *   pairs    host int32 [capacity][2] or NULL (call with NULL to size it).
 *   npairs   host int64; receives the number of pairs of the shard.
 * Errors: INVALID_ARG.
 */
fock_status fock_schedule(int nb, int band_block, int shard, int nshards, int32_t* pairs,
                          int64_t capacity, int64_t* npairs);

/* Number of plane waves npw in the sphere.  npw: host int64. */
fock_status fock_plan_npw(fock_plan_t plan, int64_t* npw);

/* Miller indices of the sphere in canonical order.  miller: host int32[npw][3]. */
fock_status fock_plan_gvectors(fock_plan_t plan, int32_t* miller);

/* Grow the workspace now for up to nb_max bands (otherwise the first apply
 * grows it).  Errors: INVALID_ARG, OOM. */
fock_status fock_plan_reserve(fock_plan_t plan, int nb_max);

/* Number of band-pair chains (two pairs per complex transform) each launch of
 * the pair passes processes; sets the size of the plan's transform buffer
 * (chain_batch x N^2 (N+2) complex elements).  The default is the largest
 * multiple of SMs / gcd(N, SMs) chains (whole waves of the plane passes) whose
 * buffer fits 320 MiB, or as many chains as fit when one such group does not.
 * Takes effect at the next call.  Errors: INVALID_ARG. */
fock_status fock_plan_set_batch(fock_plan_t plan, int chain_batch);

/* Streams of the pair loop of fock_apply and fock_apply_shard (1 to 4, default
 * 1).  With S > 1, launch k of the pair passes runs on stream k mod S: the
 * call's stream or one of S - 1 streams the plan owns, each with its own
 * transform buffer (S times the buffer memory), so that the kernels of
 * neighbouring launches run side by side; the call's stream waits for all of
 * them before the energies are reduced, and results agree up to the order of
 * the floating-point accumulations.  Takes effect at the next call.
 * Errors: INVALID_ARG. */
fock_status fock_plan_set_streams(fock_plan_t plan, int streams);

/* Phases of a call, for fock_plan_stats. */
enum {
  FOCK_PHASE_TO_REAL = 0,   /* G-sphere scatter + inverse 3D FFT of the orbitals */
  FOCK_PHASE_PAIR_FWD = 1,  /* pair products + forward plane FFTs */
  FOCK_PHASE_PAIR_COL = 2,  /* column FFTs, kernel multiply, energy partials, inverse */
  FOCK_PHASE_PAIR_INV = 3,  /* inverse plane FFTs + V_x psi accumulation */
  FOCK_PHASE_TO_SPHERE = 4, /* forward 3D FFT of V_x psi + gather to the sphere */
  FOCK_PHASE_ENERGY = 5,    /* E_x reduction */
  FOCK_NPHASES = 6
};

typedef struct {
  int64_t launches;                   /* kernels the last call launched */
  int64_t phase_launches[FOCK_NPHASES];
  double phase_ms[FOCK_NPHASES];      /* device time per phase of the last call (timing on), else 0 */
  int64_t chains;                     /* pair chains the last call processed */
  int64_t pairs;                      /* unique pairs the last call processed */
  int chain_batch;                    /* chains per launch of the pair passes */
  int band_batch;                     /* bands per launch of the O(nb) transforms */
} fock_stats;

/* Time every launch with CUDA events on the call's stream (enable != 0).  A
 * timed call synchronises its stream before returning.  Errors: INVALID_ARG, CUDA. */
fock_status fock_plan_set_timing(fock_plan_t plan, int enable);

/* Counters and (with timing on) per-phase device times of the last call.
 * stats: host.  Errors: INVALID_ARG. */
fock_status fock_plan_stats(fock_plan_t plan, fock_stats* stats);

/* Bands per block of the pair schedule (default 16): pairs are visited in
 * band_block x band_block blocks so consecutive chains share orbitals and
 * accumulators in L2.  Takes effect at the next call.  Errors: INVALID_ARG. */
fock_status fock_plan_set_band_block(fock_plan_t plan, int band_block);

/*
 * FFT tilings of the pair passes.  Each of the three pair passes (pass 0: the
 * forward plane pass, 1: the column pass, 2: the inverse plane pass) has one
 * or two compiled radix plans ("tilings"): tile 0 holds FftTraits' element
 * budget per thread (24 complex values in the mixed form, 12 in FP64 and
 * double-float), tile 1 the plan found with the other budget (12 in the mixed
 * form, 24 in FP64; none in double-float).  When both budgets give the same
 * plan for N, the pass has one tiling.  The results do not depend on the
 * tiling beyond rounding; the speed does (the tuner in autotune.py times them).
 *
 * fock_plan_tiling_info: the plan of tile `tile` of pass `pass`: radices
 *   (host int[8], stage order), nstages, threads per transformed line,
 *   threads per CTA, and ntiles (1 or 2) for that pass.  INVALID_ARG for a
 *   tile the pass does not have.
 * fock_plan_set_tiling: tiles host int[3], the tile of each pass (each below
 *   that pass's ntiles); takes effect at the next call (fock_apply,
 *   fock_apply_shard, fock_apply_fixed, fock_pair_energies).  Default 0, 0, 0.
 *   Errors: INVALID_ARG.
 */
fock_status fock_plan_tiling_info(fock_plan_t plan, int pass, int tile, int* radices, int* nstages,
                                  int* threads_per_line, int* threads, int* ntiles);
fock_status fock_plan_set_tiling(fock_plan_t plan, const int tiles[3]);

/* Bytes of device memory the plan holds (tables + workspace).  bytes: host. */
fock_status fock_plan_device_bytes(fock_plan_t plan, int64_t* bytes);

/* Deterministic accumulation (enable != 0; FP64 and double-float plans): the
 * V_x psi accumulators are summed exactly in 64-bit fixed point (integer
 * atomics; the scale 2^s is set per call from a bound on the sums of absolute
 * values, |W_t(r)| <= ||v||_2 ||psi_t||_2 sum_s |f_s| max|psi_s|^2 / sqrt(Ntot),
 * that leaves them two bits of headroom) and the per-pair energies are summed in a
 * fixed order, so fock_apply, fock_apply_shard and fock_apply_fixed give
 * bitwise identical results run to run and for every chain batch.  The
 * rounding of each contribution to the fixed-point grid adds at most
 * nb * 2^-(s+1) per accumulator.  Default off.  Errors: INVALID_ARG (mixed
 * plans). */
fock_status fock_plan_set_deterministic(fock_plan_t plan, int enable);

/* Columns of the stored half spectrum (N x 2(N/2+1) per plane, both pairs of a
 * chain) that the pair-density ball |G| <= 2 Gmax reaches and the column pass
 * transforms (`kept`), out of `total`: the overlap densities of §4 are products
 * of two orbitals on the sphere, so their spectra live in that ball.  Host
 * outputs; either may be NULL.  Errors: INVALID_ARG (plan NULL). */
fock_status fock_plan_columns(fock_plan_t plan, int64_t* kept, int64_t* total);

/*
 * fock_apply — V_x psi and E_x for nb orbitals (§4, V_x equation and E_x).
 *   psi_G   device complex128 [nb][npw] (interleaved re, im), canonical order.
 *   nb      number of orbitals, >= 1.
 *   occ     host double [nb]; occupations f_i (any real values).
 *   vpsi_G  device complex128 [nb][npw]; receives (V_x psi_j)(G).  Must not
 *           overlap psi_G.
 *   ex      host double or NULL; receives E_x.
 *   dex     host double or NULL; receives dE_x/domega (erfc kernel; 0 for
 *           Spencer-Alavi).
 *   stream  cudaStream_t or NULL.
 * Every unique pair i <= j is evaluated once (phi_ji = phi_ij for real
 * orbitals); two pairs share one complex transform.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
fock_status fock_apply(fock_plan_t plan, const void* psi_G, int nb, const double* occ,
                       void* vpsi_G, double* ex, double* dex, fock_stream_t stream);

/*
 * fock_apply_shard — one part of fock_apply's pair loop: the band-group
 * distribution of §5 (Fig. 3: the band loop is split over groups and the
 * results are summed at the end).  The unique pairs are cut, in the library's
 * fixed schedule, into nshards contiguous parts of near-equal size; this call
 * evaluates part `shard` (0 <= shard < nshards) and returns the partial
 * V_x psi and partial E_x, dE_x/domega.  Summing the results of all shards
 * reproduces fock_apply up to rounding.  Arguments as in fock_apply.
 */
fock_status fock_apply_shard(fock_plan_t plan, const void* psi_G, int nb, const double* occ,
                             int shard, int nshards, void* vpsi_G, double* ex, double* dex,
                             fock_stream_t stream);

/*
 * fock_set_occupied / fock_apply_fixed — the operator held fixed and applied
 * many times: the inner loop of the nested SCF of §4 (the Kohn-Sham equations
 * are converged at fixed V_x; the outer loop updates V_x).
 *
 * fock_set_occupied fixes the occupied orbitals (psi_G device complex128
 * [nb][npw], occ host [nb]) that define V_x; they are transformed to real
 * space once and kept in the plan (in FOCK_PREC_MIXED32 the plan also keeps
 * a copy of psi_G, for the FP64 overlaps of the G = 0 terms).  fock_apply_fixed then returns, for nt
 * trial orbitals phi_a (phi_G device complex128 [nt][npw]),
 *   (V_x phi_a)(r) = - sum_i f_i psi_i(r) IFFT[v FFT(psi_i* phi_a)](r)
 * on the sphere (vphi_G device complex128 [nt][npw], must not overlap phi_G):
 * nb*nt pairs, two per complex transform, the occupied orbitals are not
 * transformed again.  With phi = psi it equals fock_apply's V_x psi.
 * Any other apply on the plan (fock_apply, fock_apply_shard,
 * fock_pair_energies) replaces the occupied set; fock_apply_fixed then
 * fails with INVALID_ARG until fock_set_occupied is called again.
 * Both are stream-ordered and return without synchronising.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
fock_status fock_set_occupied(fock_plan_t plan, const void* psi_G, int nb, const double* occ,
                              fock_stream_t stream);
fock_status fock_apply_fixed(fock_plan_t plan, const void* phi_G, int nt, void* vphi_G,
                             fock_stream_t stream);

/*
 * fock_pair_energies — the pair terms of the §4 E_x sum,
 *   e_ij = sum_G v(G) |FFT(psi_i psi_j)(G)/Ntot|^2,   d_ij = the same with dv/domega,
 * for an explicit list of pairs.
 *   pairs   host int32 [npairs][2]; band indices (i, j), 0 <= i, j < nb.
 *   e, d    host double [npairs]; d may be NULL.
 * Synchronises the stream.  Errors: INVALID_ARG, OOM, CUDA.
 */
fock_status fock_pair_energies(fock_plan_t plan, const void* psi_G, int nb, const int32_t* pairs,
                               int npairs, double* e, double* d, fock_stream_t stream);

/*
 * fock_pair_energies_static — fock_pair_energies without any device
 * allocation.  The paper has no counterpart: this serves callers that must not
 * call cudaMalloc when they need the pair energies (frameworks that own every
 * device allocation or hold the process to a fixed memory budget, loops that
 * cannot take an allocation's latency or the device-wide synchronisation
 * cudaMalloc and cudaFree may imply).
 *   Arguments, results and errors as in fock_pair_energies (pairs, e and d are
 *   host arrays).
 *   It is a synchronising call: it copies the host pair list to the device,
 *   waits for the stream and scales the results on the host, so it must not be
 *   issued on a stream that is being captured into a CUDA graph.
 *   Working memory: one static device array of 32 MiB per device, held from
 *   library load to process exit.  It must hold nb*N^3 reals of the plan's
 *   precision (8 or 4 bytes), 8*npairs + 16*npairs + 16*npairs bytes, and one
 *   transform buffer of N^2 (N+2) complex elements; larger requests fail with
 *   FOCK_ERR_INVALID_ARG before any work is queued.
 *   The first call in a CUDA context of a device (with that device current)
 *   looks up the array's device address; a new context (after a device reset)
 *   looks it up again.
 *   All calls share the array: calls whose work overlaps on the GPU race.
 *   The plan's own workspace is not touched, but its tables are used.
 */
fock_status fock_pair_energies_static(fock_plan_t plan, const void* psi_G, int nb,
                                      const int32_t* pairs, int npairs, double* e, double* d,
                                      fock_stream_t stream);

/*
 * fock_sternheimer_solve — the linear-response step of the paper's GIPAW code
 * (§3.1, the Sternheimer equation and the CG paragraph after it): for each
 * right-hand ket w_n, solve
 *     (H - eps_n + alpha P) g_n = -Q w_n,   P = sum_i |u_i><u_i|,  Q = 1 - P,
 * by conjugate gradients, for the model Gamma-point Hamiltonian
 * H = -1/2 nabla^2 + V(r) on the plan's plane-wave sphere:
 *     (H c)(G) = |G|^2/2 c(G) + (sqrt(Omega)/Ntot) FFT[V(r) psi(r)](G),
 *     psi(r) = Omega^-1/2 sum_{G in S} c(G) exp(iG.r) on the plan's grid.
 * The first CG iteration updates every band; from then on the bands are kept
 * in two contiguous groups, not converged and converged, and only the first is
 * updated (a band converges when its residual norm ||-Q w_n - A_n g_n|| falls
 * below tol); the result is returned in the original band order.  Plain CG
 * from g = 0, no preconditioner.  alpha should exceed the occupied bandwidth
 * (the paper takes twice it) so that every A_n is positive definite.
 *   plan     an FP64 plan (INVALID_ARG otherwise): sphere, grid, transforms.
 *   vloc     device double [N^3]: V(r) on the grid, index (i1 N + i2) N + i3.
 *   u_G      device complex128 [nocc][npw]: the occupied states (orthonormal,
 *            Gamma-point real: c(-G) = c(G)*).
 *   eps      host double [nrhs]: eps_n.
 *   w_G      device complex128 [nrhs][npw]: the kets w_n (Gamma-point real).
 *   alpha, tol, maxiter   projector shift, residual threshold (> 0), CG
 *            iteration limit (>= 1).
 *   g_G      device complex128 [nrhs][npw]: receives g_n; must not overlap
 *            u_G or w_G.
 *   iters    host int [nrhs] or NULL: CG updates each band received.
 *   resid    host double [nrhs] or NULL: final residual norms (a band that
 *            did not reach tol within maxiter keeps its last iterate).
 * Uses the plan's real-space workspace (any fixed operator set by
 * fock_set_occupied is dropped) and allocates its own CG vectors for the
 * call.  Synchronises the stream once per CG iteration.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
fock_status fock_sternheimer_solve(fock_plan_t plan, const double* vloc, const void* u_G, int nocc,
                                   const double* eps, const void* w_G, int nrhs, double alpha, double tol,
                                   int maxiter, void* g_G, int* iters, double* resid, fock_stream_t stream);

/* ---------------------------------------------------------------- batches
 *
 * Many independent systems (uneven grids and band counts) in one batched
 * apply: the O(nb) transforms of every system, then the pair passes of all
 * systems in one persistent kernel launch that takes (chain x plane/row)
 * tasks in dependency order from a global ticket counter, then V_x psi and
 * E_x of every system; the whole sequence is captured once into a CUDA graph
 * and replayed by fock_batch_run.  This is the band-pair distribution of §5
 * applied across systems as well as across bands: no data dependency between
 * pairs except the final sums.
 */
typedef struct fock_batch* fock_batch_t;

typedef struct {
  int slot_chains;      /* chains of the largest grid per transform-buffer slot (default 8) */
  int ring;             /* transform-buffer slots in the ring, >= 3 (default 3) */
  int ctas_per_sm;      /* resident CTAs per SM of the persistent launch (0: as many as fit) */
  int use_graph;        /* 1: capture once into a CUDA graph and replay it (default 1) */
  int want_dex;         /* 1: also produce dE_x/domega (erfc plans) */
  double wait_limit_s;  /* bound on each device-side dependency wait (default 10 s) */
  int stall_segment;    /* TEST ONLY (leave at -1): >= 0 makes that segment wait for itself,
                           which can never finish, so that tests can drive the bounded-wait
                           path (FOCK_ERR_TIMEOUT) without a GPU fault */
  int persistent;       /* pair passes of the systems:
                           1: one persistent launch of resident CTAs that take (system, pass,
                              chain, plane/column) tasks in dependency order (default);
                           2: one dataflow launch with one CTA per task: each CTA takes a ticket
                              when it starts, waits (bounded) for the tasks its own depends on,
                              then runs it;
                           0: each system's pair passes as size-specialised launches on its own
                              branch of the graph (branches run concurrently) */
} fock_batch_options;

/* Fill `opt` with the defaults above. */
fock_status fock_batch_default_options(fock_batch_options* opt);

/*
 * fock_batch_create — set up a batched apply over nsys systems.
 *   plans    host [nsys] distinct plans of one precision on the current device,
 *            each on a grid of 24, 32, 48, 64, 72 or 96 points per axis.  While
 *            the batch exists it owns the plans' workspaces: do not call other
 *            entry points on them.
 *   nb       host [nsys] band counts.
 *   psi_G    host [nsys] device pointers, complex128 [nb_s][npw_s] each.
 *   occ      host [nsys] host pointers, double [nb_s] each (copied now).
 *   vpsi_G   host [nsys] device pointers, complex128 [nb_s][npw_s] each.
 *   opt      NULL for the defaults.
 * The device buffers are captured by address: fock_batch_run reads psi_G and
 * writes vpsi_G at those addresses every time (update their contents in
 * place between runs).
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, OOM, CUDA.
 */
fock_status fock_batch_create(fock_batch_t* out, int nsys, const fock_plan_t* plans, const int* nb,
                              const void* const* psi_G, const double* const* occ,
                              void* const* vpsi_G, const fock_batch_options* opt);

/*
 * fock_batch_run — run the batched apply on `stream` and wait for it.
 *   ex, dex  host double [nsys] or NULL; E_x and dE_x/domega per system.
 * Errors: CUDA, TIMEOUT (a device-side wait gave up; the outputs are invalid,
 * the batch and the device stay usable).
 */
fock_status fock_batch_run(fock_batch_t batch, double* ex, double* dex, fock_stream_t stream);

/* Kernel launches per run (the persistent launch counts once), tasks of the
 * persistent launch, its grid size, the number of segments, and the device
 * time of the persistent launch in the last run (CUDA events; -1 before the
 * first run).  Host outputs; any may be NULL. */
fock_status fock_batch_info(fock_batch_t batch, int64_t* launches, int64_t* tasks, int* grid,
                            int* segments, double* persist_ms);

/* Description of the last failure of this batch ("" if none). */
const char* fock_batch_last_error(fock_batch_t batch);

/* Release the batch (not the plans).  NULL is accepted. */
fock_status fock_batch_destroy(fock_batch_t batch);

/* ---------------------------------------------------------------- k points
 *
 * The general form of §4's E_x and V_x equations: Bloch orbitals
 * psi_nk(r) = exp(i k.r) u_nk(r) at nk points k of the Brillouin zone, the sums
 * over k and q = k - k', and the kernel at |G + q| (the 1/|G+q|^2 of §4, made
 * finite as in fock_kernel).  With states s = k * nb + n and weights w_k:
 *   psi_nk(r)       = Omega^-1/2 sum_{G in S_k} c_nk(G) exp(i (k + G).r),
 *                     S_k = {G : |k + G|^2 / 2 <= Ecut}
 *   phi(r)          = IFFT[v(G + q) FFT(u_{mk'}* u_{nk})](r)
 *   (V_x psi_nk)(G) = (sqrt(Omega)/Ntot) FFT[- sum_k' w_k' sum_m f_mk' u_mk' phi](G),  G in S_k
 *   E_x             = 1/2 sum_k w_k sum_n f_nk <psi_nk | V_x psi_nk>
 * Orbitals are general complex functions (no Gamma symmetry); every unique
 * pair of states takes one complex transform, and the reverse pair's potential
 * is its complex conjugate.  That is the plain sum over ordered pairs exactly
 * when no pair density u_a* u_b reaches a Nyquist plane (frequency -N/2 of an
 * even axis), so the grid must hold every pair density: for every two k points
 * k, k' (k = k' included) and every axis a, 2 (max m_a over S_k - min m_a over
 * S_k') < N (else fock_kplan_create returns GRID_TOO_SMALL).  Each S_k is in
 * canonical order: ascending |k + G|^2 evaluated as in fock_plan_create with
 * m_a replaced by (m_a + k_a) formed first, ties lexicographic on (m1, m2, m3).
 */
typedef struct fock_kplan* fock_kplan_t;

/*
 * fock_kplan_create — spheres, v(G + q) tables for every distinct q = k_b - k_a,
 * and the FFT plan.
 *   kpts   host double [nk][3]: k in reduced coordinates (k = sum_a kpts_a b_a).
 *   wk     host double [nk]: k-point weights (usually summing to 1).
 *   Other arguments as fock_plan_create.  FOCK_PREC_MIXED32: the kernel terms
 *   with |m + q|^2 <= 3 (m + q in reduced coordinates) in FP64, and for the
 *   pairs of one k point the G = 0 value of the pair density from the FP64
 *   overlap sum_G c_a(G)* c_b(G) of the input coefficients.
 * The grid is checked on the host before any CUDA call: GRID_TOO_SMALL when
 * an S_k does not fit (2 |m_a| >= N) or a pair density reaches the Nyquist
 * frequency (the condition above).
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, GRID_TOO_SMALL, OOM, CUDA.
 */
fock_status fock_kplan_create(fock_kplan_t* out, const int grid[3], const double cell[9], double ecut_ha,
                              int nk, const double* kpts, const double* wk, fock_kernel kind,
                              const double* kparams, int nkparams, fock_precision prec);

/* The sphere S_k = {G : |k + G|^2 / 2 <= Ecut} (kpt host double[3], reduced)
 * in canonical order without creating a plan; as fock_gsphere otherwise. */
fock_status fock_gsphere_k(const int grid[3], const double cell[9], double ecut_ha, const double* kpt,
                           int64_t* npw, int32_t* miller, int64_t capacity);

/* Number of k points of the plan (host output): the length of the psi_G and
 * vpsi_G pointer arrays and the rows of occ that fock_kplan_apply reads. */
fock_status fock_kplan_nk(fock_kplan_t plan, int* nk);

/* Plane waves and Miller indices of S_k (host outputs; miller int32 [npw_k][3]). */
fock_status fock_kplan_npw(fock_kplan_t plan, int k, int64_t* npw);
fock_status fock_kplan_gvectors(fock_kplan_t plan, int k, int32_t* miller);

/* Pairs per launch of the pair passes (one pair per chain here).  INVALID_ARG. */
fock_status fock_kplan_set_batch(fock_kplan_t plan, int chain_batch);

/*
 * fock_kplan_apply — V_x psi_nk for every k and E_x.
 *   psi_G    host array [nk] of device pointers, complex128 [nb][npw_k] each;
 *            nk is the plan's (fock_kplan_nk): the call reads exactly nk
 *            entries of psi_G and vpsi_G and nk * nb occupations.
 *   nb       bands per k point.
 *   occ      host double [nk][nb]: occupations f_nk.
 *   vpsi_G   host array [nk] of device pointers, complex128 [nb][npw_k] each
 *            (each must not overlap its psi_G).
 *   ex       host double or NULL.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
fock_status fock_kplan_apply(fock_kplan_t plan, const void* const* psi_G, int nb, const double* occ,
                             void* const* vpsi_G, double* ex, fock_stream_t stream);

/* Description of the last failure ("" if none); plan may be NULL for create. */
const char* fock_kplan_last_error(fock_kplan_t plan);

/* Release the k-point plan.  NULL is accepted. */
fock_status fock_kplan_destroy(fock_kplan_t plan);

/* Release the plan and everything it holds.  NULL is accepted. */
fock_status fock_destroy(fock_plan_t plan);

/* Static, never-NULL description of a status code. */
const char* fock_status_string(fock_status s);

/* Description of the last failure on this plan ("" if none); plan may be NULL
 * for failures of fock_plan_create.  Valid until the next call on the plan. */
const char* fock_last_error(fock_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* FOCK_H */
