// fock_internal.h — what the host plan (fock_plan.cpp) and the kernel
// translation units (fock_kernels_f64.cu, fock_kernels_f32.cu) share.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>


struct fock_plan;

namespace fockx {

// Two band pairs that share one complex transform: pair a = (ai, aj) in the
// real part, pair b = (bi, bj) in the imaginary part (bi < 0: no pair b).
// pa / pb index the per-pair energy slots (< 0: no energy wanted).
// flags bit 0 / bit 1: pair a / b updates only W_aj / W_bj (the operator
// applied to a trial orbital j), not the symmetric partner W_ai / W_bi.
struct Chain {
  int ai, aj, bi, bj;
  int pa, pb;
  int flags, pad1;
};
constexpr int kChainOneSidedA = 1;
constexpr int kChainOneSidedB = 2;

// Everything a kernel needs to know about a plan (device pointers included).
struct DevPlan {
  int n;            // cubic grid N
  int k3h;          // N/2 + 1: stored half of the last axis
  int64_t ntot;     // N^3
  int64_t hsize;    // elements of one half-spectrum pair buffer: N * N * 2 * k3h
  int npw;
  const int* gidx;     // [npw] grid offset of G
  const int* gidxneg;  // [npw] grid offset of -G
  const void* tw;      // [N] exp(-2 pi i t / N) in the working precision
  const void* vtab;    // [N][N][k3h] v(G) / Ntot in the working precision
  const double* vtab64;   // [N][N][k3h] v(G) in FP64
  const double* dvtab64;  // [N][N][k3h] dv/domega in FP64 (NULL: not needed)
  const void* dvtab;      // [N][N][k3h] dv/domega in the working precision
  double inv_ntot;     // 1 / Ntot
  double psi_scale;    // 1 / sqrt(Omega)
  double out_scale;    // sqrt(Omega) / Ntot
  int msmall2;         // |m|^2 at or below which kernel terms are done in FP64 (mixed form)
  // Columns of the stored half that pair densities reach (Gamma point): row k2
  // keeps k3 < ncol[k2]; the column pass takes them NC = 2 (N/2 + 1) lines per
  // CTA from colmap (ncta_col * NC entries, (k2 << 16) | (s << 15) | k3, -1: none)
  const int* ncol;
  const int* colmap;
  int ncta_col;
  // rows k2 that have kept columns are [0, row_lo) and [N - row_hi, N) (a
  // ball centred on G = 0 reaches a symmetric range of m2; row_lo = N,
  // row_hi = 0 when every row is kept); col_max = the largest ncol[k2]
  int row_lo, row_hi, col_max;
  // the kept columns (k2 << 16) | k3 in row order (nkept entries)
  const int* kept;
  int nkept;
  // radix-plan variant ("tiling", 0 or 1) of the forward plane, column and
  // inverse plane passes
  int tile[3];
  // deterministic accumulation: W holds 64-bit fixed point scaled by det_scale[0]
  // (= 2^s), the column pass stores per-CTA energy partials at [pair * ncta_col + cta]
  int det;
  const double* det_scale;
  // Brillouin-zone sampling: full-grid tables [nq][N][N][N] of v(G + q)
  const void* vtabq;      // v / Ntot in the working precision
  const double* vtabq64;  // v in FP64
  // mixed form with k points: q of each table in reduced coordinates
  // ([nq][3]; terms with |m + q|^2 <= msmall2 are done in FP64), the index of
  // q = 0 (-1: none), and the FP64 overlaps of the states of each k point
  // (kovl_re/im [nk][nb][nb], entries n <= n'), whose q = 0 pairs take their
  // G = 0 value from them (times ovl_scale).  NULL: transform values.
  const float* qfrac;
  int q0;
  const double* kovl_re;
  const double* kovl_im;
  int kovl_nb;
  // mixed form: FP64 overlaps S(i, j) = Re sum_G conj(c_i(G)) c_j(G) of the
  // pairs (i <= j) at ovl[i * ovl_ld + j - ovl_j0]; the column pass takes the
  // G = 0 value of a pair density as ovl_scale * S(i, j) (= sum over the grid
  // of psi_i psi_j, ovl_scale = Ntot / Omega).  NULL: the transform's value.
  const double* ovl;
  int ovl_ld, ovl_j0;
  double ovl_scale;
  // FP64 form with one occupation f0 for every band: vtab
  // then holds -f0 v / Ntot (and vtab_f points at it), so that phi arrives at
  // the inverse pass already scaled by -f0 and its accumulator update saves
  // the two multiplications by -f per point.  NULL: vtab is v / Ntot, and the
  // update multiplies by -f itself.  vtab_f_factor = -f0 (nonzero).
  const void* vtab_f;
  double vtab_f_factor;
};

struct KernelOps {
  int real_bytes;  // sizeof of the working real type
  int prec;        // 0 FP64, 1 mixed FP32, 2 double-float (fock_precision)
  int n;           // grid size these kernels are compiled for
  int col_lines;   // lines of the column map a column-pass CTA takes
  size_t smem;     // largest dynamic shared memory of its kernels
  cudaError_t (*configure)(const DevPlan&);
  // c(G) of bands [band0, band0 + nbat) to psi(r); X is scratch of >= ceil(nbat/2) grids.
  cudaError_t (*to_real)(const DevPlan&, const double2* psiG, int nb, int band0, int nbat, void* X,
                         void* psi, cudaStream_t);
  // Forward plane pass of the pair densities of `nch` chains into H.
  cudaError_t (*pair_fwd)(const DevPlan&, const void* psi, const Chain* ch, int nch, void* H,
                          cudaStream_t);
  // Column pass: forward, times v, energy partials, inverse.
  cudaError_t (*pair_col)(const DevPlan&, void* H, const Chain* ch, int nch, double* epair,
                          double* dpair, cudaStream_t);
  // Inverse plane pass and W -= f psi phi accumulation.
  cudaError_t (*pair_inv)(const DevPlan&, const void* psi, void* W, const void* occ,
                          const Chain* ch, int nch, const void* H, cudaStream_t);
  // W(r) of bands [band0, band0 + nbat) to (V_x psi)(G) on the sphere.
  cudaError_t (*to_sphere)(const DevPlan&, const void* W, int nb, int band0, int nbat, void* X,
                           double2* vpsiG, cudaStream_t);
  // radix plan of a tiling of a pair pass (pass 0 fwd, 1 col, 2 inv; tile 0/1):
  // radices[nst], threads per line, threads per CTA; returns the number of
  // distinct tilings (1 or 2)
  int (*tile_plan)(int pass, int tile, int* radices, int* nst, int* threads_per_line, int* threads);
};

// Kernels for grid size n and precision (0: FP64, 1: mixed); NULL if not built.
const KernelOps* find_kernel_ops(int prec, int n);

// Kernels of the Brillouin-zone-sampled apply (complex periodic parts, one pair
// per transform; band0 is a global state index, psiG / vpsiG point at the
// first band of the batch).
struct KOps {
  cudaError_t (*configure)();
  cudaError_t (*to_real)(const DevPlan&, const double2* psiG, int npw, const int* gidx, int band0, int nbat,
                         void* X, void* u, cudaStream_t);
  cudaError_t (*pair_fwd)(const DevPlan&, const void* u, const Chain* ch, int nch, void* H, cudaStream_t);
  cudaError_t (*pair_col)(const DevPlan&, void* H, const Chain* ch, int nch, double* epair, cudaStream_t);
  cudaError_t (*pair_inv)(const DevPlan&, const void* u, void* W, const void* occw, const Chain* ch, int nch,
                          const void* H, cudaStream_t);
  cudaError_t (*to_sphere)(const DevPlan&, const void* W, int band0, int nbat, int npw, const int* gidx,
                           void* X, double2* vpsiG, cudaStream_t);
};
const KOps* find_kops(int prec, int n);

// One system of a batch as the persistent kernel sees it.
struct SysDesc {
  DevPlan g;
  const void* psi;
  void* W;
  const void* occT;
  const Chain* chains;
  double* epair;
  double* dpair;
};

// A run of tasks of one pass kind over consecutive chains of one system.
struct Segment {
  int kind;    // 0: forward plane pass, 1: column pass, 2: inverse plane pass
  int sys;     // system index
  int chain0;  // first chain (index into the system's chain list)
  int nch;     // chains
  int slot;    // transform-buffer slot; chain k of the run uses slot + k * hsize elements
  int dep;     // segment that must be complete first (-1: none)
  int dep2;    // second such segment (-1: none)
  int task0;   // first ticket
  int ntasks;  // (N, or ncta_col for the column pass) * nch
  int pad;
};

struct PersistOps {
  int real_bytes;
  size_t smem;
  cudaError_t (*configure)();
  cudaError_t (*occupancy)(int* ctas_per_sm);
  cudaError_t (*launch)(int grid, const SysDesc* sys, const Segment* seg, int nseg, int ntasks,
                        unsigned* counters, unsigned char* hring, size_t slot_bytes,
                        unsigned long long limit_ns, cudaStream_t s);
  // one CTA per task, inlined bodies, dependency waits (grid = ntasks)
  cudaError_t (*launch_dataflow)(const SysDesc* sys, const Segment* seg, int nseg, int ntasks,
                                 unsigned* counters, unsigned char* hring, size_t slot_bytes,
                                 unsigned long long limit_ns, cudaStream_t s);
};

// Persistent pair kernel of a precision (0: FP64, 1: mixed).
const PersistOps* find_persist_ops(int prec);
// Grid sizes the persistent kernel runs.
bool persist_supports(int n);

// What code outside fock_plan.cpp may read of a plan.
struct PlanView {
  int device;
  const KernelOps* ops;
  DevPlan dp;
};
bool plan_view(struct ::fock_plan* plan, PlanView* out);
void plan_set_error(struct ::fock_plan* plan, const char* msg);

// Deterministic accumulation.  Per band b of psi (real-space, type code prec):
// stats[2b] = max |psi_b|, stats[2b+1] = sum psi_b^2; then the fixed-point scale
// [2^s, 2^-s] into scale from the bound of the header (vnorm = ||v||_2 over the
// grid, occupations of the nsrc source bands); W (int64 fixed point) to double
// in place; per-pair sums of the per-CTA energy partials in a fixed order.
cudaError_t launch_orbital_stats(int prec, const void* psi, int nbands, int64_t ntot, double* stats,
                                 cudaStream_t s);
cudaError_t launch_det_scale(const double* stats, int nbands, const double* occ, int nsrc, double vnorm,
                             int64_t ntot, double* scale, cudaStream_t s);
cudaError_t launch_det_to_double(void* w, int64_t n, const double* scale, cudaStream_t s);
cudaError_t launch_det_pair_sums(const double* part, int npairs, int ncta, double* out, cudaStream_t s);

// Sternheimer CG (fock_sternheimer.cu): kets are complex128 [m][npw], FP64.
cudaError_t st_vmul(const double* v, const double* psi, double* w, int m, int64_t ntot, cudaStream_t s);
cudaError_t st_dots(const double2* a, const double2* b, int m, int npw, double* out, cudaStream_t s);
cudaError_t st_proj_coef(const double2* u, int nocc, const double2* x, int m, int npw, double* c, cudaStream_t s);
cudaError_t st_rhs(const double2* w, const double2* u, const double* c, int nocc, int m, int npw, double2* b,
                   cudaStream_t s);
cudaError_t st_finish(double2* ap, const double2* p, const double* kin, const double* eps, const double2* u,
                      const double* c, int nocc, double alpha, int m, int npw, cudaStream_t s);
cudaError_t st_step(double2* x, double2* r, const double2* p, const double2* ap, const double* rr, const double* pap,
                    int m, int npw, cudaStream_t s);
cudaError_t st_dir(double2* p, const double2* r, const double* rr_new, const double* rr, int m, int npw,
                   cudaStream_t s);
cudaError_t st_gather_rows(const double2* src, double2* dst, const int* perm, int m, int npw, cudaStream_t s);
cudaError_t st_gather_scalars(const double* src, double* dst, const int* perm, int m, cudaStream_t s);

// out[i] = factor * v[i], i < n (FP64).
cudaError_t launch_scaled_table(const double* v, int64_t n, double factor, double* out, cudaStream_t s);

// S[i * ld + j] = Re sum_G conj(a_i(G)) b_j(G) for i < na, j < nb (sym: a = b
// and only j >= i), in FP64, a and b complex128 rows of npw; S is overwritten
// at those entries (others untouched).  half (device, nhalf positions, or
// NULL): G = 0 first, then one of each pair G, -G; for Gamma-point rows
// (c(-G) = conj c(G)) the sum is then taken over that half of the sphere,
// the pairs' terms doubled.
cudaError_t launch_overlap(const double2* a, int na, const double2* b, int nb, int npw, const int* half, int nhalf,
                           bool sym, double* S, int ld, cudaStream_t s);
// Complex overlaps of nsets sets of nb rows with themselves (set z: the
// device pointer rows[z] to nb rows of npw[z] complex128; rows and npw are
// device arrays, npw_max their largest npw): Sre/Sim[z][i][j] = Re/Im
// sum_G conj(c_i(G)) c_j(G) for j >= i, in FP64 (Sre, Sim [nsets][nb][nb],
// overwritten).
cudaError_t launch_overlap_sets(const double2* const* rows, const int* npw, int npw_max, int nsets, int nb,
                                double* Sre, double* Sim, cudaStream_t s);

// E = scale * sum_p f_i f_j (1 or 2) e_p over the pairs; out[0] = E, out[1] = dE.
cudaError_t launch_energy_reduce(const int2* pairs, int npairs, const double* occ,
                                 const double* epair, const double* dpair, double scale,
                                 double* out, cudaStream_t s);

}  // namespace fockx
