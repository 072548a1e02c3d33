// One (precision, grid size) instantiation of the Fock apply kernels (Gamma
// point, and Brillouin-zone sampled when FOCK_KOPS_NAME is given).  Built with
// -DFOCK_T=<double|float|df64> -DFOCK_N=<N> -DFOCK_OPS_NAME=<symbol>
// [-DFOCK_KOPS_NAME=<symbol>].
#include "fock_kernels.cuh"
#ifdef FOCK_KOPS_NAME
#include "fock_kernels_k.cuh"
#endif

#if !defined(FOCK_T) || !defined(FOCK_N) || !defined(FOCK_OPS_NAME)
#error "compile with -DFOCK_T, -DFOCK_N and -DFOCK_OPS_NAME"
#endif

namespace fockx {
extern const KernelOps FOCK_OPS_NAME;
const KernelOps FOCK_OPS_NAME = Launch<FOCK_T, FOCK_N>::ops();
#ifdef FOCK_KOPS_NAME
extern const KOps FOCK_KOPS_NAME;
const KOps FOCK_KOPS_NAME = LaunchK<FOCK_T, FOCK_N>::ops();
#endif
}  // namespace fockx
