// One (precision, grid size) instantiation of the Fock apply kernels (Gamma
// point and Brillouin-zone sampled).  Built with -DFOCK_T=<double|float>
// -DFOCK_N=<N> -DFOCK_OPS_NAME=<symbol> -DFOCK_KOPS_NAME=<symbol>.
#include "fock_kernels.cuh"
#include "fock_kernels_k.cuh"

#if !defined(FOCK_T) || !defined(FOCK_N) || !defined(FOCK_OPS_NAME) || !defined(FOCK_KOPS_NAME)
#error "compile with -DFOCK_T, -DFOCK_N, -DFOCK_OPS_NAME and -DFOCK_KOPS_NAME"
#endif

namespace fockx {
extern const KernelOps FOCK_OPS_NAME;
const KernelOps FOCK_OPS_NAME = Launch<FOCK_T, FOCK_N>::ops();
extern const KOps FOCK_KOPS_NAME;
const KOps FOCK_KOPS_NAME = LaunchK<FOCK_T, FOCK_N>::ops();
}  // namespace fockx
