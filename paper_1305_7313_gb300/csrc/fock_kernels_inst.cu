// One (precision, grid size) instantiation of the Fock apply kernels.  Built
// with -DFOCK_T=<double|float> -DFOCK_N=<N> -DFOCK_OPS_NAME=<symbol>.
#include "fock_kernels.cuh"

#if !defined(FOCK_T) || !defined(FOCK_N) || !defined(FOCK_OPS_NAME)
#error "compile with -DFOCK_T, -DFOCK_N and -DFOCK_OPS_NAME"
#endif

namespace fockx {
extern const KernelOps FOCK_OPS_NAME;
const KernelOps FOCK_OPS_NAME = Launch<FOCK_T, FOCK_N>::ops();
}  // namespace fockx
