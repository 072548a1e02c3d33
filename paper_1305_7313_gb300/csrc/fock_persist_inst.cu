// One precision of the persistent batched pair kernel.  Built with
// -DFOCK_T=<double|float> -DFOCK_OPS_NAME=<symbol>.
#include "fock_persist.cuh"

#if !defined(FOCK_T) || !defined(FOCK_OPS_NAME)
#error "compile with -DFOCK_T and -DFOCK_OPS_NAME"
#endif

namespace fockx {
extern const PersistOps FOCK_OPS_NAME;
const PersistOps FOCK_OPS_NAME = PersistLaunch<FOCK_T>::ops();
}  // namespace fockx
