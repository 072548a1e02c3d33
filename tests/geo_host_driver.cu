// Host check of the pair passes' compile-time geometry (Geo in
// fock_kernels.cuh).  For every compiled grid size, real type and FFT tiling
// it prints one line:
//   <type 0 FP64 | 1 FP32 | 2 double-float> <N> <tile> <NC> <NLC> <TLC>
//   <THR_COL> <THR_COLH> <SMEM_COLH> <MIN_CTAS_COL> <SMEM_PLANE> <SMEM_INV>
//   <THR_PLANE> <MIN_CTAS> <bytes of a complex value>
// The test checks the launch constraints these numbers must meet; nothing
// here runs on a GPU.
#include <cstdio>

#include "fock_kernels.cuh"
#include "fock_sizes.h"

using namespace fockx;

namespace {

template <class T, int N, int E>
void row(int type, int tile) {
  using G = Geo<T, N, kMaxThreads, E>;
  std::printf("%d %d %d %d %d %d %d %d %zu %d %zu %zu %d %d %zu\n", type, N, tile, G::NC, G::NLC, G::TLC,
              G::THR_COL, G::THR_COLH, G::SMEM_COLH, G::MIN_CTAS_COL, G::SMEM_PLANE, G::SMEM_INV, G::THR_PLANE,
              G::MIN_CTAS, sizeof(typename G::C));
}

template <class T, int N>
void rows(int type) {
  row<T, N, 0>(type, 0);
  constexpr int E1 = tile1_emax<T, N>();
  if constexpr (E1 != 0) row<T, N, E1>(type, 1);
}

}  // namespace

int main() {
#define FOCK_GEO_ROWS(N) \
  rows<double, N>(0);    \
  rows<float, N>(1);     \
  rows<df64, N>(2);
  FOCK_GRID_SIZES(FOCK_GEO_ROWS)
#undef FOCK_GEO_ROWS
  return 0;
}
