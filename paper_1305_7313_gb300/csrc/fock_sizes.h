// fock_sizes.h — the cubic grid sizes N the kernels are compiled for.  The
// build compiles fock_kernels_inst.cu once per (precision, N) of this list.
#pragma once
#define FOCK_GRID_SIZES(X) X(8) X(12) X(16) X(24) X(32) X(36) X(48) X(64) X(72) X(96)
