// Host check of the Coulomb kernels the plans tabulate (fock_lattice.h,
// kernel_value): prints, as exact hexadecimal doubles, one value per line
//   <kind 0 spencer-alavi | 1 erfc> <volume> <omega> <|G|^2> <v> <dv/domega>
// over cell volumes, screening parameters and |G|^2 from 0 to beyond 8 Ecut of
// the workloads; the test compares them with the oracle's kernels.
#include <cmath>
#include <cstdio>

#include "fock_lattice.h"

using namespace fockx;

int main() {
  const double volumes[] = {1000.0, 19683.0, 8000.0, 27000.0, 736.3};
  const double omegas[] = {0.106, 0.3, 0.5, 1.0};
  const double g2s[] = {0.0, 1e-12, 1e-8, 1e-4, 1e-2, 0.05, 0.1, 0.3947841760435743, 1.0, 2.5, 7.0, 24.0,
                        96.0, 200.0, 400.0, 1000.0};
  for (double vol : volumes) {
    for (double g2 : g2s) {
      double v, dv;
      lattice::kernel_value(FOCK_KERNEL_SPENCER_ALAVI, vol, 0.0, g2, &v, &dv);
      std::printf("0 %a %a %a %a %a\n", vol, 0.0, g2, v, dv);
    }
    for (double om : omegas) {
      for (double g2 : g2s) {
        double v, dv;
        lattice::kernel_value(FOCK_KERNEL_ERFC, vol, om, g2, &v, &dv);
        std::printf("1 %a %a %a %a %a\n", vol, om, g2, v, dv);
      }
    }
  }
  return 0;
}
