"""The synthetic workloads the library is measured and tested on.

They stand in for the paper's hybrid-functional benchmark (§6: amorphous SiO2
with an oxygen interstitial, about 108 atoms and 800 bands, EXX cutoff equal to
the density cutoff), whose data set is not available: cubic cells with many
occupied bands and FFT grids large enough to hold the pair-density sphere.
"""

import numpy as np

SPENCER_ALAVI = 0
ERFC = 1
PREC_FP64 = 0
PREC_MIXED32 = 1
PREC_DF64 = 2


def cubic_cell(length):
    return (float(length) * np.eye(3)).ravel().tolist()


WORKLOADS = {
    # small parity case: 24^3 grid, 8 bands, Spencer-Alavi kernel, FP64
    "gamma_fp64_L10_N24_nb8": dict(L=10.0, N=24, ecut=10.0, nb=8, kernel=SPENCER_ALAVI,
                                   omega=None, prec=PREC_FP64, seed=1305),
    # large cell: 96^3 grid, 512 bands, all 131,328 pairs, FP64
    "gamma_fp64_L27_N96_nb512": dict(L=27.0, N=96, ecut=12.0, nb=512, kernel=SPENCER_ALAVI,
                                     omega=None, prec=PREC_FP64, seed=1306),
    # the FP64 workload in double-float arithmetic (FP64-class accuracy on the FP32 pipe)
    "gamma_df64_L27_N96_nb512": dict(L=27.0, N=96, ecut=12.0, nb=512, kernel=SPENCER_ALAVI,
                                     omega=None, prec=PREC_DF64, seed=1306),
    # complex64 transforms with FP64 energy sums, erfc kernel
    "gamma_mixed32_erfc_L27_N96_nb512": dict(L=27.0, N=96, ecut=12.0, nb=512, kernel=ERFC,
                                             omega=0.106, prec=PREC_MIXED32, seed=1307),
    # differentiation: 72^3 grid, L = 20, 256 bands, erfc kernel
    "grad_erfc_L20_N72_nb256": dict(L=20.0, N=72, ecut=12.0, nb=256, kernel=ERFC,
                                    omega=0.106, prec=PREC_MIXED32, seed=1309),
}


def batched_systems(seed=3):
    """Sixteen uneven systems: grids 48/64/72/96 (four each), L = 27 N / 96, bands in [32, 384]."""
    nbs = np.random.default_rng(seed).integers(32, 385, 16)
    out = []
    for k, n in enumerate([48] * 4 + [64] * 4 + [72] * 4 + [96] * 4):
        out.append(dict(L=27.0 * n / 96.0, N=n, ecut=12.0, nb=int(nbs[k]), kernel=SPENCER_ALAVI,
                        omega=None, prec=PREC_MIXED32, seed=1308 + 100 * k))
    return out
