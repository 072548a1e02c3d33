"""fock_pair_energies_static — the entry point for callers that cannot allocate
device memory (a framework that owns all device memory or holds the process to
a fixed budget, a loop that cannot take an allocation's latency) — against the
allocating fock_pair_energies.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  It builds its own inputs, so it passes alone
in a fresh process as well as after the rest of the suite.
"""

import numpy as np
import pytest

from paper_1305_7313_gb300 import FockPlan, synth
from paper_1305_7313_gb300 import _lib
from tests._common import cubic, require_gpu

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 5e-6


# The last two cases need more chains than one transform buffer of the static
# array holds (48^3 FP64: 13 chains per block for 24 chains; 48^3 mixed with the
# list repeated three times: 30 per block for 72 chains), so the call runs its
# loop over several chain blocks.
@pytest.mark.parametrize("N,L,ecut,nb,kind,omega,prec,tol,reps", [
    (24, 10.0, 10.0, 8, _lib.SPENCER_ALAVI, None, _lib.PREC_FP64, TOL64, 1),
    (24, 10.0, 10.0, 8, _lib.SPENCER_ALAVI, None, _lib.PREC_DF64, TOL64, 1),
    (48, 13.5, 12.0, 9, _lib.ERFC, 0.106, _lib.PREC_MIXED32, TOL32, 1),
    (48, 13.5, 12.0, 9, _lib.SPENCER_ALAVI, None, _lib.PREC_FP64, TOL64, 1),
    (48, 13.5, 12.0, 9, _lib.ERFC, 0.106, _lib.PREC_MIXED32, TOL32, 3),
])
def test_static_scratch_matches_the_allocating_entry_point(N, L, ecut, nb, kind, omega, prec, tol, reps):
    torch = require_gpu()
    cell = cubic(L)
    plan = FockPlan(N, cell, ecut, kind, omega, prec)
    c = synth.orbitals(plan.miller, cell, nb, 2024 + N)
    psi = torch.from_numpy(c).cuda()
    pairs = ([(i, j) for i in range(nb) for j in range(i, nb)] + [(3, 1), (2, 2), (nb - 1, 0)]) * reps
    e_ref, d_ref = plan.pair_energies(psi, pairs, want_d=True)
    for _ in range(2):  # the second call must not see the first call's leftovers
        e, d = _lib.fock_pair_energies_static(plan.handle, psi, pairs, want_d=True)
        assert np.max(np.abs(e - e_ref)) <= tol * np.max(np.abs(e_ref))
        assert np.max(np.abs(d - d_ref)) <= tol * max(np.max(np.abs(d_ref)), 1e-300)
    # a different, shorter pair list right after still gives the right values
    e2 = _lib.fock_pair_energies_static(plan.handle, psi, pairs[:3])
    assert np.max(np.abs(e2 - e_ref[:3])) <= tol * np.max(np.abs(e_ref[:3]))
    plan.close()


def test_static_scratch_rejects_requests_beyond_its_size():
    torch = require_gpu()
    cell = cubic(10.0)
    plan = FockPlan(24, cell, 10.0)
    nb = 400  # 400 * 24^3 doubles = 44 MB of real-space orbitals > 32 MiB
    psi = torch.zeros((nb, plan.npw), dtype=torch.complex128, device="cuda")
    with pytest.raises(_lib.FockError) as err:
        _lib.fock_pair_energies_static(plan.handle, psi, [(0, 1)])
    assert err.value.status == 1 and "32 MiB" in str(err.value)
    plan.close()
