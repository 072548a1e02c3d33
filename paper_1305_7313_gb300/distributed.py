"""Band groups over several GPUs: the distribution of the paper's exact-exchange
loop (§5, Fig. 3: the band-pair loop is split across groups of processes and
the partial results are summed at the end).

Every rank holds all orbitals.  :func:`apply` evaluates this rank's share of
the unique band pairs with the library's ``fock_apply_shard`` (contiguous
shards of the library's fixed pair schedule, one per rank of the group), then
sums the partial V_x psi and the partial [E_x, dE_x/domega] over the group
with two all-reduces.  The result on every rank equals ``fock_apply`` on one
GPU up to the order of the floating-point sums.
"""

import numpy as np


def apply(plan, psi_G, occ, group=None, vpsi_G=None, want_dex=False, stream=None):
    """(V_x psi, E_x, dE_x/domega) summed over the ranks of ``group``.

    ``plan``: a :class:`FockPlan` (or any object with the same ``apply_shard``);
    ``psi_G``: this rank's copy of all orbitals, complex128 [nb, npw] on the
    device the process group's backend reduces (CUDA for NCCL); ``occ``: host
    occupations [nb].  ``group``: a ``torch.distributed`` process group (None:
    the default group).  Shard k of the pair schedule goes to the rank of index
    k in the group.  Returns the summed V_x psi (in ``vpsi_G`` when given), E_x
    and dE_x/domega (None unless ``want_dex``).
    """
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    vpsi, ex, dex = plan.apply_shard(psi_G, occ, rank, world, vpsi_G, True, want_dex, stream)
    energies = torch.tensor([ex, dex if dex is not None else 0.0], dtype=torch.float64, device=vpsi.device)
    if world > 1:
        dist.all_reduce(torch.view_as_real(vpsi), group=group)
        dist.all_reduce(energies, group=group)
    e = energies.cpu().numpy().astype(np.float64)
    return vpsi, float(e[0]), (float(e[1]) if want_dex else None)
