"""The band-group distribution of the paper (§5, Fig. 3: the band loop is split
across groups and the results are summed at the end) as the library shards it,
on two CPU ranks over gloo.

Each rank asks the library (host-only ``fock_schedule``, no GPU) for its share
of the unique pairs, evaluates those pairs with the FP64 oracle's primitives,
and the partial V_x psi and E_x are summed with all_reduce; the sum must equal
the oracle's full apply.  This is the exchange step a multi-GPU run would do
with NCCL.  The second test runs the product's reduce,
``paper_1305_7313_gb300.distributed.apply``, over the same ranks with a plan
whose shard is computed by the oracle.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case():
    import oracle
    from paper_1305_7313_gb300 import synth
    grid = (24, 24, 24)
    cell = (10.0 * np.eye(3)).ravel()
    mill, _ = oracle.gsphere(grid, cell, 10.0)
    nb = 9
    c = synth.orbitals(mill, cell, nb, 99)
    occ = np.linspace(2.0, 1.0, nb)
    return grid, cell, mill, c, occ


def _partial(rank, world, grid, cell, mill, c, occ, kind="spencer_alavi", omega=None):
    import oracle
    from oracle.fock import kernel_grid
    from paper_1305_7313_gb300 import _lib
    pairs = _lib.fock_schedule(len(c), rank, world)
    psi = oracle.orbitals_to_real(c, mill, grid, cell, real=True)
    vg, dvg = kernel_grid(kind, grid, cell, omega)
    w = np.zeros_like(psi)
    e = d = 0.0
    for i, j in pairs:
        phi = oracle.pair_potential(psi[i], psi[j], vg).real
        w[j] -= occ[i] * psi[i] * phi
        if i != j:
            w[i] -= occ[j] * psi[j] * phi
        eij, dij = oracle.pair_energy(psi[i], psi[j], vg, dvg)
        e += occ[i] * occ[j] * (1.0 if i == j else 2.0) * eij
        d += occ[i] * occ[j] * (1.0 if i == j else 2.0) * dij
    vol = abs(np.linalg.det(np.asarray(cell).reshape(3, 3)))
    if kind == "spencer_alavi":
        return oracle.real_to_sphere(w, mill, grid, cell), -0.5 * vol * e, pairs
    return oracle.real_to_sphere(w, mill, grid, cell), (-0.5 * vol * e, -0.5 * vol * d), pairs


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    grid, cell, mill, c, occ = _case()
    vpart, epart, pairs = _partial(rank, world, grid, cell, mill, c, occ)
    v = torch.from_numpy(np.ascontiguousarray(np.stack([vpart.real, vpart.imag])))
    e = torch.tensor([epart], dtype=torch.float64)
    dist.all_reduce(v)
    dist.all_reduce(e)
    np.save(os.path.join(outdir, "pairs_%d.npy" % rank), np.asarray(pairs))
    if rank == 0:
        np.save(os.path.join(outdir, "vsum.npy"), (v[0] + 1j * v[1]).numpy())
        np.save(os.path.join(outdir, "esum.npy"), e.numpy())
    dist.destroy_process_group()


def test_two_rank_band_groups_sum_to_the_full_result(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from tests._common import built_library
    built_library()
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    grid, cell, mill, c, occ = _case()
    vref, eref, _ = oracle.fock_apply(c, occ, mill, grid, cell, "spencer_alavi")
    vsum = np.load(tmp_path / "vsum.npy")
    esum = float(np.load(tmp_path / "esum.npy")[0])
    assert np.max(np.abs(vsum - vref)) <= 1e-12 * np.max(np.abs(vref))
    assert abs(esum - eref) <= 1e-12 * abs(eref)
    # the shards are disjoint and cover every unique pair once
    allp = [tuple(p) for r in range(world) for p in np.load(tmp_path / ("pairs_%d.npy" % r)).tolist()]
    nb = len(c)
    assert len(allp) == len(set(allp)) == nb * (nb + 1) // 2
    assert set(allp) == {(i, j) for i in range(nb) for j in range(i, nb)}


OMEGA = 0.5


class _OracleShardPlan:
    """Stands in for a FockPlan on a CPU rank: apply_shard evaluates the
    shard's pairs with the oracle and returns a CPU tensor."""

    def __init__(self, grid, cell, mill, c):
        self.args = (grid, cell, mill, c)

    def apply_shard(self, psi_G, occ, shard, nshards, vpsi_G=None, want_ex=True, want_dex=False, stream=None):
        grid, cell, mill, c = self.args
        v, (e, d), _ = _partial(shard, nshards, grid, cell, mill, c, occ, "erfc", OMEGA)
        out = torch.from_numpy(np.ascontiguousarray(v))
        if vpsi_G is not None:
            vpsi_G.copy_(out)
            out = vpsi_G
        return out, e, (d if want_dex else None)


def _product_worker(rank, world, port, outdir):
    import torch.distributed as dist
    from paper_1305_7313_gb300 import distributed
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    grid, cell, mill, c, occ = _case()
    plan = _OracleShardPlan(grid, cell, mill, c)
    psi = torch.from_numpy(c)
    vpsi, ex, dex = distributed.apply(plan, psi, occ, want_dex=True)
    np.save(os.path.join(outdir, "v_%d.npy" % rank), vpsi.numpy())
    np.save(os.path.join(outdir, "e_%d.npy" % rank), np.array([ex, dex]))
    dist.destroy_process_group()


def test_distributed_apply_sums_vpsi_and_both_energies_over_the_group(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from tests._common import built_library
    built_library()
    world = 2
    mp.spawn(_product_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    grid, cell, mill, c, occ = _case()
    vref, eref, dref = oracle.fock_apply(c, occ, mill, grid, cell, "erfc", OMEGA)
    for r in range(world):  # every rank holds the full result
        v = np.load(tmp_path / ("v_%d.npy" % r))
        ex, dex = np.load(tmp_path / ("e_%d.npy" % r))
        assert np.max(np.abs(v - vref)) <= 1e-12 * np.max(np.abs(vref))
        assert abs(ex - eref) <= 1e-12 * abs(eref)
        assert abs(dex - dref) <= 1e-12 * abs(dref)
