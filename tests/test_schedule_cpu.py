"""The pair schedule (host-only ``fock_schedule``): the band-group split of the
pair loop (the paper's §5, Fig. 3) as the library draws it.  The shards are
contiguous runs of chains (two pairs per transform) of one fixed, band-blocked
order of the unique pairs i <= j; together they hold every pair once.  No GPU."""

import ctypes
import itertools

import numpy as np
import pytest

from paper_1305_7313_gb300 import _lib
from tests._common import built_library


@pytest.fixture(scope="module")
def lib():
    return built_library()


def all_pairs(nb):
    return {(i, j) for i in range(nb) for j in range(i, nb)}


@pytest.mark.parametrize("nb", [1, 2, 7, 33, 64])
@pytest.mark.parametrize("band_block", [0, 1, 4, 16, 40])
def test_shards_partition_the_unique_pairs_in_schedule_order(lib, nb, band_block):
    full = _lib.fock_schedule(nb, 0, 1, band_block)
    assert full.shape == (nb * (nb + 1) // 2, 2)
    assert {tuple(p) for p in full.tolist()} == all_pairs(nb)  # every pair once ...
    assert len({tuple(p) for p in full.tolist()}) == len(full)  # ... and no pair twice
    for nshards in (2, 3, 8, 100):
        parts = [_lib.fock_schedule(nb, s, nshards, band_block) for s in range(nshards)]
        assert np.array_equal(np.concatenate(parts), full)  # contiguous runs of one order
        chains = [(len(p) + 1) // 2 for p in parts]
        assert max(chains) - min(chains) <= 1  # balanced to one chain (two pairs)


@pytest.mark.parametrize("nb,band_block", [(37, 8), (64, 16), (20, 7)])
def test_order_is_band_blocked_with_block_rows_outer(lib, nb, band_block):
    full = _lib.fock_schedule(nb, 0, 1, band_block).tolist()
    blocks = [(i // band_block, j // band_block) for i, j in full]
    # block pairs (bi <= bj) are visited in row-major order, each in one run
    runs = [b for b, _ in itertools.groupby(blocks)]
    assert runs == sorted(runs) and len(runs) == len(set(runs))
    assert all(bi <= bj for bi, bj in runs)
    # inside a block, pairs go row by row (i outer, j inner)
    for b, grp in itertools.groupby(zip(blocks, full), key=lambda t: t[0]):
        ps = [p for _, p in grp]
        assert ps == sorted(ps)


def test_a_band_block_of_at_least_nb_is_the_plain_triangle(lib):
    nb = 9
    tri = [(i, j) for i in range(nb) for j in range(i, nb)]
    for bb in (9, 10, 1000):
        assert [tuple(p) for p in _lib.fock_schedule(nb, 0, 1, bb).tolist()] == tri


@pytest.mark.parametrize("nb,bb,shard,nshards", [(0, 0, 0, 1), (-3, 0, 0, 1), ((1 << 15) + 1, 0, 0, 1),
                                                 (5, -1, 0, 1), (5, 0, 1, 1), (5, 0, -1, 2), (5, 0, 0, 0)])
def test_bad_arguments_are_rejected(lib, nb, bb, shard, nshards):
    with pytest.raises(_lib.FockError):
        _lib.fock_schedule(nb, shard, nshards, bb)


def test_a_short_pairs_buffer_is_rejected(lib):
    n = ctypes.c_int64()
    out = np.empty((2, 2), dtype=np.int32)
    st = lib.fock_schedule(5, 0, 0, 1, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 2, ctypes.byref(n))
    assert _lib.STATUS[st] == "FOCK_ERR_INVALID_ARG"
