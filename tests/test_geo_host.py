"""The pair passes' launch geometry (``Geo`` in ``csrc/fock_kernels.cuh``),
printed by a host program that nvcc compiles from the kernels' header, against
the constraints its launches rely on (CPU; no GPU needed):

* CTA sizes are whole warps, hold every (line, sub-thread) of their pass and
  stay within 1024 threads;
* dynamic shared memory stays within the 227 KB a CTA may have (sm_103);
* the column pass takes at most a row's width of lines a CTA, and where it
  takes fewer, about half as many in multiples of 8 (whole warps at 4 and 8
  threads a line);
* at least two column-pass CTAs fit an SM's shared memory (233,472 B, 1 KB
  reserved per CTA), so that one's barriers overlap another's work;
* a launch-bound minimum of CTAs per SM is one the SM can honour: its CTAs
  fit the shared memory, and each thread keeps at least 64 registers.
"""

import subprocess

import pytest

from tests._common import host_program

SMEM_PER_SM = 233472
SMEM_PER_CTA = 232448
RESERVED = 1024


@pytest.fixture(scope="module")
def rows(tmp_path_factory):
    exe = host_program("geo_host_driver.cu", tmp_path_factory.mktemp("geo_host"),
                       extra=("-gencode", "arch=compute_103a,code=sm_103a"))
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    keys = ("type", "N", "tile", "NC", "NLC", "TLC", "THR_COL", "THR_COLH", "SMEM_COLH", "MIN_CTAS_COL",
            "SMEM_PLANE", "SMEM_INV", "THR_PLANE", "MIN_CTAS", "cbytes")
    parsed = [dict(zip(keys, (int(v) for v in line.split()))) for line in out.splitlines()]
    assert parsed
    return parsed


def test_every_compiled_size_type_and_tiling_is_listed(rows):
    sizes = {8, 12, 16, 24, 32, 36, 48, 64, 72, 96}
    for t in (0, 1, 2):
        assert {r["N"] for r in rows if r["type"] == t and r["tile"] == 0} == sizes
    # the second tilings at 96^3 the tuner picks between
    assert any(r["type"] == 0 and r["N"] == 96 and r["tile"] == 1 for r in rows)
    assert any(r["type"] == 1 and r["N"] == 96 and r["tile"] == 1 for r in rows)


def test_cta_sizes_are_whole_warps_holding_every_line(rows):
    for r in rows:
        assert r["THR_COL"] % 32 == 0 and r["THR_COLH"] % 32 == 0 and r["THR_PLANE"] % 32 == 0, r
        assert r["NLC"] * r["TLC"] <= r["THR_COL"] < r["NLC"] * r["TLC"] + 32, r
        assert r["NC"] * r["TLC"] <= r["THR_COLH"] < r["NC"] * r["TLC"] + 32, r
        assert max(r["THR_COL"], r["THR_COLH"], r["THR_PLANE"]) <= 1024, r


def test_shared_memory_fits_a_cta(rows):
    for r in rows:
        assert max(r["SMEM_COLH"], r["SMEM_PLANE"], r["SMEM_INV"]) <= SMEM_PER_CTA, r


def test_column_lines_a_cta(rows):
    for r in rows:
        assert r["NC"] == 2 * (r["N"] // 2 + 1)
        assert 1 <= r["NLC"] <= r["NC"], r
        if r["NLC"] < r["NC"]:
            assert r["NLC"] % 8 == 0 and r["NC"] // 2 <= r["NLC"] < r["NC"] // 2 + 8, r
    # at 96^3 every form takes about half a row's width (two FP64 or
    # double-float CTAs, four FP32 ones, an SM)
    assert all(r["NLC"] == 56 for r in rows if r["N"] == 96)


def test_two_column_ctas_fit_an_sm(rows):
    for r in rows:
        assert SMEM_PER_SM // (r["SMEM_COLH"] + RESERVED) >= 2, r


def test_launch_bound_minimums_can_be_honoured(rows):
    for r in rows:
        for thr, m, smem in ((r["THR_COL"], r["MIN_CTAS_COL"], r["SMEM_COLH"]),
                             (r["THR_COLH"], r["MIN_CTAS"], r["SMEM_INV"])):
            assert m >= 1, r
            if m > 1:
                assert m * (smem + RESERVED) <= SMEM_PER_SM, r
                assert 65536 // (m * thr) >= 64, r
