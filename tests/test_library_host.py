"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every entry point the header declares, and its TTM schedule is the oracle's."""
import os
import re

import numpy as np
import pytest

from oracle import cpqr_oracle as o
from paper_2503_18759_gb300 import binding as b
from paper_2503_18759_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "cpqr.h")


@pytest.fixture(scope="module")
def L():
    build.build()
    return b.lib()


def test_library_exports_every_declared_symbol(L):
    text = open(HEADER).read()
    names = re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(c[pq][a-z_0-9]+)\s*\(", text, flags=re.M)
    assert "cp_als_qr_init" in names and "cpqr_ttm" in names
    for n in names:
        assert hasattr(L, n), n


def test_strerror_and_options(L):
    assert b.cp_als_qr_strerror(0) == "ok"
    assert "invalid" in b.cp_als_qr_strerror(1)
    o_ = b.cp_als_qr_default_options()
    assert o_.tree == b.TREE_RESTRUCTURED and o_.prec == b.PREC_FP64 and o_.extrap == b.EXTRAP_PAPER
    assert o_.alpha == pytest.approx(0.1)


def test_init_rejects_bad_arguments_without_a_gpu(L):
    with pytest.raises(b.CpqrError) as e:
        b.cp_als_qr_init([10, 10], 3, 1, False)  # order 2
    assert e.value.status == 1
    with pytest.raises(b.CpqrError):
        b.cp_als_qr_init([10, 10, 2], 3, 1, False)  # R > I_n
    with pytest.raises(b.CpqrError):
        b.cp_als_qr_init([10, 10, 10], 33, 1, False)  # R > 32


def _oracle_ops(dims, R, tree, sweeps):
    return np.array(o.schedule_ops(dims, R, tree, sweeps), dtype=np.int32).reshape(-1, 4)


@pytest.mark.parametrize("tree", [0, 1, 2])
@pytest.mark.parametrize("dims,R", [((400, 400, 400), 32), ((5, 7, 11), 3), ((128,) * 4, 24), ((5, 7, 11, 13), 3),
                                    ((48,) * 5, 16), ((9, 4, 7, 5, 6), 3), ((60, 60, 60), 5), ((10, 30, 20), 4),
                                    ((25,) * 6, 8), ((5, 4, 6, 3, 5, 4), 2)])
def test_schedule_identical_to_oracle(L, tree, dims, R):
    sweeps = 9
    ops, flops = b.cp_als_qr_schedule(dims, R, tree, sweeps)
    ref = _oracle_ops(dims, R, tree, sweeps)
    assert ops.shape == ref.shape
    assert np.array_equal(ops, ref)
    s = o.Schedule(dims, R, tree)
    for _ in range(sweeps):
        s.next_sweep()
    assert flops == s.flops


def test_history_jsonl_lines_round_trip():
    """Per-sweep metrics lines: one JSON object per sweep, 1-based sweep index, the extra keys on
    every line, values that read back exactly."""
    import json
    fits = np.array([0.5, 0.75, 0.875])
    betas = np.array([0.0, 0.004, 0.004])
    lines = b.history_jsonl_lines(fits, betas, workload="w", ms_per_sweep_timed_avg=0.25)
    assert len(lines) == 3
    recs = [json.loads(ln) for ln in lines]
    assert [r["sweep"] for r in recs] == [1, 2, 3]
    assert [r["fit"] for r in recs] == list(fits)
    assert [r["beta"] for r in recs] == list(betas)
    assert all(r["workload"] == "w" and r["ms_per_sweep_timed_avg"] == 0.25 for r in recs)
    assert b.history_jsonl_lines([], []) == []


def test_release_cached_memory_without_a_gpu(L):
    """Releasing the block cache succeeds; with nothing cached (as on a machine without a GPU) it
    frees nothing."""
    assert L.cpqr_release_cached_memory() == b.OK
