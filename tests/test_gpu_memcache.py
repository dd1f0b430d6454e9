"""The library's device block cache: contexts that reuse blocks a destroyed context left (holding
that context's data) give bit-identical results, and releasing the cache leaves the library
usable."""
import numpy as np
import pytest

from paper_2503_18759_gb300 import binding as b
from paper_2503_18759_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_18759_gb300 import build
    build.build()
    b.lib()


def _run(prob, sweeps=6):
    X = torch.from_numpy(np.ascontiguousarray(prob.X)).to(DEV)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_PAPER)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        fits = d.sweep(sweeps)
        A, lam, _, _ = d.factors()
    return fits, A, lam


@pytest.mark.parametrize("dims,R", [([40, 36, 48], 8), ([20, 18, 16, 24], 6)])
def test_reused_blocks_give_identical_results(dims, R):
    """Run, run another tensor of the same shape (its context takes the first one's blocks and
    leaves its own data in them), run the first again: identical fits and factors, also after
    the cache is released."""
    p1 = inputs.make_problem("cache1", dims, R, seed=21, c=0.5, eta=1e-3, dtype=np.float32)
    p2 = inputs.make_problem("cache2", dims, R, seed=22, c=0.3, eta=1e-2, dtype=np.float32)
    f1, A1, l1 = _run(p1)
    f2, _, _ = _run(p2)
    assert not np.array_equal(f1, f2)
    g1, B1, m1 = _run(p1)
    assert np.array_equal(f1, g1)
    for a, c in zip(A1, B1):
        assert np.array_equal(a, c)
    assert np.array_equal(l1, m1)
    b.cpqr_release_cached_memory()
    h1, C1, n1 = _run(p1)
    assert np.array_equal(f1, h1)
    for a, c in zip(A1, C1):
        assert np.array_equal(a, c)
    b.cpqr_release_cached_memory()


def test_run_host_twice_matches_context_path():
    """cp_als_qr_run_host called twice (the second call served by the cache) returns the factors of
    the context path."""
    prob = inputs.make_problem("cache_rh", [32, 28, 24], 5, seed=23, c=0.4, eta=1e-3, dtype=np.float32)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_PAPER)
    outs = [b.cp_als_qr_run_host(prob.dims, prob.R, prob.X, prob.A0, opts, tol=0.0, max_sweeps=5) for _ in range(2)]
    fits, A, lam = _run(prob, sweeps=5)
    for got in outs:
        for a, c in zip(got[0], A):
            assert np.array_equal(a, c)
        assert np.array_equal(got[1], lam)
        assert abs(got[2] - fits[-1]) <= 1e-12
