"""Failure detection without a GPU fault: a bounded device wait that runs out (a tile load that
nothing issues), and faults injected on the host (a NaN, a zero column).  Each must come back
as a status code, stay sticky in its context, and leave the GPU usable for the next context."""
import numpy as np
import pytest

from oracle import cpqr_oracle as o
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


def _problem(dtype=np.float32):
    # the first TTM contracts the last mode (K-major, K = 16): on the tensor cores
    return inputs.make_problem("fail", [24, 20, 16], 4, seed=21, c=0.3, eta=1e-3, dtype=dtype)


def _status(fn, *a):
    with pytest.raises(b.CpqrError) as e:
        fn(*a)
    return e.value.status


def test_tensor_core_wait_that_runs_out_is_reported_sticky_and_the_gpu_stays_usable():
    prob = _problem()
    X = torch.from_numpy(prob.X).to(DEV)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_NONE)
    d = b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts)
    b.cp_als_qr_test_wait_timeout(d.ctx, 1_000_000)  # 1 ms
    assert _status(d.sweep, 1) == b.ETIMEOUT
    # sticky: every later call reports the same status
    assert _status(d.sweep, 1) == b.ETIMEOUT
    assert _status(d.fit_exact) == b.ETIMEOUT
    assert _status(d.factors) == b.ETIMEOUT
    assert _status(d.fit, 1e-6, 5) == b.ETIMEOUT
    d.close()
    torch.cuda.synchronize()  # the context of the process is intact
    # a new context on the same tensor runs normally and tracks the oracle
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d2:
        fits = d2.sweep(3)
    ref = o.cp_als_qr(prob.X, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, extrapolate=False, max_sweeps=3)
    assert np.max(np.abs(fits - np.array(ref.fits))) <= 1e-4


def test_wait_timeout_hook_needs_a_tensor_core_context():
    prob = _problem(np.float64)
    X = torch.from_numpy(prob.X).to(DEV)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=b.EXTRAP_NONE)
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), True, prob.A0, opts) as d:
        assert _status(b.cp_als_qr_test_wait_timeout, d.ctx, 1000) == b.EUNSUPPORTED
        d.sweep(1)  # a refused hook leaves the context as it was


@pytest.mark.parametrize("where", ["A0", "X"])
def test_nan_input_gives_enonfinite(where):
    prob = _problem(np.float64)
    Xh = prob.X.copy()
    A0 = [a.copy() for a in prob.A0]
    if where == "A0":
        A0[1][3, 2] = np.nan
    else:
        Xh[5, 6, 7] = np.inf
    X = torch.from_numpy(Xh).to(DEV)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=b.EXTRAP_PAPER)
    assert _status(b.Decomposition, prob.dims, prob.R, X.data_ptr(), True, A0, opts) == b.ENONFINITE


def test_zero_column_in_starting_factor_gives_esingular():
    prob = _problem(np.float64)
    A0 = [a.copy() for a in prob.A0]
    A0[2][:, 1] = 0.0
    X = torch.from_numpy(prob.X).to(DEV)
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_FP64, extrap=b.EXTRAP_PAPER)
    assert _status(b.Decomposition, prob.dims, prob.R, X.data_ptr(), True, A0, opts) == b.ESINGULAR
    # the same problem without the zero column runs
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), True, prob.A0, opts) as d:
        assert np.all(np.isfinite(d.sweep(2)))
