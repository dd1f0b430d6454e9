"""cpqr_house_qr_noalloc — the QR entry point for callers that may not allocate device
memory (their scratch lives in one static device array) — against cpqr_house_qr, which
allocates its scratch per call, and against the oracle's Householder QR.  Collected last on
purpose."""
import numpy as np
import pytest

from oracle import cpqr_oracle as o
from paper_2503_18759_gb300 import binding as b

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_18759_gb300 import build
    build.build()
    b.lib()


def _qr(fn, A):
    M, R = A.shape
    Ad = torch.from_numpy(A).to(DEV)
    Q = torch.empty((M, R), dtype=torch.float64, device=DEV)
    Rm = torch.empty((R, R), dtype=torch.float64, device=DEV)
    fn(Ad.data_ptr(), M, R, Q.data_ptr(), Rm.data_ptr())
    torch.cuda.synchronize()
    return Q.cpu().numpy(), Rm.cpu().numpy()


# 400 x 32: the rows fit in the cluster's shared memory, the scratch holds the status word;
# 16384 x 32: the working rows themselves live in the scratch array.
@pytest.mark.parametrize("M,R", [(400, 32), (16384, 32)])
def test_noalloc_qr_matches_allocating_qr_on_two_calls_in_a_row(M, R):
    g = np.random.default_rng(M + R)
    for call in range(2):
        A = g.standard_normal((M, R))
        Qa, Ra = _qr(b.cpqr_house_qr, A)
        Qn, Rn = _qr(b.cpqr_house_qr_noalloc, A)
        assert np.allclose(Rn, Ra, rtol=0, atol=1e-12 * np.linalg.norm(A)), call
        assert np.allclose(Qn, Qa, rtol=0, atol=1e-12), call
        assert np.allclose(Qn @ Rn, A, atol=1e-11 * np.linalg.norm(A))
        Qo, Ro = o.householder_qr(A)
        assert np.allclose(Rn, Ro, rtol=0, atol=1e-12 * np.linalg.norm(A)), call
        assert np.allclose(Qn, Qo, rtol=0, atol=1e-12), call


@pytest.mark.parametrize("fn", ["cpqr_house_qr_noalloc", "cpqr_house_qr"])
def test_zero_column_reports_singular(fn):
    """A zero column has no Householder reflector (zero norm): the device flags it and the entry
    point returns CPQR_ESINGULAR instead of a silent success; the next call is unaffected."""
    g = np.random.default_rng(5)
    A = g.standard_normal((300, 8))
    A[:, 3] = 0.0
    with pytest.raises(b.CpqrError) as e:
        _qr(getattr(b, fn), A)
    assert e.value.status == b.ESINGULAR
    A[:, 3] = g.standard_normal(300)
    Q, Rm = _qr(getattr(b, fn), A)
    Qo, Ro = o.householder_qr(A)
    assert np.allclose(Rm, Ro, atol=1e-12 * np.linalg.norm(A))


def test_noalloc_qr_rejects_sizes_beyond_its_scratch():
    M, R = b.NOALLOC_QR_MAX_ELEMS // 32 + 1, 32
    with pytest.raises(b.CpqrError) as e:
        b.cpqr_house_qr_noalloc(1, M, R, 1, 1)
    assert e.value.status == 1
