"""GPU parity of the split-bf16 tensor-core TTM (tcgen05) against the FP64 oracle TTM."""
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


# (P, K, S, R): several tiles, ragged s blocks, odd half-tile counts, K not a multiple of 64,
# R padded to 16 / 32, and the 400^3 mode-1 / mode-2 shapes.
SHAPES = [(1, 64, 128, 32), (3, 64, 64, 16), (2, 50, 72, 5), (5, 37, 8, 24), (7, 129, 200, 32), (1, 400, 4096, 32),
          (40, 48, 48, 16), (400, 400, 400, 32), (1, 400, 160000, 32), (3, 512, 136, 30)]
# S == 1 (the contracted mode is the contiguous one: K-major operand): one row, a ragged last
# 128-row tile, K a multiple of 8 but not of 64, R padded to 16 / 32, K at its 512 maximum,
# and the 400^3 R = 32 deeper-level shape
SHAPES_KMAJOR = [(1, 64, 1, 8), (1000, 400, 1, 32), (130, 48, 1, 24), (77, 72, 1, 16), (128, 512, 1, 32),
                 (12800, 400, 1, 32)]


@pytest.mark.parametrize("P,K,S,R", SHAPES + SHAPES_KMAJOR)
def test_ttm_split_bf16_tensor_cores(P, K, S, R):
    g = np.random.default_rng(P * 1000 + K + S + R)
    X = g.standard_normal((P, K, S)).astype(np.float32)
    Q, _ = np.linalg.qr(g.standard_normal((K, R)))
    ref = o.ttm_qt(X.astype(np.float64), Q, 1)
    Xd = torch.from_numpy(X).to(DEV)
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).to(DEV)
    out = torch.full(ref.shape, float("nan"), dtype=torch.float32, device=DEV)
    b.cpqr_ttm(Xd.data_ptr(), [P, K, S], 1, Qd.data_ptr(), R, out.data_ptr(), b.TTM_SPLIT_BF16)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all()
    # hi + lo keeps ~16 significant bits of each operand (all four products kept): per-term error
    # about 2^-16, summed with random signs over K terms, against outputs of size ~sqrt(K).
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < 2e-4, err


@pytest.mark.parametrize("P,K,S,R", [(300, 64, 1, 32), (130, 48, 1, 16), (5, 72, 40, 24)])
def test_ttm_output_at_an_odd_word_offset(P, K, S, R):
    """An output pointer that is 4 but not 8-byte aligned (a view into a larger buffer): the
    K-major epilogue then stores single columns instead of column pairs; results as the oracle."""
    g = np.random.default_rng(P + K + S + R)
    X = g.standard_normal((P, K, S)).astype(np.float32)
    Q, _ = np.linalg.qr(g.standard_normal((K, R)))
    ref = o.ttm_qt(X.astype(np.float64), Q, 1)
    Xd = torch.from_numpy(X).to(DEV)
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).to(DEV)
    buf = torch.full((ref.size + 1,), float("nan"), dtype=torch.float32, device=DEV)
    assert buf.data_ptr() % 8 == 0
    b.cpqr_ttm(Xd.data_ptr(), [P, K, S], 1, Qd.data_ptr(), R, buf.data_ptr() + 4, b.TTM_SPLIT_BF16)
    torch.cuda.synchronize()
    got = buf[1:].cpu().numpy().astype(np.float64).reshape(ref.shape)
    assert np.isfinite(got).all() and np.isnan(buf[0].item())
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 2e-4


@pytest.mark.parametrize("P,K,S", [(4096, 400, 1), (1, 400, 4096), (2048, 512, 1)])
def test_split_ttm_has_no_systematic_bias(P, K, S):
    """Positive X and Q (entries in [0.5, 1.5]), so every output is a sum of K positive terms: the
    mean signed relative error against FP64 shows any bias.  Tensor-core FP32 accumulation
    truncates toward zero (one accumulator for all K/16 x 4 MMAs gave -1.3e-6 at K = 400); with
    hi*hi split over two accumulators and the corrections in a third the mean stays below 1e-7,
    under the rms error of the bf16 hi + lo operands."""
    g = np.random.default_rng(K + S)
    X = g.uniform(0.5, 1.5, (P, K, S)).astype(np.float32)
    Q = g.uniform(0.5, 1.5, (K, 32))
    Xd, Qd = torch.from_numpy(X).to(DEV), torch.from_numpy(Q).to(DEV)
    out = torch.empty((P, 32, S), dtype=torch.float32, device=DEV)
    b.cpqr_ttm(Xd.data_ptr(), [P, K, S], 1, Qd.data_ptr(), 32, out.data_ptr(), b.TTM_SPLIT_BF16)
    ref = torch.einsum("pks,kr->prs", Xd.double(), Qd)
    rel = (out.double() - ref) / ref
    assert abs(rel.mean().item()) < 1e-7, rel.mean().item()
    assert rel.pow(2).mean().sqrt().item() < 5e-7


# wide ranks (the high-rank regime): MN-major and K-major, Rp = 48 .. 192, ragged tails, two
# accumulator buffers (Rp <= 128) and one (Rp > 128)
SHAPES_WIDE = [(1, 64, 200, 48), (3, 130, 72, 64), (2, 400, 136, 100), (1, 160, 1000, 150), (300, 200, 1, 150),
               (77, 200, 1, 192), (2, 200, 64, 176), (1000, 400, 1, 64)]


@pytest.mark.parametrize("P,K,S,R", SHAPES_WIDE)
def test_wide_split_ttm_matches_oracle(P, K, S, R):
    g = np.random.default_rng(P * 31 + K * 7 + S + R)
    X = g.standard_normal((P, K, S)).astype(np.float32)
    Q = np.linalg.qr(g.standard_normal((K, R)))[0]
    ref = o.ttm_qt(X.astype(np.float64), Q, 1)
    Xd, Qd = torch.from_numpy(X).to(DEV), torch.from_numpy(Q).to(DEV)
    out = torch.empty((P, R, S), dtype=torch.float32, device=DEV)
    b.cpqr_ttm(Xd.data_ptr(), [P, K, S], 1, Qd.data_ptr(), R, out.data_ptr(), b.TTM_SPLIT_BF16)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 2e-4
