"""The float-float arithmetic and the square-root-free pipelined Cholesky of csrc/krp_gram.cu,
restated on the host with bit-faithful FP32 rounding (numpy float32; an FMA is the float64
product of two float32 values, which is exact, plus the addend, rounded once to float32).

The kernel's Cholesky factor R1 only preconditions Q1 = Z R1^{-1}, formed in FP64, and the
guard accepts the Gram-route QR when E = Q1^T Q1 - I stays below 1e-8.  These tests pin what
that design relies on: R1 agrees with the FP64 Cholesky to the float-float precision (~2^-46),
E stays near kappa^2 * 1e-16 on the method's collinear factors, and plain FP32 would not do."""
import numpy as np
import pytest

f32 = np.float32


def _fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _mul(a, b):
    p = f32(a[0] * b[0])
    e = _fma(a[0], b[0], -p)
    e = _fma(a[0], b[1], e)
    e = _fma(a[1], b[0], e)
    h = f32(p + e)
    return (h, f32(e - f32(h - p)))


def _fms(t, a, b):  # t - a b
    p = f32(a[0] * b[0])
    pe = _fma(a[0], b[0], -p)
    pe = _fma(a[0], b[1], pe)
    pe = _fma(a[1], b[0], pe)
    s = f32(t[0] - p)
    bb = f32(s - t[0])
    err = f32(f32(t[0] - f32(s - bb)) + f32(-p - bb))
    err = f32(err + f32(t[1] - pe))
    h = f32(s + err)
    return (h, f32(err - f32(h - s)))


def _recip(d):
    y = f32(1.0) / d[0]
    p = f32(d[0] * y)
    pe = _fma(d[0], y, -p)
    pe = _fma(d[1], y, pe)
    r = f32(f32(f32(1.0) - p) - pe)
    c = f32(y * r)
    h = f32(y + c)
    return (h, f32(c - f32(h - y)))


def _split(x):
    h = f32(x)
    return (h, f32(x - np.float64(h)))


def _val(a):
    return np.float64(a[0]) + np.float64(a[1])


def chol_float_float(G):
    """Square-root-free Cholesky in the kernel's order: warp 0 finishes row j by applying step
    j - 1 to the copy of row j it prepared one iteration earlier (that copy got step j - 2 from
    warp 0 and the steps before from the other warps), z = U[j-1][j] U[j-1]; the other warps
    apply step s to rows >= s + 3."""
    R = G.shape[0]
    zero = (f32(0), f32(0))
    T = [[_split(G[i, j]) for j in range(R)] for i in range(R)]
    U = [[zero] * R for _ in range(R)]
    V = [[zero] * R for _ in range(R)]

    def trailing(s):
        for k in range(s + 3, R):
            for l in range(k, R):
                T[k][l] = _fms(T[k][l], V[s][k], U[s][l])

    def pick(row, l):
        return row[l] if l < R else zero

    u = [T[0][l] for l in range(R)]
    nxt = [T[1][l] if (R > 1 and l >= 1) else zero for l in range(R)]
    w = _recip(u[0])
    z = [_mul(pick(u, 1), u[l]) for l in range(R)]
    z2 = [_mul(pick(u, 2), u[l]) for l in range(R)]
    U[0], V[0] = u[:], [_mul(u[l], w) for l in range(R)]
    for j in range(1, R):
        u = [_fms(nxt[l], w, z[l]) if l >= j else zero for l in range(R)]
        if j >= 2:
            trailing(j - 2)
        t = [T[j + 1][l] if (j + 1 < R and l >= j + 1) else zero for l in range(R)]
        w1, z21 = w, z2
        w = _recip(u[j])
        z = [_mul(pick(u, j + 1), u[l]) for l in range(R)]
        z2 = [_mul(pick(u, j + 2), u[l]) for l in range(R)]
        nxt = [_fms(t[l], w1, z21[l]) if (j + 1 < R and l >= j + 1) else zero for l in range(R)]
        U[j], V[j] = u[:], [_mul(u[l], w) if l >= j else zero for l in range(R)]
    Ud = np.array([[_val(U[i][j]) for j in range(R)] for i in range(R)])
    return np.triu(Ud / np.sqrt(np.diag(Ud))[:, None])


def _collinear(I, R, c, seed):
    g = np.random.default_rng(seed)
    A = g.standard_normal((I, R)) * np.sqrt(1 - c) + np.sqrt(c) * g.standard_normal((I, 1))
    return A / np.linalg.norm(A, axis=0)


@pytest.mark.parametrize("R,c", [(5, 0.3), (16, 0.9), (32, 0.9), (32, 0.99)])
def test_float_float_cholesky_preconditions_to_the_guard(R, c):
    A = _collinear(400, R, c, seed=R)
    G = A.T @ A
    R1 = chol_float_float(G)
    ref = np.linalg.cholesky(G).T
    kappa = np.linalg.cond(A)
    assert np.abs(R1 - ref).max() <= 2e-13 * np.abs(ref).max()
    Q1 = np.linalg.solve(R1.T, A.T).T
    E = np.abs(Q1.T @ Q1 - np.eye(R)).max()
    assert E <= 1e-15 * kappa ** 2 + 1e-14
    assert E <= 1e-8  # the guard accepts: first-order correction leaves O(E^2)


def test_plain_fp32_cholesky_would_trip_the_guard():
    A = _collinear(400, 16, 0.9, seed=3)
    G = (A.T @ A).astype(np.float32)
    R1 = np.linalg.cholesky(G.astype(np.float64)).T.astype(np.float32).astype(np.float64)
    Q1 = np.linalg.solve(R1.T, A.T).T
    assert np.abs(Q1.T @ Q1 - np.eye(16)).max() > 1e-8
