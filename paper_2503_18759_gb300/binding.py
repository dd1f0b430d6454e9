"""ctypes binding of libcpqr.so: the C ABI of include/cpqr.h with the same names.

Argument marshalling only: every step of the decomposition runs in the CUDA
library.  Device buffers are passed as integer addresses (e.g. a torch
tensor's ``data_ptr()``), host buffers as numpy arrays.  A missing library or
a non-OK status raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpqr.so")

TREE_NONE, TREE_STANDARD, TREE_RESTRUCTURED = 0, 1, 2
PREC_FP64, PREC_SPLIT_BF16 = 0, 1
EXTRAP_NONE, EXTRAP_PAPER, EXTRAP_FIXED, EXTRAP_LEARNED = 0, 1, 2, 3
QR_GRAM, QR_HOUSEHOLDER = 0, 1
TTM_F64, TTM_F32, TTM_F32_IN_F64, TTM_SPLIT_BF16 = 0, 1, 2, 3

OK, EINVAL, ENOMEM, ECUDA, ESINGULAR, ENONFINITE, ETIMEOUT, ENOTCONV, EUNSUPPORTED = 0, 1, 2, 3, 4, 5, 6, 7, 8


class CpqrError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {cp_als_qr_strerror(status)} (status {status})")
        self.status = status


class Options(C.Structure):
    _fields_ = [("tree", C.c_int32), ("prec", C.c_int32), ("extrap", C.c_int32), ("qr_route", C.c_int32),
                ("alpha", C.c_double), ("beta_fixed", C.c_double), ("seed", C.c_uint64),
                ("mlp_weights", C.POINTER(C.c_float))]


NBUCKETS = 7
BUCKETS = ("ttm_full", "ttm_deep", "q0", "apply_q0", "qr", "other", "fit")


class Stats(C.Structure):
    _fields_ = [("sweeps", C.c_int64), ("ttm_flops", C.c_int64), ("full_ttms", C.c_int64),
                ("last_fit", C.c_double), ("beta", C.c_double), ("proposals", C.c_int64),
                ("accepted", C.c_int64), ("launches", C.c_int64), ("ms_bucket", C.c_double * NBUCKETS),
                ("n_bucket", C.c_int64 * NBUCKETS), ("qr_fallbacks", C.c_int64),
                ("krp_split", C.c_int64), ("judged", C.c_int64), ("preapproved", C.c_int64),
                ("deferred", C.c_int64), ("qr_second_pass", C.c_int64), ("lagged_fits", C.c_int64)]


_lib = None


def lib() -> C.CDLL:
    """Load libcpqr.so (built in-tree); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2503_18759_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    P = C.POINTER
    L.cp_als_qr_default_options.argtypes = [P(Options)]
    L.cp_als_qr_default_options.restype = None
    L.cp_als_qr_init.argtypes = [P(vp), i32, P(i64), i32, vp, i32, P(P(dbl)), P(Options), vp]
    L.cp_als_qr_sweep.argtypes = [vp, i32, P(dbl)]
    L.cp_als_qr_fit.argtypes = [vp, dbl, i32, P(dbl), P(i32)]
    L.cp_als_qr_get.argtypes = [vp, i32, P(dbl), P(dbl), P(dbl), P(dbl)]
    L.cp_als_qr_stats.argtypes = [vp, P(Stats)]
    L.cp_als_qr_fit_exact.argtypes = [vp, P(dbl)]
    L.cp_als_qr_set_timing.argtypes = [vp, i32]
    L.cp_als_qr_destroy.argtypes = [vp]
    L.cp_als_qr_destroy.restype = None
    L.cpqr_release_cached_memory.argtypes = []
    L.cp_als_qr_strerror.argtypes = [i32]
    L.cp_als_qr_strerror.restype = C.c_char_p
    L.cp_als_qr_schedule.argtypes = [i32, P(i64), i32, i32, i32, P(i32), i64, P(i64), P(i64)]
    L.cp_als_qr_run_host.argtypes = [i32, P(i64), i32, vp, i32, P(P(dbl)), P(Options), dbl, i32, P(P(dbl)),
                                     P(dbl), P(dbl), P(i32), vp]
    L.cpqr_ttm.argtypes = [vp, i32, P(i64), i32, vp, i32, vp, i32, vp]
    L.cp_als_qr_mlp_beta.argtypes = [i32]
    L.cp_als_qr_mlp_beta.restype = dbl
    L.cpqr_mlp_features.argtypes = [P(dbl), P(dbl), i32, dbl, i32, P(C.c_float)]
    L.cpqr_mlp_work_bytes.argtypes = [i32]
    L.cpqr_mlp_work_bytes.restype = i64
    L.cpqr_mlp_forward.argtypes = [vp, vp, i32, vp, vp, vp]
    L.cpqr_mlp_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
    L.cpqr_mlp_adam.argtypes = [vp, vp, vp, vp, C.c_float, i32, vp]
    L.cp_als_qr_checkpoint.argtypes = [vp]
    L.cp_als_qr_rollback.argtypes = [vp]
    L.cp_als_qr_commit.argtypes = [vp]
    L.cp_als_qr_sweep_beta.argtypes = [vp, dbl, P(dbl)]
    L.cp_als_qr_test_wait_timeout.argtypes = [vp, C.c_uint64]
    L.cp_als_qr_mlp_state.argtypes = [vp, P(C.c_float), P(C.c_float), P(i32)]
    L.cp_als_qr_history.argtypes = [vp, P(dbl), P(dbl), i32, P(i32), P(dbl), P(i32)]
    L.cpqr_house_qr.argtypes = [vp, i64, i32, vp, vp, vp]
    L.cpqr_krp_qr.argtypes = [vp, i32, i32, vp, vp, vp]
    L.cpqr_house_qr_noalloc.argtypes = [vp, i64, i32, vp, vp, vp]
    for name in ("cp_als_qr_init", "cp_als_qr_sweep", "cp_als_qr_fit", "cp_als_qr_get", "cp_als_qr_stats",
                 "cp_als_qr_fit_exact", "cp_als_qr_set_timing", "cp_als_qr_schedule", "cp_als_qr_run_host",
                 "cpqr_mlp_features", "cpqr_mlp_forward", "cpqr_mlp_grad", "cpqr_mlp_adam", "cp_als_qr_checkpoint",
                 "cp_als_qr_rollback", "cp_als_qr_commit", "cp_als_qr_sweep_beta", "cp_als_qr_test_wait_timeout", "cp_als_qr_mlp_state", "cp_als_qr_history", "cpqr_ttm", "cpqr_house_qr", "cpqr_krp_qr", "cpqr_house_qr_noalloc"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def _check(status: int, where: str, allow=(OK,)) -> int:
    if status not in allow:
        raise CpqrError(status, where)
    return status


def _i64(seq) -> C.Array:
    return (C.c_int64 * len(seq))(*[int(v) for v in seq])


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def cp_als_qr_strerror(status: int) -> str:
    return lib().cp_als_qr_strerror(int(status)).decode()


def cpqr_release_cached_memory() -> None:
    """Free the device and pinned blocks that destroyed contexts left in the library's cache."""
    _check(lib().cpqr_release_cached_memory(), "cpqr_release_cached_memory")


def cp_als_qr_default_options() -> Options:
    o = Options()
    lib().cp_als_qr_default_options(C.byref(o))
    return o


def make_options(tree=TREE_RESTRUCTURED, prec=PREC_FP64, extrap=EXTRAP_PAPER, alpha=0.1, beta_fixed=0.0,
                 seed=0, mlp_weights: Optional[np.ndarray] = None, qr_route=QR_GRAM) -> Options:
    o = cp_als_qr_default_options()
    o.tree, o.prec, o.extrap, o.qr_route = int(tree), int(prec), int(extrap), int(qr_route)
    o.alpha, o.beta_fixed, o.seed = float(alpha), float(beta_fixed), int(seed)
    if mlp_weights is not None:
        w = np.ascontiguousarray(mlp_weights, dtype=np.float32)
        o._keep = w  # keep alive while the struct is used
        o.mlp_weights = w.ctypes.data_as(C.POINTER(C.c_float))
    return o


def cp_als_qr_init(dims: Sequence[int], R: int, X_dev: int, x_is_fp64: bool,
                   A0: Optional[Sequence[np.ndarray]] = None, options: Optional[Options] = None,
                   stream: int = 0) -> C.c_void_p:
    ctx = C.c_void_p()
    N = len(dims)
    a0 = None
    keep = []
    if A0 is not None:
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in A0]
        keep = arrs
        a0 = (C.POINTER(C.c_double) * N)(*[_dptr(a) for a in arrs])
    st = lib().cp_als_qr_init(C.byref(ctx), N, _i64(dims), int(R), C.c_void_p(int(X_dev)), int(bool(x_is_fp64)),
                              a0, C.byref(options) if options is not None else None, C.c_void_p(int(stream)))
    del keep
    _check(st, "cp_als_qr_init")
    return ctx


def cp_als_qr_sweep(ctx, nsweeps: int) -> np.ndarray:
    fits = np.zeros(max(int(nsweeps), 1))
    _check(lib().cp_als_qr_sweep(ctx, int(nsweeps), _dptr(fits)), "cp_als_qr_sweep")
    return fits[:nsweeps]


def cp_als_qr_fit(ctx, tol: float, max_sweeps: int) -> Tuple[bool, float, int]:
    f = C.c_double()
    n = C.c_int32()
    st = _check(lib().cp_als_qr_fit(ctx, float(tol), int(max_sweeps), C.byref(f), C.byref(n)), "cp_als_qr_fit",
                allow=(OK, ENOTCONV))
    return st == OK, f.value, n.value


def cp_als_qr_get(ctx, n: int, I: int, R: int):
    A = np.zeros((I, R))
    lam = np.zeros(R)
    Q = np.zeros((I, R))
    Rn = np.zeros((R, R))
    _check(lib().cp_als_qr_get(ctx, int(n), _dptr(A), _dptr(lam), _dptr(Q), _dptr(Rn)), "cp_als_qr_get")
    return A, lam, Q, Rn


def cp_als_qr_stats(ctx) -> Stats:
    s = Stats()
    _check(lib().cp_als_qr_stats(ctx, C.byref(s)), "cp_als_qr_stats")
    return s


def cp_als_qr_fit_exact(ctx) -> float:
    f = C.c_double()
    _check(lib().cp_als_qr_fit_exact(ctx, C.byref(f)), "cp_als_qr_fit_exact")
    return f.value


def cp_als_qr_set_timing(ctx, on: bool) -> None:
    _check(lib().cp_als_qr_set_timing(ctx, int(bool(on))), "cp_als_qr_set_timing")


def cp_als_qr_run_host(dims: Sequence[int], R: int, X_host: np.ndarray, A0=None, options: Optional[Options] = None,
                       tol: float = 1e-6, max_sweeps: int = 100, stream: int = 0):
    """Host tensor in, host factors out (copies inside the call).  Returns (A list, lambda,
    final_fit, sweeps, converged)."""
    X_host = np.ascontiguousarray(X_host)
    x64 = X_host.dtype == np.float64
    N = len(dims)
    a0 = None
    keep = []
    if A0 is not None:
        keep = [np.ascontiguousarray(a, dtype=np.float64) for a in A0]
        a0 = (C.POINTER(C.c_double) * N)(*[_dptr(a) for a in keep])
    outs = [np.zeros((int(d), int(R))) for d in dims]
    aout = (C.POINTER(C.c_double) * N)(*[_dptr(a) for a in outs])
    lam = np.zeros(int(R))
    f = C.c_double()
    ns = C.c_int32()
    st = lib().cp_als_qr_run_host(N, _i64(dims), int(R), C.c_void_p(X_host.ctypes.data), int(x64), a0,
                                  C.byref(options) if options is not None else None, float(tol), int(max_sweeps),
                                  aout, _dptr(lam), C.byref(f), C.byref(ns), C.c_void_p(int(stream)))
    _check(st, "cp_als_qr_run_host", allow=(OK, ENOTCONV))
    return outs, lam, f.value, ns.value, st == OK


MLP_FEATURES, MLP_HIDDEN, MLP_CLASSES = 32, 128, 8
MLP_NPARAMS = 32 * 128 + 128 + 2 * (128 * 128 + 128) + 128 * 8 + 8


def cp_als_qr_mlp_beta(c: int) -> float:
    return lib().cp_als_qr_mlp_beta(int(c))


def cpqr_mlp_features(fits, betas, rule_beta: float, activated: bool) -> np.ndarray:
    f = np.ascontiguousarray(fits, dtype=np.float64)
    bt = np.ascontiguousarray(betas, dtype=np.float64)
    out = np.zeros(MLP_FEATURES, dtype=np.float32)
    _check(lib().cpqr_mlp_features(_dptr(f), _dptr(bt), len(f), float(rule_beta), int(bool(activated)),
                                   out.ctypes.data_as(C.POINTER(C.c_float))), "cpqr_mlp_features")
    return out


def cpqr_mlp_work_bytes(B: int) -> int:
    return int(lib().cpqr_mlp_work_bytes(int(B)))


def cpqr_mlp_forward(params_dev: int, X_dev: int, B: int, logits_dev: int, work_dev: int, stream: int = 0) -> None:
    _check(lib().cpqr_mlp_forward(C.c_void_p(params_dev), C.c_void_p(X_dev), int(B), C.c_void_p(logits_dev),
                                  C.c_void_p(work_dev), C.c_void_p(stream)), "cpqr_mlp_forward")


def cpqr_mlp_grad(params_dev: int, X_dev: int, y_dev: int, B: int, grad_dev: int, loss_dev: int, work_dev: int,
                  stream: int = 0) -> None:
    _check(lib().cpqr_mlp_grad(C.c_void_p(params_dev), C.c_void_p(X_dev), C.c_void_p(y_dev), int(B),
                               C.c_void_p(grad_dev), C.c_void_p(loss_dev), C.c_void_p(work_dev), C.c_void_p(stream)),
           "cpqr_mlp_grad")


def cpqr_mlp_adam(params_dev: int, m_dev: int, v_dev: int, grad_dev: int, lr: float, step: int,
                  stream: int = 0) -> None:
    _check(lib().cpqr_mlp_adam(C.c_void_p(params_dev), C.c_void_p(m_dev), C.c_void_p(v_dev), C.c_void_p(grad_dev),
                               float(lr), int(step), C.c_void_p(stream)), "cpqr_mlp_adam")


def cp_als_qr_checkpoint(ctx) -> None:
    _check(lib().cp_als_qr_checkpoint(ctx), "cp_als_qr_checkpoint")


def cp_als_qr_rollback(ctx) -> None:
    _check(lib().cp_als_qr_rollback(ctx), "cp_als_qr_rollback")


def cp_als_qr_commit(ctx) -> None:
    _check(lib().cp_als_qr_commit(ctx), "cp_als_qr_commit")


def cp_als_qr_sweep_beta(ctx, beta: float) -> float:
    f = C.c_double()
    _check(lib().cp_als_qr_sweep_beta(ctx, float(beta), C.byref(f)), "cp_als_qr_sweep_beta")
    return f.value


def cp_als_qr_mlp_state(ctx):
    """(features, logits, proposed class) of a learned context's device proposer."""
    f = np.zeros(MLP_FEATURES, dtype=np.float32)
    lg = np.zeros(MLP_CLASSES, dtype=np.float32)
    c = C.c_int32()
    _check(lib().cp_als_qr_mlp_state(ctx, f.ctypes.data_as(C.POINTER(C.c_float)),
                                     lg.ctypes.data_as(C.POINTER(C.c_float)), C.byref(c)), "cp_als_qr_mlp_state")
    return f, lg, c.value


def cp_als_qr_test_wait_timeout(ctx, limit_ns: int) -> None:
    _check(lib().cp_als_qr_test_wait_timeout(ctx, int(limit_ns)), "cp_als_qr_test_wait_timeout")


def cp_als_qr_history(ctx, cap: int = 100000):
    fits = np.zeros(cap)
    betas = np.zeros(cap)
    n = C.c_int32()
    rb = C.c_double()
    act = C.c_int32()
    _check(lib().cp_als_qr_history(ctx, _dptr(fits), _dptr(betas), int(cap), C.byref(n), C.byref(rb), C.byref(act)),
           "cp_als_qr_history")
    m = min(n.value, cap)
    return fits[:m], betas[:m], rb.value, bool(act.value)


def history_jsonl_lines(fits, betas, **extra) -> List[str]:
    """Per-sweep metrics as JSON lines: {"sweep": k (1-based), "fit": ..., "beta": ..., **extra}."""
    import json
    out = []
    for k, (f, bt) in enumerate(zip(fits, betas)):
        rec = {"sweep": k + 1, "fit": float(f), "beta": float(bt)}
        rec.update(extra)
        out.append(json.dumps(rec))
    return out


def cp_als_qr_destroy(ctx) -> None:
    if ctx:
        lib().cp_als_qr_destroy(ctx)


def cp_als_qr_schedule(dims: Sequence[int], R: int, tree: int, nsweeps: int) -> Tuple[np.ndarray, int]:
    cnt = C.c_int64()
    fl = C.c_int64()
    _check(lib().cp_als_qr_schedule(len(dims), _i64(dims), int(R), int(tree), int(nsweeps), None, 0,
                                    C.byref(cnt), C.byref(fl)), "cp_als_qr_schedule")
    ops = np.zeros((cnt.value, 4), dtype=np.int32)
    _check(lib().cp_als_qr_schedule(len(dims), _i64(dims), int(R), int(tree), int(nsweeps),
                                    ops.ctypes.data_as(C.POINTER(C.c_int32)), cnt.value, C.byref(cnt),
                                    C.byref(fl)), "cp_als_qr_schedule")
    return ops, fl.value


def cpqr_ttm(T_dev: int, tdims: Sequence[int], k: int, Q_dev: int, R: int, out_dev: int, dtype: int,
             stream: int = 0) -> None:
    _check(lib().cpqr_ttm(C.c_void_p(int(T_dev)), len(tdims), _i64(tdims), int(k), C.c_void_p(int(Q_dev)), int(R),
                          C.c_void_p(int(out_dev)), int(dtype), C.c_void_p(int(stream))), "cpqr_ttm")


def cpqr_house_qr(A_dev: int, M: int, R: int, Q_dev: int, R_dev: int, stream: int = 0) -> None:
    _check(lib().cpqr_house_qr(C.c_void_p(int(A_dev)), int(M), int(R), C.c_void_p(int(Q_dev)),
                               C.c_void_p(int(R_dev)), C.c_void_p(int(stream))), "cpqr_house_qr")


NOALLOC_QR_MAX_ELEMS = 1 << 20


def cpqr_house_qr_noalloc(A_dev: int, M: int, R: int, Q_dev: int, R_dev: int, stream: int = 0) -> None:
    """cpqr_house_qr without device allocation (fixed static scratch; M * R <= NOALLOC_QR_MAX_ELEMS;
    calls that overlap on the GPU race)."""
    _check(lib().cpqr_house_qr_noalloc(C.c_void_p(int(A_dev)), int(M), int(R), C.c_void_p(int(Q_dev)),
                                       C.c_void_p(int(R_dev)), C.c_void_p(int(stream))), "cpqr_house_qr_noalloc")


def cpqr_krp_qr(Rs_dev: int, m: int, R: int, Q0_dev: int, R0_dev: int, stream: int = 0) -> None:
    _check(lib().cpqr_krp_qr(C.c_void_p(int(Rs_dev)), int(m), int(R), C.c_void_p(int(Q0_dev)),
                             C.c_void_p(int(R0_dev)), C.c_void_p(int(stream))), "cpqr_krp_qr")


class Decomposition:
    """Owns one context; X must stay alive (device memory) while it exists."""

    def __init__(self, dims, R, X_dev: int, x_is_fp64: bool, A0=None, options: Optional[Options] = None,
                 stream: int = 0):
        self.dims = [int(d) for d in dims]
        self.R = int(R)
        self.ctx = cp_als_qr_init(self.dims, self.R, X_dev, x_is_fp64, A0, options, stream)

    def sweep(self, n: int = 1) -> np.ndarray:
        return cp_als_qr_sweep(self.ctx, n)

    def fit(self, tol: float, max_sweeps: int):
        return cp_als_qr_fit(self.ctx, tol, max_sweeps)

    def factors(self):
        out = [cp_als_qr_get(self.ctx, n, I, self.R) for n, I in enumerate(self.dims)]
        return [o[0] for o in out], out[-1][1], [o[2] for o in out], [o[3] for o in out]

    def stats(self) -> Stats:
        return cp_als_qr_stats(self.ctx)

    def fit_exact(self) -> float:
        return cp_als_qr_fit_exact(self.ctx)

    def set_timing(self, on: bool) -> None:
        cp_als_qr_set_timing(self.ctx, on)

    def checkpoint(self):
        cp_als_qr_checkpoint(self.ctx)

    def rollback(self):
        cp_als_qr_rollback(self.ctx)

    def commit(self):
        cp_als_qr_commit(self.ctx)

    def sweep_beta(self, beta: float) -> float:
        return cp_als_qr_sweep_beta(self.ctx, beta)

    def history(self):
        return cp_als_qr_history(self.ctx)

    def write_history_jsonl(self, path: str, **extra) -> int:
        """Append one JSON line per sweep done (fit, beta, and the extra keys) to path; returns
        the number of lines."""
        fits, betas, _, _ = self.history()
        lines = history_jsonl_lines(fits, betas, **extra)
        with open(path, "a") as fh:
            for ln in lines:
                fh.write(ln + "\n")
        return len(lines)

    def close(self):
        if self.ctx:
            cp_als_qr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
