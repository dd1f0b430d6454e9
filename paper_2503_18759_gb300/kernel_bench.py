"""Runs one kernel of the library on a seeded case, for timing and for ncu captures.

  python -m paper_2503_18759_gb300.kernel_bench ttm_tc P K S R [reps]   # split-bf16 tensor-core TTM
  python -m paper_2503_18759_gb300.kernel_bench ttm_f32 P K S R [reps]  # FP32 CUDA-core TTM
  python -m paper_2503_18759_gb300.kernel_bench house_qr M R [reps]     # FP64 cluster Householder QR
  python -m paper_2503_18759_gb300.kernel_bench krp_qr m R [reps]       # QR of a Khatri-Rao product of m triangles
  add --phases to house_qr / krp_qr to use the profiling build and print per-phase times.
"""
from __future__ import annotations

import ctypes
import os
import sys
import time

import numpy as np


def main(argv):
    import torch

    from . import binding as b
    from . import build

    phases = "--phases" in argv
    argv = [a for a in argv if a != "--phases"]
    if phases:
        b.LIB_PATH = build.build(variant="phases")
    else:
        build.build()
    L = b.lib()
    kind = argv[0]
    g = np.random.default_rng(0)
    dev = "cuda"
    if kind in ("ttm_tc", "ttm_f32"):
        P, K, S, R = (int(v) for v in argv[1:5])
        reps = int(argv[5]) if len(argv) > 5 else 3
        X = torch.from_numpy(g.standard_normal((P, K, S)).astype(np.float32)).to(dev)
        Qn = np.linalg.qr(g.standard_normal((K, R)))[0]
        Q = torch.from_numpy(Qn if kind == "ttm_tc" else Qn.astype(np.float32)).to(dev)
        out = torch.empty((P, R, S), dtype=torch.float32, device=dev)
        dt = b.TTM_SPLIT_BF16 if kind == "ttm_tc" else b.TTM_F32
        run = lambda: b.cpqr_ttm(X.data_ptr(), [P, K, S], 1, Q.data_ptr(), R, out.data_ptr(), dt)
    elif kind == "house_qr":
        M, R = int(argv[1]), int(argv[2])
        reps = int(argv[3]) if len(argv) > 3 else 3
        A = torch.from_numpy(g.standard_normal((M, R))).to(dev)
        Q = torch.empty((M, R), dtype=torch.float64, device=dev)
        Rm = torch.empty((R, R), dtype=torch.float64, device=dev)
        run = lambda: b.cpqr_house_qr(A.data_ptr(), M, R, Q.data_ptr(), Rm.data_ptr())
    elif kind == "krp_qr":
        m, R = int(argv[1]), int(argv[2])
        reps = int(argv[3]) if len(argv) > 3 else 3
        tri = [np.linalg.qr(g.standard_normal((R + 8, R)))[1] for _ in range(m)]
        tri = [t * np.sign(np.diag(t))[:, None] for t in tri]
        Rs = torch.from_numpy(np.stack(tri)).to(dev)
        Q0 = torch.empty((R ** m, R), dtype=torch.float64, device=dev)
        R0 = torch.empty((R, R), dtype=torch.float64, device=dev)
        run = lambda: b.cpqr_krp_qr(Rs.data_ptr(), m, R, Q0.data_ptr(), R0.data_ptr())
    else:
        raise SystemExit(__doc__)
    run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        run()
    torch.cuda.synchronize()
    print(f"{kind} {argv[1:]}: {(time.perf_counter() - t0) / reps * 1e6:.1f} us per call (incl. host work)")
    if phases and kind in ("house_qr", "krp_qr"):
        buf = (ctypes.c_ulonglong * 8)()
        L.cpqr_debug_qr_phases(buf)
        t = [buf[i] for i in range(7)]
        names = ["prologue", "householder", "R out", "T solve", "W2 gather", "Q rows"]
        print(" ".join(f"{n} {(t[i + 1] - t[i]) / 1000:.1f}us" for i, n in enumerate(names)),
              f"total {(t[6] - t[0]) / 1000:.1f}us")
        cb = (ctypes.c_longlong * 16)()
        L.cpqr_debug_qr_columns(cb)
        R = int(argv[2])
        cn = ["loop-top", "update+dots", "sync", "send", "wait", "consume", "scalars", "step-sync"]
        for rk in range(2):
            print(f"  rank {'0' if rk == 0 else 'last'} cycles/column:",
                  " ".join(f"{cn[i]} {cb[8 * rk + i] / R:.0f}" for i in range(8)),
                  f"sum {sum(cb[8 * rk + i] for i in range(8)) / R:.0f}")


if __name__ == "__main__":
    main(sys.argv[1:])
