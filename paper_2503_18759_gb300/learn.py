"""Training and evaluation of the learned extrapolation proposer.

The solver itself generates the data: along a trajectory, every `stride` sweeps from the
second on, the state is checkpointed and each candidate beta (cp_als_qr_mlp_beta) is run
for `horizon` sweeps; the candidate with the highest fit (ties: the smaller beta) is the
label of the features of that state, and the trajectory continues with it.  The network
(3 hidden layers of 128, bf16) is trained with the library's own forward / backward /
Adam kernels.  Evaluation compares, on held-out tensors, sweeps and time to the fit
tolerance with the learned proposer (judged against the Section 4.2 rule), with the rule
alone and without extrapolation.

  python -m paper_2503_18759_gb300.learn train --problems 2000 --out weights.npy --eval-problems 200 --record r.json
  python -m paper_2503_18759_gb300.learn eval --weights weights.npy --problems 200
"""
from __future__ import annotations

import argparse
import json
import time
from typing import List, Sequence

import numpy as np

from . import binding as b
from . import inputs


WEIGHTS = __import__("os").path.join(__import__("os").path.dirname(__file__), "weights", "beta_mlp.npy")


def load_weights(path: str = WEIGHTS) -> np.ndarray:
    """The committed trained parameters (float32, CPQR_MLP_NPARAMS)."""
    w = np.load(path).astype(np.float32)
    if w.size != b.MLP_NPARAMS:
        raise ValueError(f"{path}: {w.size} parameters, expected {b.MLP_NPARAMS}")
    return w


def candidates() -> List[float]:
    return [b.cp_als_qr_mlp_beta(c) for c in range(b.MLP_CLASSES)]


def problem_set(start: int, count: int, order: int = 3, base_seed: int = 0):
    """Seeded problems of the training distribution: order 3 sides U{64..256} (order 4:
    U{24..64}), rank U{8..32}, congruence U[0, 0.95], noise log-uniform in [1e-4, 1e-2]."""
    for i in range(start, start + count):
        g = np.random.default_rng([base_seed, i, order])
        if order == 3:
            dims = [int(v) for v in g.integers(64, 257, size=3)]
        else:
            dims = [int(v) for v in g.integers(24, 65, size=order)]
        R = min(int(g.integers(8, 33)), min(dims))
        c = float(g.uniform(0.0, 0.95))
        eta = float(10.0 ** g.uniform(-4.0, -2.0))
        yield inputs.make_problem_device(f"p{order}_{i}", dims, R, seed=base_seed * 100003 + i * 7 + order, c=c,
                                         eta=eta)


def trajectories(problems, sweeps: int = 60, horizon: int = 2, start: int = 2, stride: int = 5,
                 prec: int = b.PREC_SPLIT_BF16):
    """Labelled states every `stride` sweeps from `start` to `sweeps`: features of the history and
    the candidate with the highest fit after `horizon` sweeps from that state (ties: the smaller
    beta).  The trajectory advances with the label between labelled states."""
    cand = candidates()
    feats, labels = [], []
    for prob in problems:
        opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=prec, extrap=b.EXTRAP_PAPER)
        with b.Decomposition(prob.dims, prob.R, prob.X.data_ptr(), False, prob.A0, opts) as d:
            d.sweep(start)
            best = 0
            for k in range(start, sweeps):
                if (k - start) % stride:
                    d.sweep_beta(cand[best])
                    continue
                fits, betas, rule, act = d.history()
                f = b.cpqr_mlp_features(fits, betas, rule, act)
                d.checkpoint()
                res = []
                for ci, beta in enumerate(cand):
                    if ci:
                        d.rollback()
                    fit = 0.0
                    for _ in range(horizon):
                        fit = d.sweep_beta(beta)
                    res.append(fit)
                d.rollback()
                d.commit()
                res = np.array(res)
                best = int(np.min(np.nonzero(res >= res.max() - 1e-13)[0]))
                feats.append(f)
                labels.append(best)
                d.sweep_beta(cand[best])
    return np.array(feats, dtype=np.float32), np.array(labels, dtype=np.int32)


def init_params(seed: int = 0) -> np.ndarray:
    g = np.random.default_rng(seed)
    shapes = [(b.MLP_HIDDEN, b.MLP_FEATURES), (b.MLP_HIDDEN, b.MLP_HIDDEN), (b.MLP_HIDDEN, b.MLP_HIDDEN),
              (b.MLP_CLASSES, b.MLP_HIDDEN)]
    parts = []
    for o, i in shapes:
        parts.append(g.standard_normal(o * i) * np.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == b.MLP_NPARAMS
    return p


def train(feats: np.ndarray, labels: np.ndarray, epochs: int = 60, batch: int = 256, lr: float = 1e-3,
          seed: int = 0, log=None) -> np.ndarray:
    import torch

    dev = "cuda"
    params = torch.from_numpy(init_params(seed)).to(dev)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    Xall = torch.from_numpy(feats).to(dev)
    yall = torch.from_numpy(labels.astype(np.int32)).to(dev)
    n = len(labels)
    B = min(batch, n)
    work = torch.empty(b.cpqr_mlp_work_bytes(B), dtype=torch.uint8, device=dev)
    g = np.random.default_rng(seed)
    step = 0
    for ep in range(epochs):
        perm = torch.from_numpy(g.permutation(n)).to(dev)
        tot = 0.0
        for i in range(0, n - B + 1, B):
            idx = perm[i:i + B]
            Xb = Xall[idx].contiguous()
            yb = yall[idx].contiguous()
            b.cpqr_mlp_grad(params.data_ptr(), Xb.data_ptr(), yb.data_ptr(), B, grad.data_ptr(), loss.data_ptr(),
                            work.data_ptr())
            step += 1
            b.cpqr_mlp_adam(params.data_ptr(), m.data_ptr(), v.data_ptr(), grad.data_ptr(), lr, step)
            tot += loss.item()
        if log is not None:
            log(ep, tot / max(1, n // B))
    torch.cuda.synchronize()
    return params.cpu().numpy()


def accuracy(params: np.ndarray, feats: np.ndarray, labels: np.ndarray) -> float:
    import torch

    dev = "cuda"
    n = len(labels)
    pd = torch.from_numpy(params).to(dev)
    X = torch.from_numpy(feats).to(dev)
    logits = torch.empty((n, b.MLP_CLASSES), dtype=torch.float32, device=dev)
    work = torch.empty(b.cpqr_mlp_work_bytes(n), dtype=torch.uint8, device=dev)
    b.cpqr_mlp_forward(pd.data_ptr(), X.data_ptr(), n, logits.data_ptr(), work.data_ptr())
    pred = logits.argmax(dim=1).cpu().numpy()
    return float(np.mean(pred == labels))


def evaluate(params, problems, max_sweeps: int = 120, prec: int = b.PREC_SPLIT_BF16, gap: float = 1e-6):
    """Per problem: every mode (no extrapolation, the Section 4.2 rule, the learned proposer)
    runs max_sweeps sweeps; f* is the best fit any of them reaches; reported are the sweeps and
    the seconds each mode needs to reach f* - gap (max_sweeps / its full time if never), the
    final fit and the proposal counters.  The split path's per-sweep fits come from the explicit
    residual (~1e-7 of the fit), fine enough for the 1e-6 target."""
    import torch

    out = []
    modes = [("none", b.EXTRAP_NONE, None), ("paper", b.EXTRAP_PAPER, None), ("learned", b.EXTRAP_LEARNED, params)]
    for prob in problems:
        traces = {}
        for name, ex, w in modes:
            opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=prec, extrap=ex, mlp_weights=w)
            with b.Decomposition(prob.dims, prob.R, prob.X.data_ptr(), False, prob.A0, opts) as d:
                fits, stamps = [], []
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(max_sweeps):
                    fits.append(float(d.sweep(1)[0]))
                    stamps.append(time.perf_counter() - t0)
                st = d.stats()
                traces[name] = (np.array(fits), np.array(stamps), st.proposals, st.accepted, st.judged)
        fstar = max(float(t[0].max()) for t in traces.values())
        row = {"name": prob.name, "dims": prob.dims, "R": prob.R, "fstar": fstar}
        for name, (f, t, props, acc, jd) in traces.items():
            hit = np.nonzero(f >= fstar - gap)[0]
            k = int(hit[0]) if len(hit) else max_sweeps - 1
            row[name] = {"sweeps_to_target": k + 1, "seconds_to_target": float(t[k]), "reached": bool(len(hit)),
                         "final_fit": float(f[-1]), "s_per_sweep": float(t[-1] / len(t)), "proposals": int(props),
                         "accepted": int(acc), "judged": int(jd), "sweeps_run": int(len(f))}
        out.append(row)
    return out


def summarize(rows):
    s = {"problems": len(rows)}
    for name in ("none", "paper", "learned"):
        s[name] = {"mean_sweeps_to_target": float(np.mean([r[name]["sweeps_to_target"] for r in rows])),
                   "mean_seconds_to_target": float(np.mean([r[name]["seconds_to_target"] for r in rows])),
                   "reached": int(sum(r[name]["reached"] for r in rows)),
                   "mean_final_fit": float(np.mean([r[name]["final_fit"] for r in rows])),
                   "mean_s_per_sweep": float(np.mean([r[name]["s_per_sweep"] for r in rows]))}
    s["learned"]["accept_rate"] = float(sum(r["learned"]["accepted"] for r in rows) /
                                        max(1, sum(r["learned"]["proposals"] for r in rows)))
    s["learned"]["judged_per_sweep"] = float(sum(r["learned"]["judged"] for r in rows) /
                                             max(1, sum(r["learned"]["sweeps_run"] for r in rows)))
    # head-to-head: problems where the learned proposer reaches the target in fewer / more
    # seconds than each other mode
    for other in ("none", "paper"):
        faster = sum(1 for r in rows if r["learned"]["seconds_to_target"] < r[other]["seconds_to_target"])
        s["learned"][f"faster_than_{other}"] = faster
        s["learned"][f"slower_than_{other}"] = len(rows) - faster
    return s


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--problems", type=int, default=200)
    ap.add_argument("--sweeps", type=int, default=60)
    ap.add_argument("--stride", type=int, default=5)
    ap.add_argument("--record", default=None, help="write the training / evaluation record (JSON) here")
    ap.add_argument("--eval-problems", type=int, default=0, help="after training: evaluate on this many held-out "
                    "problems, half order 3 and half order 4")
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", default="beta_mlp.npy")
    ap.add_argument("--weights", default="beta_mlp.npy")
    ap.add_argument("--order", type=int, default=3, help="eval: 3 or 4, or 0 for half of each")
    ap.add_argument("--start", type=int, default=0)
    ap.add_argument("--horizon", type=int, default=3)
    ap.add_argument("--max-sweeps", type=int, default=120)
    args = ap.parse_args()
    b.lib()
    if args.cmd == "train":
        t0 = time.time()
        F, y = trajectories(problem_set(args.start, args.problems), sweeps=args.sweeps, horizon=args.horizon,
                            stride=args.stride)
        t1 = time.time()
        w = train(F, y, epochs=args.epochs)
        np.save(args.out, w)
        rec = {"command": "python -m paper_2503_18759_gb300.learn " + " ".join(__import__("sys").argv[1:]),
               "data": f"{args.problems} seeded order-3 training problems (sides U{{64..256}}, rank U{{8..32}}, "
                       f"congruence U[0,0.95], noise log-uniform [1e-4,1e-2]); a labelled state every "
                       f"{args.stride} sweeps from sweep 2 to {args.sweeps}; label = candidate beta with the highest "
                       f"fit after {args.horizon} sweeps (ties: the smaller beta); split-precision solver",
               "states": int(len(y)), "label_counts": np.bincount(y, minlength=b.MLP_CLASSES).tolist(),
               "generate_s": t1 - t0, "train_s": time.time() - t1, "train_accuracy": accuracy(w, F, y)}
        if args.eval_problems:
            half = args.eval_problems // 2
            rows = evaluate(w, problem_set(10000, half, order=3), max_sweeps=args.max_sweeps)
            rows += evaluate(w, problem_set(10000, args.eval_problems - half, order=4), max_sweeps=args.max_sweeps)
            rec["heldout"] = {"problems": f"{half} order-3 and {args.eval_problems - half} order-4 held-out problems "
                                          f"(seeds apart from training; order-4 sides U{{24..64}}), split path, "
                                          f"{args.max_sweeps} sweeps each, target f* - 1e-6 with f* the best fit "
                                          f"of the three modes",
                              "summary": summarize(rows)}
        print(json.dumps(rec))
        if args.record:
            with open(args.record, "w") as fh:
                json.dump(rec, fh, indent=1)
    else:
        w = np.load(args.weights).astype(np.float32)
        if args.order == 0:  # half order 3, half order 4 (the held-out set of the training record)
            half = args.problems // 2
            rows = evaluate(w, problem_set(10000 + args.start, half, order=3), max_sweeps=args.max_sweeps)
            rows += evaluate(w, problem_set(10000 + args.start, args.problems - half, order=4),
                             max_sweeps=args.max_sweeps)
        else:
            rows = evaluate(w, problem_set(10000 + args.start, args.problems, order=args.order),
                            max_sweeps=args.max_sweeps)
        summary = summarize(rows)
        print(json.dumps(summary))
        if args.record:  # update the held-out part of an existing training record
            with open(args.record) as fh:
                rec = json.load(fh)
            rec["heldout"] = {"problems": f"{args.problems} held-out problems (order " +
                                          ("3 and 4, half each" if args.order == 0 else str(args.order)) +
                                          f"; order-4 sides U{{24..64}}), split path, {args.max_sweeps} sweeps each, "
                                          "target f* - 1e-6 with f* the best fit of the three modes",
                              "command": "python -m paper_2503_18759_gb300.learn " +
                                         " ".join(__import__("sys").argv[1:]),
                              "summary": summary}
            with open(args.record, "w") as fh:
                json.dump(rec, fh, indent=1)


if __name__ == "__main__":
    main()
