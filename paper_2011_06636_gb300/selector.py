"""Learned scheme selector: trace collection, training, and the stored weights.

Traces follow the paper's data-collection procedure (Sec. 3): the solver
starts a problem at level 0; at each later decision it tries the three moves
(level - 1, same, level + 1) from the same iterate, records the average
convergence rate -log(r_after / r_before) / M of each (Sec. 3, Eq.
average-convergence-rate), and continues with one of the moves.  The paper
draws that move at random; here half of the moves follow the best-rated one
and half are random, so that trajectories of the larger problems reach the
high levels they need within a bounded number of cycles (a purely random walk
spends nearly all its samples at low levels).  Each decision becomes one
training sample: the features of the state (see csrc/mlp.cuh) labelled with
the move of the best rate.  Every cycle runs in
the library (FP64 sweeps through ``srj_run_levels``); training runs in the
library's CUDA kernel (``srj_mlp_train``).

    python -m paper_2011_06636_gb300.selector --out selector_bf16.bin

writes the BF16 weights (6617 little-endian uint16) next to this file by
default; ``load_weights()`` reads them back.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "selector_bf16.bin")
N_PARAMS = 6617
LEVEL_M = [1, 2, 3, 5, 7, 10, 14, 19, 26, 35, 47, 63, 84, 111, 147, 194, 256, 338, 446, 589,
           778, 1027, 1356, 1790, 2362]


def features(hist, npoints, dim, level):
    """The 12 selector inputs (same definition as csrc/mlp.cuh)."""
    x = np.zeros(12, dtype=np.float32)
    for i, v in enumerate(hist[:8]):
        x[i] = v
    x[8] = math.log10(npoints) / 10.0
    x[9] = dim / 3.0
    x[10] = level / 24.0
    x[11] = math.log(LEVEL_M[level]) / math.log(2362.0)
    return x


def _log_ratio(r):
    return float(min(5.0, max(-20.0, math.log(r)))) if r > 0 else -20.0


def collect(problem, seed, max_cycles=160, tol=1e-8, records=None, greedy=0.5):
    """One trajectory of the paper's data-collection walk on `problem`
    (dict n, eps, f).  Returns (X, y) lists; when `records` is a list, every
    tried move is appended to it as (previous ratio, level, move, rate), the
    data of Sec. 3's post-processing."""
    import torch

    from . import srj
    n = problem["n"]
    f = torch.as_tensor(np.ascontiguousarray(problem["f"]), device="cuda")
    h = srj.srj_create(n, eps=problem.get("eps"), precision=srj.SRJ_PREC_F64,
                       trace_capacity=8)
    rng = np.random.default_rng(seed)
    npts = int(np.prod(n))
    X, y = [], []
    try:
        u = torch.zeros_like(f)
        r0 = srj.srj_residual_norm(h, f.data_ptr(), u.data_ptr())
        rn = srj.srj_run_levels(h, f.data_ptr(), u.data_ptr(), [0])[0]  # first cycle at level 0
        hist = [_log_ratio(rn / r0)]
        level = 0
        for _ in range(max_cycles):
            if rn / r0 < tol:
                break
            cands = [c for c in (level - 1, level, level + 1) if 0 <= c <= 24]
            outs = []
            for c in cands:
                uc = u.clone()
                rc = srj.srj_run_levels(h, f.data_ptr(), uc.data_ptr(), [c])[0]
                rate = -math.log(max(rc, 1e-300) / rn) / LEVEL_M[c]
                outs.append((rate, c, uc, rc))
            best = max(outs, key=lambda t: t[0])
            if records is not None:
                for rate_c, c, _, _ in outs:
                    records.append((math.exp(hist[0]), level, c - level, rate_c))
            X.append(features(hist, npts, len(n), level))
            y.append(best[1])
            pick = best if rng.random() < greedy else outs[int(rng.integers(len(outs)))]
            rate, level, u, rnew = pick
            hist = [_log_ratio(rnew / rn)] + hist
            rn = rnew
    finally:
        srj.srj_destroy(h)
    return X, y


def rollout_collect(problem, seed, explore=0.3, max_cycles=200, tol=1e-8, horizon=1e-2,
                    deadline=None):
    """States along Alg. 1 trajectories on `problem` (dict n, eps, f), with a
    random move instead of Alg. 1's one with probability `explore` so that
    other states are visited too.  Each state is labelled with the move after
    which Alg. 1 reduces the residual by `horizon` in the fewest sweeps (a
    rollout per move: a library solve from the state whose first cycle runs at
    the tried level and whose later cycles follow Alg. 1), i.e. one step of
    policy improvement over Alg. 1; ties go to Alg. 1's own move.  Returns
    (X, y, number of states where the label differs from Alg. 1's move)."""
    import torch

    from . import srj
    n = problem["n"]
    f = torch.as_tensor(np.ascontiguousarray(problem["f"]), device="cuda")
    npts = int(np.prod(n))
    handles = {}

    def handle(level0):
        if level0 not in handles:
            handles[level0] = srj.srj_create(n, eps=problem.get("eps"),
                                             precision=srj.SRJ_PREC_F64, level0=level0,
                                             trace_capacity=8)
        return handles[level0]

    rng = np.random.default_rng(seed)
    X, y, differ = [], [], 0
    try:
        h0 = handle(0)
        u = torch.zeros_like(f)
        r0 = srj.srj_residual_norm(h0, f.data_ptr(), u.data_ptr())
        rn = srj.srj_run_levels(h0, f.data_ptr(), u.data_ptr(), [0])[0]
        hist = [_log_ratio(rn / r0)]
        level = 0
        for _ in range(max_cycles):
            if rn / r0 < tol or (deadline is not None and time.time() > deadline):
                break
            ratio = math.exp(hist[0])
            alg1 = min(24, level + 1) if ratio > 0.4 else (
                max(0, level - 1) if 0.2 < ratio < 0.4 else level)
            cands = [c for c in (level - 1, level, level + 1) if 0 <= c <= 24]
            cost = {}
            for c in cands:
                uc = u.clone()
                st = srj.srj_solve(handle(c), f.data_ptr(), uc.data_ptr(), horizon)
                cost[c] = st["sweeps"] if st["status"] == srj.SRJ_OK else 10 ** 9
            best = min(cands, key=lambda c: (cost[c], c != alg1))
            differ += int(best != alg1)
            X.append(features(hist, npts, len(n), level))
            y.append(best)
            nxt = alg1 if rng.random() >= explore else cands[int(rng.integers(len(cands)))]
            rnew = srj.srj_run_levels(h0, f.data_ptr(), u.data_ptr(), [nxt])[0]
            hist = [_log_ratio(rnew / rn)] + hist
            rn = rnew
            level = nxt
    finally:
        for hh in handles.values():
            srj.srj_destroy(hh)
    return X, y, differ


def training_problems(seed=0, small=False):
    """Seeded 1D and 2D Poisson problems (b = 1 as in Sec. 3 and random f),
    sizes interleaved; small=True keeps 1D up to 4096 points and 2D up to
    256^2 (what the rollout labels can afford)."""
    from . import inputs
    n1 = (16, 32, 64, 128, 256, 512, 1024, 2048, 4096) + (() if small else (8192, 16384))
    n2 = (16, 32, 64, 128, 256) + (() if small else (512, 1024))
    probs = []
    for i in range(max(len(n1), len(n2))):
        for N in ([n1[i]] if i < len(n1) else []):
            probs.append({"n": [N], "f": np.ones(N)})
            probs.append({"n": [N], "f": inputs.uniform_rhs([N], seed=seed + N).ravel()})
        for s_ in ([n2[i]] if i < len(n2) else []):
            probs.append({"n": [s_, s_], "f": np.ones(s_ * s_)})
            probs.append({"n": [s_, s_], "f": inputs.uniform_rhs([s_, s_], seed=seed + s_).ravel()})
    return probs


def analyse(records, n_set=200):
    """Sec. 3 post-processing of the collected moves: per level, sort by the
    previous residual ratio, cut into clusters of n_set records, and in each
    cluster take the mean rate of each move with a 95 % confidence interval;
    a cluster's winner is the move with the best mean whose interval does not
    overlap the others'.  Returns the winners (mean ratio, level, move) and
    the ratio thresholds they imply: the largest ratio won by 'keep' and the
    smallest ratio won by 'up' (the paper reads 0.2 and 0.4 off this plot)."""
    rec = np.asarray(records, dtype=np.float64)
    winners = []
    for level in np.unique(rec[:, 1]).astype(int):
        sub = rec[rec[:, 1] == level]
        sub = sub[np.argsort(sub[:, 0], kind="stable")]
        for c0 in range(0, len(sub) - n_set + 1, n_set):
            cl = sub[c0:c0 + n_set]
            stats = {}
            for mv in (-1, 0, 1):
                r = cl[cl[:, 2] == mv][:, 3]
                if len(r) >= 5:
                    half = 1.96 * r.std(ddof=1) / math.sqrt(len(r))
                    stats[mv] = (r.mean(), r.mean() - half, r.mean() + half)
            if len(stats) < 2:
                continue
            best = max(stats, key=lambda m: stats[m][0])
            if all(stats[best][1] > stats[m][2] for m in stats if m != best):
                winners.append((float(cl[:, 0].mean()), int(level), int(best)))
    keep = [w[0] for w in winners if w[2] == 0]
    up = [w[0] for w in winners if w[2] == 1]
    down = [w[0] for w in winners if w[2] == -1]
    return {"clusters_with_winner": len(winners),
            "keep_max_ratio": max(keep) if keep else None,
            "down_ratio_range": [min(down), max(down)] if down else None,
            "up_min_ratio": min(up) if up else None,
            "winners": winners}


# ------------------------------------------------ Sec. 3, the paper's study
# The matrix sizes of the paper's data collection (Sec. 3): 1D Poisson, b = 1,
# x0 = 0, trials until ||r||_2 < 1e-8, about one million data points per size.
SEC3_N = (2, 5, 10, 20, 30, 40, 50, 60, 70, 80, 90, 100, 200, 300, 400)
SEC3_JSON = os.path.join(HERE, "sec3_thresholds.json")


def sec3_collect(n, target=1_000_000, seed=0, tol=1e-8, max_steps=4000, mem_bytes=2 << 30):
    """Records of the Sec. 3 collection on the size-n system (library
    kernel, one trial per CTA), in batches of trials until at least `target`
    records.  Returns (records as a numpy structured array, number of trials,
    number of trials cut at max_steps)."""
    import torch

    from . import srj
    dt = np.dtype(srj.MOVE_RECORD_DTYPE)
    per_trial = 3 * max_steps
    cap = max(1, mem_bytes // (per_trial * dt.itemsize))
    parts, total, trial0, cut = [], 0, 0, 0
    est = None  # records per trial seen so far
    while total < target:
        left = target - total
        ntr = 256 if est is None else int(min(cap, max(64, 1.2 * left / est + 1)))
        out = torch.empty(ntr * per_trial * dt.itemsize // 8, dtype=torch.float64, device="cuda")
        counts = torch.zeros(ntr, dtype=torch.int32, device="cuda")
        srj.srj_collect_moves(n, None, tol, 24, seed, trial0, ntr, max_steps, out.data_ptr(),
                              counts.data_ptr())
        # keep each trial's written records (device-side gather, then one copy)
        rec = out.view(ntr, per_trial * dt.itemsize // 8)
        words = dt.itemsize // 8
        idx = torch.arange(per_trial, device="cuda")[None, :] < counts[:, None].long()
        flat = rec.view(ntr, per_trial, words)[idx]
        parts.append(flat.cpu().numpy().reshape(-1).view(dt))
        c = counts.cpu().numpy()
        cut += int(np.sum(c >= per_trial - 2))
        total += int(c.sum())
        trial0 += ntr
        est = total / trial0
    return np.concatenate(parts), trial0, cut


def sec3_rates(rec):
    """Average convergence rate of every record (Sec. 3, Eq.
    average-convergence-rate): -log(r_after / r_before) / M of the tried level."""
    m = np.asarray(LEVEL_M, dtype=np.float64)[rec["level"] + rec["action"]]
    return -np.log(rec["r_after"] / rec["r_before"]) / m


def alg1_action(ratio):
    """Alg. 1's move for a previous residual ratio (the rule the study is
    meant to recover): +1 above 0.4, -1 strictly between 0.2 and 0.4, else 0."""
    return 1 if ratio > 0.4 else (-1 if 0.2 < ratio < 0.4 else 0)


def sec3_study(sizes=SEC3_N, target=1_000_000, n_set=10000, seed=0):
    """The paper's data collection on every size, post-processed together
    (Sec. 3): per level, clusters of n_set records sorted by previous ratio,
    the winning move of each cluster with non-overlapping 95 % intervals.
    Returns a summary with the winners and how well Alg. 1's thresholds
    (0.2, 0.4) and the best-fitting pair explain them."""
    t0 = time.time()
    allrec, per_size = [], {}
    for n in sizes:
        rec, trials, cut = sec3_collect(n, target=target, seed=seed + n)
        allrec.append(rec)
        per_size[str(n)] = {"records": int(len(rec)), "trials": trials, "trials_cut": cut,
                            "max_level": int((rec["level"] + rec["action"]).max())}
    rec = np.concatenate(allrec)
    rows = np.stack([rec["prev_ratio"], rec["level"].astype(np.float64),
                     rec["action"].astype(np.float64), sec3_rates(rec)], axis=1)
    out = {"sizes": list(sizes), "records_total": int(len(rec)), "n_set": n_set,
           "per_size": per_size}
    out.update(sec3_summary(rows, n_set))
    out["seconds"] = time.time() - t0
    return out


def sec3_summary(rows, n_set):
    """Post-processing of Sec. 3 on rows (previous ratio, level, move, rate):
    the cluster winners (analyse), the share of them Alg. 1's thresholds
    (0.2, 0.4) explain, and the pair of thresholds (grid step 0.02) that
    explains the most."""
    res = analyse(rows, n_set=n_set)
    win = res["winners"]
    agree = sum(1 for r, _, a in win if alg1_action(r) == a)
    best = (0, None, None)
    grid = np.round(np.arange(0.02, 0.99, 0.02), 2)
    for lo in grid:
        for hi in grid[grid > lo]:
            k = sum(1 for r, _, a in win
                    if (1 if r > hi else (-1 if lo < r < hi else 0)) == a)
            if k > best[0]:
                best = (k, float(lo), float(hi))
    return {"clusters_with_winner": res["clusters_with_winner"],
            "keep_max_ratio": res["keep_max_ratio"], "down_ratio_range": res["down_ratio_range"],
            "up_min_ratio": res["up_min_ratio"],
            "alg1_agreement": agree / len(win) if win else None,
            "best_fit_thresholds": {"low": best[1], "high": best[2],
                                    "agreement": best[0] / len(win) if win else None},
            "winners": [{"mean_ratio": r, "level": lv, "action": a} for r, lv, a in win]}


def train(X, y, epochs=40, batch=64, lr=3e-3, seed=0):
    import torch

    from . import inputs, srj
    X = np.asarray(X, dtype=np.float32)
    y = np.asarray(y, dtype=np.int32)
    n = len(y)
    order = inputs.minibatch_order(n, epochs, seed)
    steps = len(order) // batch
    theta = torch.as_tensor(inputs.mlp_init(seed), device="cuda")
    xd = torch.as_tensor(X, device="cuda")
    yd = torch.as_tensor(y, device="cuda")
    od = torch.as_tensor(order[:steps * batch], device="cuda")
    loss = srj.srj_mlp_train(xd.data_ptr(), yd.data_ptr(), n, od.data_ptr(), steps, batch, lr,
                             theta.data_ptr())
    return theta.cpu().numpy(), loss


def to_bf16_bits(theta):
    a = np.asarray(theta, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def load_weights(path=WEIGHTS):
    w = np.fromfile(path, dtype="<u2")
    if w.size != N_PARAMS:
        raise ValueError("selector weights: expected %d values, got %d" % (N_PARAMS, w.size))
    return w


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--seeds", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--labels", choices=["greedy", "rollout"], default="rollout",
                    help="training labels: best next-cycle rate, or the move after which "
                         "Alg. 1 reaches a 1e-2 reduction in the fewest sweeps")
    ap.add_argument("--budget", type=float, default=900.0,
                    help="seconds of trace collection for the rollout labels")
    ap.add_argument("--sec3", action="store_true",
                    help="run the paper's Sec. 3 data collection and post-processing instead")
    ap.add_argument("--sec3-target", type=int, default=1_000_000,
                    help="records per matrix size (the paper: about one million)")
    args = ap.parse_args()
    if args.sec3:
        out = sec3_study(target=args.sec3_target)
        with open(SEC3_JSON, "w") as fh:
            json.dump(out, fh, indent=1)
        print(json.dumps({k: v for k, v in out.items() if k != "winners"}))
        return
    t0 = time.time()
    X, y, records = [], [], []
    differ = 0
    deadline = t0 + args.budget
    for s in range(args.seeds):
        for i, p in enumerate(training_problems(seed=100 * s, small=args.labels == "rollout")):
            if args.labels == "rollout":
                if time.time() > deadline:
                    break
                a, b, d = rollout_collect(p, seed=1000 * s + i, deadline=deadline)
                differ += d
            else:
                a, b = collect(p, seed=1000 * s + i, records=records)
            X += a
            y += b
    t1 = time.time()
    theta, loss = train(X, y, epochs=args.epochs)
    from . import srj
    bits = to_bf16_bits(theta)
    picks, _ = srj.srj_mlp_forward(bits, np.asarray(X, dtype=np.float32))
    acc = float(np.mean(picks == np.asarray(y)))
    bits.astype("<u2").tofile(args.out)
    info = {"samples": len(y), "collect_s": t1 - t0, "train_s": time.time() - t1,
            "loss_first": float(loss[:50].mean()), "loss_last": float(loss[-50:].mean()),
            "train_accuracy": acc, "epochs": args.epochs,
            "label_counts": np.bincount(np.asarray(y), minlength=25).tolist(),
            "labels": args.labels}
    if args.labels == "rollout":
        info["labels_differing_from_alg1"] = differ
    else:
        info["sec3_postprocessing"] = {k: v for k, v in analyse(records).items()
                                       if k != "winners"}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as fh:
        json.dump(info, fh, indent=1)
    print(json.dumps(info))


if __name__ == "__main__":
    main()
