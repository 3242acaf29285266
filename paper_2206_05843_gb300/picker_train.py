"""Training and evaluation of the learned rewrite picker on timings the library measures
itself.

Harvest (per training matrix): the plain system is solved with per-level %globaltimer
stamps; then, for every candidate depth g, the matrix is rewritten with targets every
g+1 levels (under the nnz cap) and solved with stamps.  For a target level t the label is
  dt(t, g) = time of the rewritten levels that hold original levels t..t+g
           - time of original levels t..t+g in the plain solve            (nanoseconds)
and the sample's input is the 12-feature vector of candidate (t, g) computed on the
original matrix.  Training runs the library's own MLP forward, backward and Adam kernels.

Evaluation (held-out matrices): solve time of the learned strategy (and of the model's plan
alone) against the paper's naive strategy, the row-capped plan and no rewrite, with the
residual of each.

Usage: python -m paper_2206_05843_gb300.picker_train --train 600 --heldout 200 --out picker.bin
"""
from __future__ import annotations

import argparse
import json
import statistics
import sys
import time

import numpy as np

from . import binding as B
from . import synth as S

DEPTHS = list(B.DEFAULT_DEPTHS)


def _torch():
    import torch
    return torch


def level_spans(new_level: np.ndarray, old_level: np.ndarray, m_old: int):
    """For every original level: the lowest and highest level its rows land on."""
    lo = np.full(m_old, np.iinfo(np.int64).max, dtype=np.int64)
    hi = np.full(m_old, -1, dtype=np.int64)
    np.minimum.at(lo, old_level, new_level)
    np.maximum.at(hi, old_level, new_level)
    return lo, hi


def timed_stamps(sysm, bt, reps):
    torch = _torch()
    st = torch.empty(max(sysm.m, 1), dtype=torch.int64, device=bt.device)
    x = torch.empty_like(bt)
    out = []
    sysm.solve(bt, x, stamps=st)
    for _ in range(reps):
        sysm.solve(bt, x, stamps=st)
        torch.cuda.synchronize()
        out.append(st[:sysm.m].cpu().numpy().astype(np.int64))
    sysm.status()
    return out


def harvest(m, depths=DEPTHS, cap=1.5, reps=3, seed=0):
    """Samples (features, dt in ns) of one matrix."""
    torch = _torch()
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    mm = lv.m
    if mm < 3:
        return np.zeros((0, 12), np.float32), np.zeros(0, np.float32)
    old_level = lv.export()["level"].astype(np.int64)
    b = S.rhs_uniform(m.n, 1, seed)
    bt = torch.from_numpy(b[0]).cuda()
    feats = B.features(M, lv, depths).cpu().numpy().reshape(mm, len(depths), 12)
    plain = B.System(M, lv)
    sp = timed_stamps(plain, bt, reps)
    X, Y = [], []
    for d, g in enumerate(depths):
        try:
            s = B.System(M, lv, B.DEPTH_K, k=g, cap=cap)
        except B.SptrsvError:
            continue
        new_level = s.export()["level"].astype(np.int64)
        lo, hi = level_spans(new_level, old_level, mm)
        sr = timed_stamps(s, bt, reps)
        for t in range(g + 1, mm, g + 1):
            te = min(t + g, mm - 1)
            nlo, nhi = int(lo[t:te + 1].min()), int(hi[t:te + 1].max())
            if nlo <= 0:
                continue
            deltas = [(r[nhi] - r[nlo - 1]) - (p[te] - p[t - 1]) for r, p in zip(sr, sp)]
            X.append(feats[t, d])
            Y.append(statistics.median(deltas))
        del s
    return np.asarray(X, np.float32).reshape(-1, 12), np.asarray(Y, np.float32)


def train(X, Y, seed=0, epochs=60, batch=4096, lr=2e-3, log=None):
    torch = _torch()
    pk = B.Picker(seed=seed)
    mean = X.mean(axis=0)
    std = np.maximum(X.std(axis=0), 1e-3)
    scale = float(max(np.std(Y), 1.0))
    pk.set_norm(mean, std, scale)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    n = X.shape[0]
    gen = torch.Generator(device="cuda").manual_seed(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        tot = 0.0
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            loss = pk.train_step(Xd[idx].contiguous(), Yd[idx].contiguous(), lr * (0.5 ** (ep // 20)))
            tot += float(loss.item()) * idx.numel()
        hist.append(tot / n)
        if log:
            log(f"epoch {ep} loss {hist[-1]:.4f}")
    return pk, hist


def solve_time_us(sysm, bt, reps=5):
    torch = _torch()
    x = torch.empty_like(bt)
    sysm.solve(bt, x)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sysm.solve(bt, x)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e3)
    sysm.status()
    return statistics.median(ts), x


def evaluate(pk, mats, cap=1.5, log=None, time_budget=1e9):
    """Solve time of none / naive / learned; errors against x_true (b = L x_true)."""
    torch = _torch()
    rows = []
    t0 = time.time()
    for m in mats:
        if callable(m):
            if time.time() - t0 > time_budget:
                break
            m = m()
        M = B.Matrix.from_host(m)
        lv = B.Levels(M)
        xt, b = S.rhs_from_xtrue(m, 1, 7)
        bt = torch.from_numpy(b[0]).cuda()
        ref = xt[0]
        res = {"n": m.n, "levels": lv.m}
        for name, kw in (("none", {}), ("naive", dict(kind=B.NAIVE, cap=cap)),
                         ("rowcap", dict(kind=B.ROWCAP, k=32, cap=cap)),
                         ("learned", dict(kind=B.LEARNED, cap=cap, picker=pk)),
                         ("learned_model_only", dict(kind=B.LEARNED, cap=cap, picker=pk, model_only=True))):
            s = B.System(M, lv, **kw)
            us, x = solve_time_us(s, bt)
            err = float(np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref))
            res[name] = {"us": us, "levels": s.m, "rel_err": err, "strategy_used": int(s.info["strategy_used"])}
        rows.append(res)
        if log:
            log(json.dumps(res))
    def gmean(key):
        return float(np.exp(np.mean([np.log(r["none"]["us"] / r[key]["us"]) for r in rows])))
    summary = {"matrices": len(rows),
               "geomean_speedup_vs_none": {"naive": gmean("naive"), "rowcap": gmean("rowcap"),
                                           "learned": gmean("learned"),
                                           "learned_model_only": gmean("learned_model_only")},
               "geomean_speedup_learned_vs_naive": float(np.exp(np.mean(
                   [np.log(r["naive"]["us"] / r["learned"]["us"]) for r in rows]))),
               "geomean_speedup_model_only_vs_naive": float(np.exp(np.mean(
                   [np.log(r["naive"]["us"] / r["learned_model_only"]["us"]) for r in rows]))),
               "model_plan_kept": int(sum(r["learned"]["strategy_used"] == B.CHOSEN for r in rows)),
               "max_rel_err": max(max(r[k]["rel_err"] for k in ("none", "naive", "rowcap", "learned",
                                                                "learned_model_only"))
                                  for r in rows)}
    return rows, summary


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--n-lo", type=int, default=10_000)
    ap.add_argument("--n-hi", type=int, default=1_000_000)
    ap.add_argument("--eval-lo", type=int, default=100_000)
    ap.add_argument("--eval-hi", type=int, default=2_000_000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", default="picker_trained.bin")
    ap.add_argument("--report", default="picker_report.json")
    ap.add_argument("--time-budget", type=float, default=1e9, help="seconds for the harvest")
    ap.add_argument("--eval-budget", type=float, default=1e9, help="seconds for the held-out evaluation")
    ap.add_argument("--evaluate", default=None, help="evaluate this trained picker file only (no training)")
    a = ap.parse_args(argv)

    def log(s):
        print(s, flush=True)

    if a.evaluate:
        pk = B.Picker.load(a.evaluate)
        erng = S.rng_for(54321)
        mats = []
        for i in range(a.heldout):
            n = int(round(np.exp(erng.uniform(np.log(a.eval_lo), np.log(a.eval_hi)))))
            mats.append(lambda n=n, i=i: S.gen_mixture(n, 20_000 + i))
        rows, summary = evaluate(pk, mats, log=log, time_budget=a.eval_budget)
        json.dump({"picker": a.evaluate, "summary": summary, "heldout": rows}, open(a.report, "w"), indent=1)
        log(json.dumps(summary))
        return 0
    rng = S.rng_for(12345)
    t0 = time.time()
    Xs, Ys = [], []
    used = 0
    for i in range(a.train):
        if time.time() - t0 > a.time_budget:
            break
        n = int(round(np.exp(rng.uniform(np.log(a.n_lo), np.log(a.n_hi)))))
        m = S.gen_mixture(n, 10_000 + i)
        X, Y = harvest(m, seed=i)
        Xs.append(X)
        Ys.append(Y)
        used += 1
        if i % 20 == 0:
            log(f"harvest {i}: n={m.n} samples={len(Y)} elapsed={time.time() - t0:.0f}s")
    X = np.concatenate(Xs)
    Y = np.concatenate(Ys)
    log(f"dataset: {X.shape[0]} samples from {used} matrices")
    pk, hist = train(X, Y, epochs=a.epochs, log=log)
    pk.save(a.out)
    erng = S.rng_for(54321)
    mats = []
    for i in range(a.heldout):
        n = int(round(np.exp(erng.uniform(np.log(a.eval_lo), np.log(a.eval_hi)))))
        mats.append(lambda n=n, i=i: S.gen_mixture(n, 20_000 + i))
    rows, summary = evaluate(pk, mats, log=log, time_budget=a.eval_budget)
    report = {"train_matrices": used, "heldout_requested": a.heldout, "samples": int(X.shape[0]),
              "loss_history": hist, "summary": summary,
              "heldout": rows, "depths": DEPTHS}
    json.dump(report, open(a.report, "w"), indent=1)
    log(json.dumps(summary))
    return 0


if __name__ == "__main__":
    sys.exit(main())
