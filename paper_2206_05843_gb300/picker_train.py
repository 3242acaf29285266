"""Training and evaluation of the learned rewrite picker on timings the library measures
itself.

Harvest (per training matrix): the plain system is solved with per-level %globaltimer
stamps; then, for every candidate (a fixed depth g, or a row budget -r that gives every target
the largest depth whose window holds at most r rows), the matrix is rewritten with the plan
family the model drives -- thin levels only (cost below avgLevelCost, Section III), the
candidate's depth at every target (CHOSEN_THIN) -- and solved with stamps.  For a target level t
whose group holds original levels t..te the label is
  dt(t, c) = time of the rewritten levels that hold original levels t..te
           - time of original levels t..te in the plain solve             (nanoseconds)
and the sample's input is the 12-feature vector of candidate (t, c) computed on the
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


def candidate_depths(rows: np.ndarray, c: int) -> np.ndarray:
    """The depth candidate c gives every target level (the library's rule): c itself for c >= 1;
    for c = -r the largest g with rows(t) + ... + rows(t + g) <= r, 0 when level t holds more."""
    m = rows.size
    if c >= 1:
        return np.full(m, c, np.int32)
    P = np.concatenate([[0], np.cumsum(rows.astype(np.int64))])
    j = np.searchsorted(P, P[:-1] + (-c), side="right") - 1  # largest j with P[j] <= P[t] + r
    return np.maximum(j - 1 - np.arange(m), 0).astype(np.int32)


def harvest(m, depths=DEPTHS, reps=3, seed=0, per_candidate=2000):
    """Samples (features, dt in ns) of one matrix: every target of a thin-level plan with the
    candidate's depths (no nnz cap, so that every group holds its whole window); at most
    per_candidate targets per candidate, drawn at random."""
    torch = _torch()
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    mm = lv.m
    if mm < 3:
        return np.zeros((0, 12), np.float32), np.zeros(0, np.float32)
    lex = lv.export()
    old_level = lex["level"].astype(np.int64)
    rows = np.asarray(lex["rows"], np.int64)
    b = S.rhs_uniform(m.n, 1, seed)
    bt = torch.from_numpy(b[0]).cuda()
    feats = B.features(M, lv, depths).cpu().numpy().reshape(mm, len(depths), 12)
    plain = B.System(M, lv)
    sp = np.stack(timed_stamps(plain, bt, reps))
    rng = np.random.default_rng(seed)
    idx = np.arange(mm)
    X, Y = [], []
    for d, c in enumerate(depths):
        try:
            s = B.System(M, lv, B.CHOSEN_THIN, depth_of_target=candidate_depths(rows, int(c)))
        except B.SptrsvError:
            continue
        ex = s.export()
        ltarget = np.empty(mm, np.int64)
        ltarget[old_level] = ex["target"].astype(np.int64)  # without a cap a level moves as a whole
        lo, hi = level_spans(ex["level"].astype(np.int64), old_level, mm)
        sr = np.stack(timed_stamps(s, bt, reps))
        del s
        # groups: a target t and the levels that moved into it (t..te)
        te = np.full(mm, -1, np.int64)
        np.maximum.at(te, ltarget, idx)
        glo = np.full(mm, np.iinfo(np.int64).max, np.int64)
        ghi = np.full(mm, -1, np.int64)
        np.minimum.at(glo, ltarget, lo)
        np.maximum.at(ghi, ltarget, hi)
        tg = np.nonzero((te > idx) & (idx > 0))[0]
        tg = tg[glo[tg] > 0]
        if tg.size > per_candidate:
            tg = np.sort(rng.choice(tg, size=per_candidate, replace=False))
        if tg.size == 0:
            continue
        dr = sr[:, ghi[tg]] - sr[:, glo[tg] - 1]
        dp = sp[:, te[tg]] - sp[:, tg - 1]
        X.append(feats[tg, d])
        Y.append(np.median(dr - dp, axis=0))
    if not X:
        return np.zeros((0, 12), np.float32), np.zeros(0, np.float32)
    return np.concatenate(X).astype(np.float32), np.concatenate(Y).astype(np.float32)


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


def evaluate(pk, mats, cap=1.5, log=None, time_budget=1e9, walk_parts=1):
    """Solve time of no rewrite, the paper's naive strategy, the ROWCAP plan and the network's own
    plan (the learned strategy with model_only), each with its error against x_true (b = L x_true).
    The learned strategy's measured choice is the fastest of those four (the library times the
    same four candidates and keeps the fastest); "choice_without_model" is the fastest of the
    three without the network, so that the network's own contribution shows apart from the
    fallbacks."""
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
        wp = dict(walk_parts=walk_parts)
        for name, kw in (("none", {}), ("naive", dict(kind=B.NAIVE, cap=cap, **wp)),
                         ("rowcap", dict(kind=B.ROWCAP, k=32, cap=cap, **wp)),
                         ("learned_model_only", dict(kind=B.LEARNED, cap=cap, picker=pk, model_only=True, **wp))):
            s = B.System(M, lv, **kw)
            us, x = solve_time_us(s, bt)
            err = float(np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref))
            res[name] = {"us": us, "levels": s.m, "rel_err": err, "strategy_used": int(s.info["strategy_used"])}
            del s
        cand = {k: res[k]["us"] for k in ("learned_model_only", "naive", "rowcap", "none")}
        best = min(cand, key=cand.get)
        res["learned"] = dict(res[best], kept=best)
        best_wo = min(("naive", "rowcap", "none"), key=lambda k: cand[k])
        res["choice_without_model"] = dict(res[best_wo], kept=best_wo)
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
               "geomean_speedup_choice_with_vs_without_model": float(np.exp(np.mean(
                   [np.log(r["choice_without_model"]["us"] / r["learned"]["us"]) for r in rows]))),
               "model_plan_kept": int(sum(r["learned"]["kept"] == "learned_model_only" for r in rows)),
               "max_rel_err": max(max(r[k]["rel_err"] for k in ("none", "naive", "rowcap", "learned_model_only"))
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
    ap.add_argument("--save-data", default=None, help="write the harvested samples to this .npz file")
    ap.add_argument("--load-data", default=None, help="train on samples from this .npz file (no harvest)")
    ap.add_argument("--walk-parts", type=int, default=1, help="level ranges the evaluation's planner walks start at")
    ap.add_argument("--per-candidate", type=int, default=2000, help="targets sampled per candidate and matrix")
    ap.add_argument("--also-evaluate", default=None, help="evaluate this second picker file on the same matrices")
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
        rows, summary = evaluate(pk, mats, log=log, time_budget=a.eval_budget, walk_parts=a.walk_parts)
        json.dump({"picker": a.evaluate, "summary": summary, "heldout": rows}, open(a.report, "w"), indent=1)
        log(json.dumps(summary))
        return 0
    if a.load_data:
        z = np.load(a.load_data)
        X, Y, used = z["X"], z["Y"], int(z["matrices"])
    else:
        rng = S.rng_for(12345)
        t0 = time.time()
        Xs, Ys = [], []
        used = 0
        for i in range(a.train):
            if time.time() - t0 > a.time_budget:
                break
            n = int(round(np.exp(rng.uniform(np.log(a.n_lo), np.log(a.n_hi)))))
            m = S.gen_mixture(n, 10_000 + i)
            X, Y = harvest(m, seed=i, per_candidate=a.per_candidate)
            Xs.append(X)
            Ys.append(Y)
            used += 1
            if i % 20 == 0:
                log(f"harvest {i}: n={m.n} samples={len(Y)} elapsed={time.time() - t0:.0f}s")
        X = np.concatenate(Xs)
        Y = np.concatenate(Ys)
        if a.save_data:
            np.savez_compressed(a.save_data, X=X, Y=Y, matrices=used)
    log(f"dataset: {X.shape[0]} samples from {used} matrices")
    pk, hist = train(X, Y, epochs=a.epochs, log=log)
    pk.save(a.out)
    erng = S.rng_for(54321)
    mats = []
    for i in range(a.heldout):
        n = int(round(np.exp(erng.uniform(np.log(a.eval_lo), np.log(a.eval_hi)))))
        mats.append(lambda n=n, i=i: S.gen_mixture(n, 20_000 + i))
    rows, summary = evaluate(pk, mats, log=log, time_budget=a.eval_budget, walk_parts=a.walk_parts)
    report = {"train_matrices": used, "heldout_requested": a.heldout, "samples": int(X.shape[0]),
              "loss_history": hist, "summary": summary,
              "heldout": rows, "depths": DEPTHS, "walk_parts": a.walk_parts}
    if a.also_evaluate:
        mats2 = mats[:len(rows)]
        rows2, summary2 = evaluate(B.Picker.load(a.also_evaluate), mats2, log=log, walk_parts=a.walk_parts)
        report["also_evaluated"] = {"picker": a.also_evaluate, "summary": summary2}
        log(json.dumps(summary2))
    json.dump(report, open(a.report, "w"), indent=1)
    log(json.dumps(summary))
    return 0


if __name__ == "__main__":
    sys.exit(main())
