"""Table-I-style structural report (Section IV) on lung2- and torso2-shaped matrices.

For each matrix and strategy -- no rewriting, the naive avgLevelCost strategy, and the
manual approach (every 9 thin levels into the 10th) -- the report gives the number of
levels, the average and total level cost and the rows rewritten, with the paper's own
Table I numbers beside them for context (they come from the real SuiteSparse matrices,
which are not available; the shapes here only match their sizes and level profiles).
Costs follow Section III: an original row costs 2*nnz - 1, a rewritten (rearranged) row
2 * (its remaining dependencies).  Everything is computed by the library on the GPU.

Usage: python -m paper_2206_05843_gb300.table1 [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import statistics
import sys

import numpy as np

from . import binding as B
from . import synth as S

PAPER = {
    "lung2": {"none": {"levels": 479, "avg_cost": 914.054, "total_cost": 437834, "rows_rewritten": 0},
              "naive": {"levels": 23, "avg_cost": 18938.06, "total_cost": 435588, "rows_rewritten": 1304},
              "manual": {"levels": 67, "avg_cost": 6520.42, "total_cost": 436868, "rows_rewritten": 898}},
    "torso2": {"none": {"levels": 513, "avg_cost": 2014.559, "total_cost": 1035484, "rows_rewritten": 0},
               "naive": {"levels": 341, "avg_cost": 3086.443, "total_cost": 1052477, "rows_rewritten": 14655},
               "manual": {"levels": 284, "avg_cost": 5070.183, "total_cost": 1439932, "rows_rewritten": 18147}},
}


def structure(sysm, lv_level) -> dict:
    """Levels, level costs and rows rewritten of a stored system (export in the original
    numbering)."""
    ex = sysm.export()
    deps = np.diff(ex["cptr"])
    moved = ex["target"] < lv_level
    cost = np.where(moved, 2 * deps, 2 * (deps + 1) - 1)
    total = int(cost.sum())
    return {"levels": int(sysm.m), "avg_cost": total / max(1, sysm.m), "total_cost": total,
            "rows_rewritten": int(moved.sum())}


def report(seed: int = 0, time_solves: bool = True, scale: float = 1.0, picker=None) -> dict:
    """Structure (and solve time) of none / naive / manual -- and learned, when a trained
    picker is given (nnz cap 1.5) -- on the lung2- and torso2-shaped inputs."""
    import torch
    out = {}
    for name, gen in (("lung2", S.gen_lung2_like), ("torso2", S.gen_torso2_like)):
        m = gen(seed, scale)
        M = B.Matrix.from_host(m)
        lv = B.Levels(M)
        level = lv.export()["level"]
        b = torch.from_numpy(S.rhs_from_xtrue(m, 1, 3)[1][0]).cuda()
        rows = {}
        strategies = [("none", {}), ("naive", dict(kind=B.NAIVE)), ("manual", dict(kind=B.MANUAL, k=9))]
        if picker is not None:
            strategies.append(("learned", dict(kind=B.LEARNED, cap=1.5, picker=picker)))
        for strat, kw in strategies:
            s = B.System(M, lv, **kw)
            r = structure(s, level)
            if time_solves:
                x = torch.empty_like(b)
                s.solve(b, x)
                torch.cuda.synchronize()
                ts = []
                for _ in range(5):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    s.solve(b, x)
                    e1.record()
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1) * 1e3)
                s.status()
                r["solve_us"] = statistics.median(ts)
            r["paper"] = PAPER[name].get(strat)
            rows[strat] = r
        out[name] = {"n": m.n, "nnz": m.nnz, "rows": rows}
    return out


def format_table(rep: dict) -> str:
    lines = ["| matrix (shape of) | strategy | levels | avg level cost | total level cost | rows rewritten | solve us | paper: levels / avg / total / rewritten |",
             "|---|---|---|---|---|---|---|---|"]
    for name, d in rep.items():
        for strat, r in d["rows"].items():
            p = r["paper"]
            ref = (f"{p['levels']} / {p['avg_cost']} / {p['total_cost']:,} / {p['rows_rewritten']:,}" if p
                   else "not in the paper")
            lines.append(f"| {name} (n={d['n']:,}) | {strat} | {r['levels']} | {r['avg_cost']:.1f} | {r['total_cost']:,} | "
                         f"{r['rows_rewritten']:,} | {r.get('solve_us', float('nan')):.1f} | {ref} |")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--json", default=None)
    ap.add_argument("--picker", default=None, help="trained picker file: adds the learned strategy")
    a = ap.parse_args(argv)
    rep = report(picker=B.Picker.load(a.picker) if a.picker else None)
    print(format_table(rep))
    if a.json:
        json.dump(rep, open(a.json, "w"), indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
