"""Feature oracle of the learned rewrite picker -- TEST INFRASTRUCTURE ONLY.

Twelve numbers describe the candidate "rewrite the g levels after level t into t"
(Section III: the target level, the source levels, the rewriting distance, and the
constraints the paper lists -- thin levels, in-degrees, the growth of the rewritten
rows and the neighbouring levels).  Window W = levels t..te with te = min(t+g, m-1),
source levels S = t+1..te.  Per level: rows, nnz (diagonal included), cost
2*nnz - rows, the largest in-degree of a row, and the two-hop count
sum over rows r of sum over dependencies j of indeg(j) (an upper bound of the
dependencies after one substitution).

  f0  log2(1 + g)
  f1  log2(1 + rows(W))
  f2  log2(1 + nnz(W))
  f3  log2(1 + rows(S) / max(1, te - t))
  f4  (nnz(S) - rows(S)) / max(1, rows(S))      mean in-degree of the source rows
  f5  max in-degree over S (0 without sources)
  f6  log2(1 + two-hop(S))
  f7  log2(1 + rows(t))
  f8  log2(1 + rows(t-1)), 0 for t = 0
  f9  log2(1 + rows(te+1)), 0 past the last level
  f10 cost(W) / avgLevelCost
  f11 fraction of levels of W with cost < avgLevelCost (thin levels)
Computed in float64 and returned as float32.

A candidate is a depth g >= 1, or a row budget given as a negative entry -r: then g is the
largest depth whose window t..t+g holds at most r rows (0 when level t alone holds more), and
the candidate's features are those of that window (a target that takes the following levels
while it holds at most r rows, the row-capped strategy at the granularity of whole levels).
"""
from __future__ import annotations

import numpy as np

import oracle as O


def level_aggregates(rowptr, colidx):
    rp = np.asarray(rowptr, dtype=np.int64)
    ci = np.asarray(colidx, dtype=np.int64)
    lev, m = O.levels(rowptr, colidx)
    n = rp.size - 1
    indeg = np.diff(rp) - 1
    rows = np.zeros(m, np.int64)
    nnz = np.zeros(m, np.int64)
    maxdeg = np.zeros(m, np.int64)
    twohop = np.zeros(m, np.int64)
    for i in range(n):
        lv = lev[i]
        rows[lv] += 1
        nnz[lv] += indeg[i] + 1
        if indeg[i] > maxdeg[lv]:
            maxdeg[lv] = indeg[i]
        deps = ci[rp[i]:rp[i + 1] - 1]
        twohop[lv] += int(indeg[deps].sum())
    cost = 2 * nnz - rows
    return {"level": lev, "m": m, "rows": rows, "nnz": nnz, "cost": cost, "maxdeg": maxdeg, "twohop": twohop}


def candidate_depth(rows, t, c) -> int:
    """Depth of candidate c at target t: c itself when c >= 1; for c = -r the largest g with
    rows(t) + ... + rows(t + g) <= r (t + g < m), found by adding levels one at a time."""
    if c >= 1:
        return int(c)
    r, g, held = -int(c), 0, int(rows[t])
    if held > r:
        return 0
    while t + g + 1 < len(rows) and held + int(rows[t + g + 1]) <= r:
        g += 1
        held += int(rows[t + g])
    return g


def features(rowptr, colidx, depths) -> np.ndarray:
    """Array (m * len(depths), 12), row t * len(depths) + d for candidate (t, depths[d])."""
    a = level_aggregates(rowptr, colidx)
    m = a["m"]
    rows, nnz, cost, maxdeg, two = a["rows"], a["nnz"], a["cost"], a["maxdeg"], a["twohop"]
    avg = cost.sum() / m
    out = np.zeros((m * len(depths), 12), dtype=np.float64)
    for t in range(m):
        for d, c in enumerate(depths):
            g = candidate_depth(rows, t, c)
            te = min(t + g, m - 1)
            W = slice(t, te + 1)
            S = slice(t + 1, te + 1)
            rS = rows[S].sum()
            f = out[t * len(depths) + d]
            f[0] = np.log2(1 + g)
            f[1] = np.log2(1 + rows[W].sum())
            f[2] = np.log2(1 + nnz[W].sum())
            f[3] = np.log2(1 + rS / max(1, te - t))
            f[4] = (nnz[S].sum() - rS) / max(1, rS)
            f[5] = maxdeg[S].max() if te > t else 0
            f[6] = np.log2(1 + two[S].sum())
            f[7] = np.log2(1 + rows[t])
            f[8] = np.log2(1 + rows[t - 1]) if t > 0 else 0.0
            f[9] = np.log2(1 + rows[te + 1]) if te + 1 < m else 0.0
            f[10] = cost[W].sum() / avg
            f[11] = np.count_nonzero(cost[W] < avg) / (te - t + 1)
    return out.astype(np.float32)
