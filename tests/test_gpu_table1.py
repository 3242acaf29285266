"""The Table-I-style report computed by the library equals the oracle's planner and
rewrite on the same lung2- / torso2-shaped matrices."""
import numpy as np
import pytest

import oracle as O
from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S
from paper_2206_05843_gb300 import table1
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def oracle_structure(m, kind, k=0):
    lev, mm = O.levels(m.rowptr, m.colidx)
    if kind is None:
        st = O.level_stats(m.rowptr, lev, mm)
        return {"levels": mm, "total_cost": int(st["cost"].sum()), "rows_rewritten": 0}
    p = O.plan(m.rowptr, m.colidx, lev, mm, kind, k=k)
    sy = O.rewrite(m.rowptr, m.colidx, m.vals, lev, p.target)
    _, m2 = sy.levels()
    return {"levels": m2, "total_cost": int(p.row_cost.sum()), "rows_rewritten": p.moved}


def test_table1_report_matches_oracle():
    torch_cuda()
    rep = table1.report(time_solves=False, scale=0.25)
    for name, gen in (("lung2", S.gen_lung2_like), ("torso2", S.gen_torso2_like)):
        m = gen(0, 0.25)
        for strat, (kind, k) in (("none", (None, 0)), ("naive", (O.NAIVE, 0)), ("manual", (O.MANUAL, 9))):
            want = oracle_structure(m, kind, k)
            got = rep[name]["rows"][strat]
            for key in ("levels", "total_cost", "rows_rewritten"):
                assert got[key] == want[key], (name, strat, key, got[key], want[key])
