"""GPU parity of the rewrite path against the CPU oracle: plans identical, rewritten
coefficients identical in float64 (same operation order, round-to-nearest), levels of
the rewritten system identical, and the solve of the rewritten system within 1e-10."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S
from tests.gpu_util import TOL_F32, TOL_F64, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
KIND = {B.NAIVE: O.NAIVE, B.DEPTH_K: O.DEPTH, B.CHOSEN: O.CHOSEN, B.MANUAL: O.MANUAL, B.ROWCAP: O.ROWCAP,
        B.CHOSEN_THIN: O.CHOSEN_THIN}


def run_both(m, kind, b=None, k=0, cap=0.0, depth_of_target=None, exact=True, parts=1):
    torch = torch_cuda()
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    lev, mm = O.levels(m.rowptr, m.colidx)
    p = O.plan(m.rowptr, m.colidx, lev, mm, KIND[kind], k=k, cap=cap, depth_of_target=depth_of_target, parts=parts)
    sysm = B.System(M, lv, kind, k=k, cap=cap, depth_of_target=depth_of_target, walk_parts=parts)
    ex = sysm.export()
    # the plan
    assert np.array_equal(ex["target"], p.target)
    assert sysm.info["rows_moved"] == p.moved
    assert sysm.info["stored_nnz"] == p.stored_nnz
    # the rewritten equations
    sy = O.rewrite(m.rowptr, m.colidx, m.vals, lev, p.target)
    l2, m2 = sy.levels()
    assert sysm.m == m2 and np.array_equal(ex["level"], l2)
    assert np.array_equal(ex["cptr"], sy.cptr)
    assert np.array_equal(ex["ccol"], sy.ccol)
    rp = m.rowptr.astype(np.int64)
    diag = m.vals[rp[1:] - 1]
    moved_entry = np.repeat(sy.moved.astype(bool), np.diff(sy.cptr))
    rows_of_entry = np.repeat(np.arange(m.n), np.diff(sy.cptr))
    want_c = np.where(moved_entry, sy.cval, sy.cval / diag[rows_of_entry])
    if exact:
        assert np.array_equal(ex["cval"], want_c)
        assert np.array_equal(ex["dinv"], 1.0 / diag)
    else:
        assert np.allclose(ex["cval"], want_c, rtol=1e-6, atol=1e-7)
    # E rows: the oracle keeps the diagonal term in E, the library in dinv
    e_keep = sy.ecol != np.repeat(np.arange(m.n), np.diff(sy.eptr))
    ecnt = np.bincount(np.repeat(np.arange(m.n), np.diff(sy.eptr))[e_keep], minlength=m.n)
    assert np.array_equal(np.diff(ex["eptr"]), ecnt)
    assert np.array_equal(ex["ecol"], sy.ecol[e_keep])
    if exact:
        assert np.array_equal(ex["eval"], sy.eval[e_keep])
    if b is not None:
        vt = torch.float64 if M.dtype == B.F64 else torch.float32
        x = sysm.solve(torch.from_numpy(np.ascontiguousarray(b)).to("cuda", dtype=vt), check_status=True).cpu().numpy()
        ref = O.forward_subst(m.rowptr, m.colidx, m.vals, b)
        assert rel_l2(x, ref) <= (TOL_F64 if M.dtype == B.F64 else TOL_F32)
    return sysm, p


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("cap", [0.0, 1.5, 1.05])
def test_naive_plan_and_rewrite_config0(seed, cap):
    m, b, _ = S.gen_config("c0", seed=seed)
    run_both(m, B.NAIVE, b, cap=cap)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_depth_k_grid(k):
    m, b, _ = S.gen_config("c2", scale=0.02)
    s, _ = run_both(m, B.DEPTH_K, b, k=k)
    assert s.m == -(-(2 * int(np.sqrt(m.n)) - 1) // (k + 1))


@pytest.mark.parametrize("k", [1, 3])
def test_depth_k_with_cap_uses_the_walk(k):
    m, b, _ = S.gen_config("c2", scale=0.01)
    run_both(m, B.DEPTH_K, b, k=k, cap=1.3)


def test_chosen_depths_random():
    m = S.gen_skewed(6000, 2, head=4000)
    lev, mm = O.levels(m.rowptr, m.colidx)
    dot = np.random.default_rng(0).choice([0, 1, 2, 4, 8], size=mm)
    _, b = S.rhs_from_xtrue(m, 2, 3)
    run_both(m, B.CHOSEN, b, depth_of_target=dot)
    run_both(m, B.CHOSEN, b, depth_of_target=dot, cap=1.2)


@pytest.mark.parametrize("k", [8, 32])
@pytest.mark.parametrize("cap", [0.0, 1.5])
def test_rowcap_plan_matches_oracle(k, cap):
    """ROWCAP: plan, rewritten equations and solve identical to the oracle; every target
    keeps at most k rows."""
    m = S.gen_skewed(40000, 12, head=25000)
    _, b = S.rhs_from_xtrue(m, 1, 4)
    s, p = run_both(m, B.ROWCAP, b, k=k, cap=cap)
    lev, _ = O.levels(m.rowptr, m.colidx)
    moved = p.target != lev
    assert moved.any()
    assert np.bincount(p.target)[np.unique(p.target[moved])].max() <= k
    mx = S.gen_mixture(30000, 10003)
    _, b2 = S.rhs_from_xtrue(mx, 1, 5)
    run_both(mx, B.ROWCAP, b2, k=k, cap=cap)


def test_naive_skewed_small_and_mixture():
    m = S.gen_skewed(30000, 11, head=24000)
    _, b = S.rhs_from_xtrue(m, 1, 1)
    run_both(m, B.NAIVE, b, cap=1.5)
    mx = S.gen_mixture(20000, 10001)
    _, b2 = S.rhs_from_xtrue(mx, 1, 2)
    run_both(mx, B.NAIVE, b2)


def test_naive_config1_full_size():
    m, b, _ = S.gen_config("c1")
    s, p = run_both(m, B.NAIVE, b, cap=1.5)
    assert s.m == p.levels_after  # re-levelling keeps exactly the planned non-empty levels


@pytest.mark.parametrize("k", [1, 2, 4])
def test_depth_k_config2_full_size(k):
    m, b, _ = S.gen_config("c2")
    run_both(m, B.DEPTH_K, b, k=k)


def test_rewrite_multi_rhs_and_float32():
    m = S.gen_banded_random(8000, 4, k=5, band=60)
    b = S.rhs_uniform(m.n, 16, 5)
    run_both(m, B.DEPTH_K, b, k=3)
    m32 = m.astype(np.float32)
    run_both(m32, B.DEPTH_K, b.astype(np.float32), k=3, exact=False)


def test_costmap_example_on_gpu():
    torch = torch_cuda()
    g = json.load(open(os.path.join(GOLD, "costmap_example.json")))
    deps = {0: [], 1: [], 2: [0], 3: [1], 4: [2], 5: [2, 3], 6: [4], 7: [5]}
    n = 8
    counts = np.array([len(deps[i]) for i in range(n)])
    cols = np.array([c for i in range(n) for c in deps[i]], dtype=np.int64)
    m = S.gen_from_deps(n, counts, cols, S.rng_for(0))
    inj = np.array([g["cost_on_target"].get(str(i), g["original_row_cost"][str(i)]) for i in range(n)])
    M = B.Matrix.from_host(m)
    sysm = B.System(M, B.Levels(M), B.NAIVE, avg=g["avg_level_cost"],
                    injected_cost=torch.from_numpy(inj.astype(np.int64)).cuda())
    ex = sysm.export()
    assert ex["target"].tolist() == [g["expected_target"][str(i)] for i in range(n)]


@pytest.mark.parametrize("name", ["equality", "over", "zero"])
def test_naive_rewritten_row_cost_hand_derived_on_gpu(name):
    """The GPU planner's own cost of a rewritten row (2 |D'|, no injected cost, computed average)
    reproduces the hand-derived plans of tests/naive_cost_cases.py."""
    from tests.naive_cost_cases import CASES, csr_arrays, expected_target
    case = CASES[name]
    n, counts, cols = csr_arrays(case)
    m = S.gen_from_deps(n, np.array(counts), np.array(cols, dtype=np.int64), S.rng_for(3))
    _, b = S.rhs_from_xtrue(m, 1, 5)
    s, p = run_both(m, B.NAIVE, b)
    assert s.export()["target"].tolist() == expected_target(case)
    assert s.info["avg_cost"] == pytest.approx(case["avg"], abs=1e-9)


def test_growth_guard_trips_on_far_rewrite_of_small_pivots():
    torch_cuda()
    n = 40
    counts = np.array([0] + [1] * (n - 1))
    cols = np.arange(n - 1)
    m = S.gen_from_deps(n, counts, cols, None, offdiag=1.0, diag=1e-3)
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    with pytest.raises(B.SptrsvError) as e:
        B.System(M, lv, B.DEPTH_K, k=30, guard=1e12)
    assert e.value.code == B.ERR_NUMERIC
    B.System(M, lv, B.DEPTH_K, k=2, guard=1e12)  # short distance stays under the guard


def test_empty_and_degenerate():
    torch_cuda()
    # no dependencies at all: one level, nothing moves
    m = S.gen_from_deps(500, np.zeros(500, np.int64), np.zeros(0, np.int64), None, diag=2.0)
    s, p = run_both(m, B.NAIVE, S.rhs_uniform(500, 1, 0))
    assert p.moved == 0 and s.m == 1
    # a pure chain: depth-k groups collapse it
    n = 3000
    m = S.gen_from_deps(n, np.array([0] + [1] * (n - 1)), np.arange(n - 1), S.rng_for(3))
    s, _ = run_both(m, B.DEPTH_K, S.rhs_uniform(n, 1, 1), k=7)
    assert s.m == -(-n // 8)


@pytest.mark.parametrize("alpha,beta", [(3, 0), (0, 60), (5, 200)])
def test_per_row_rules_match_oracle(alpha, beta):
    torch = torch_cuda()
    m, b, _ = S.gen_config("c0", seed=4)
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    lev, mm = O.levels(m.rowptr, m.colidx)
    for kind, okind, k in ((B.NAIVE, O.NAIVE, 0), (B.DEPTH_K, O.DEPTH, 3)):
        p = O.plan(m.rowptr, m.colidx, lev, mm, okind, k=k, alpha=alpha, beta=beta)
        s = B.System(M, lv, kind, k=k, alpha=alpha, beta=beta)
        assert np.array_equal(s.export()["target"], p.target)
        x = s.solve(torch.from_numpy(b).cuda(), check_status=True).cpu().numpy()
        assert rel_l2(x, O.forward_subst(m.rowptr, m.colidx, m.vals, b)) <= TOL_F64


@pytest.mark.parametrize("cap", [0.0, 1.5])
@pytest.mark.parametrize("which", ["c0", "mixture"])
def test_chosen_thin_per_target_depths(which, cap):
    """Depth per target over thin levels (the learned strategy's plan family), with depths drawn per
    level, with and without the nnz cap (without it the targets map level by level)."""
    m = S.gen_config("c0")[0] if which == "c0" else S.gen_mixture(40_000, 10_321)
    _, b = S.rhs_from_xtrue(m, 1, 3)
    lev, mm = O.levels(m.rowptr, m.colidx)
    dot = S.rng_for(5).integers(0, 12, size=mm)
    run_both(m, B.CHOSEN_THIN, b, cap=cap, depth_of_target=dot)


def test_manual_without_cap_maps_levels():
    m = S.gen_mixture(30_000, 10_322)
    _, b = S.rhs_from_xtrue(m, 1, 4)
    for k in (2, 9):
        run_both(m, B.MANUAL, b, k=k)


@pytest.mark.parametrize("parts", [2, 7, 64])
@pytest.mark.parametrize("kind,k", [(B.NAIVE, 0), (B.ROWCAP, 32), (B.MANUAL, 9), (B.DEPTH_K, 3)])
def test_walk_started_at_several_places(kind, k, parts):
    """The planner walk started at the beginning of every level range (one warp per range at the same
    time; 2 ranges: from both ends), with and without the nnz cap: plans identical to the oracle's."""
    m = S.gen_mixture(60_000, 10_777)
    _, b = S.rhs_from_xtrue(m, 1, 6)
    for cap in (0.0, 1.5):
        run_both(m, kind, b, k=k, cap=cap, parts=parts)


def test_walk_parts_full_size_skewed():
    m, b, _ = S.gen_config("c1")
    run_both(m, B.ROWCAP, b, k=32, cap=1.5, parts=64)
