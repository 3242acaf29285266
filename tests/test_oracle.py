"""Pins for the CPU oracle: it is checked against things other than itself.

Forward substitution: library triangular solves, b = L x_true recovery, closed forms.
Level sets: brute-force longest paths on tiny DAGs, the grid's closed form r + c.
Rewriting: the worked example of Section II.B / Fig. 2, the elimination identity
L' = E L (a dense matrix product), the grid's binomial closed form, and x' = x.
Planner: the costMap example of Section III with the paper's costs injected.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as O
from paper_2206_05843_gb300 import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def small_random_lower(n, density, seed, dominant=True):
    rng = np.random.default_rng(seed)
    counts, cols = [], []
    for i in range(n):
        c = np.nonzero(rng.random(i) < density)[0]
        counts.append(len(c))
        cols.extend(c.tolist())
    m = S.gen_from_deps(n, np.array(counts), np.array(cols, dtype=np.int64), S.rng_for(seed))
    if not dominant:
        rp = m.rowptr.astype(np.int64)
        m.vals[rp[1:] - 1] = rng.uniform(0.5, 2.0, n) * rng.choice([-1, 1], n)
    return m


# ---------------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n", [1, 7, 33, 64])
def test_forward_subst_matches_library_triangular_solve(n, seed):
    m = small_random_lower(n, 0.3, seed, dominant=(seed % 2 == 0))
    L = m.to_dense()
    b = np.random.default_rng(seed + 100).uniform(-1, 1, size=(3, n))
    x = O.forward_subst(m.rowptr, m.colidx, m.vals, b)
    ref = scipy.linalg.solve_triangular(L, b.T, lower=True).T
    ref2 = np.linalg.solve(L, b.T).T
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(x - ref).max() <= 1e-12 * scale
    assert np.abs(x - ref2).max() <= 1e-9 * scale


def test_forward_subst_recovers_x_true_config0():
    m, b, xt = S.gen_config("c0")
    x = O.forward_subst(m.rowptr, m.colidx, m.vals, b)
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) < 1e-14


def test_forward_subst_closed_forms():
    n = 50
    rng = np.random.default_rng(3)
    b = rng.uniform(-1, 1, n)
    # identity
    ident = S.gen_from_deps(n, np.zeros(n, np.int64), np.zeros(0, np.int64), None, diag=1.0)
    assert np.array_equal(O.forward_subst(ident.rowptr, ident.colidx, ident.vals, b), b)
    # diagonal
    d = rng.uniform(0.5, 3.0, n)
    diag = S.gen_from_deps(n, np.zeros(n, np.int64), np.zeros(0, np.int64), None, diag=d)
    assert np.allclose(O.forward_subst(diag.rowptr, diag.colidx, diag.vals, b), b / d, rtol=1e-15, atol=0)
    # bidiagonal: x_i - a x_{i-1} = b_i  ->  x_i = sum_{k<=i} a^{i-k} b_k
    a = 0.7
    counts = np.array([0] + [1] * (n - 1))
    cols = np.arange(n - 1)
    bi = S.gen_from_deps(n, counts, cols, None, offdiag=-a, diag=1.0)
    x = O.forward_subst(bi.rowptr, bi.colidx, bi.vals, b)
    closed = np.array([sum(a ** (i - k) * b[k] for k in range(i + 1)) for i in range(n)])
    assert np.allclose(x, closed, rtol=1e-12, atol=1e-13)


def test_validate_codes():
    m = small_random_lower(10, 0.4, 0)
    assert O.validate(m.rowptr, m.colidx, m.vals) == (0, -1)
    v = m.vals.copy()
    v[m.rowptr[4] + (m.rowptr[5] - m.rowptr[4]) - 1] = 0.0
    assert O.validate(m.rowptr, m.colidx, v) == (5, 4)
    c = m.colidx.copy()
    c[m.rowptr[6] - 1] = 2  # diagonal of row 5 replaced
    code, row = O.validate(m.rowptr, c, m.vals)
    assert code in (3, 4) and row == 5


# ---------------------------------------------------------------------------------
# level sets
# ---------------------------------------------------------------------------------

def brute_levels(n, deps):
    """Longest path (in edges) ending at each node, by enumerating every path."""
    best = [0] * n
    preds = {i: deps[i] for i in range(n)}
    # enumerate all paths backwards from every node
    for end in range(n):
        stack = [(end, 0)]
        while stack:
            node, length = stack.pop()
            if length > best[end]:
                best[end] = length
            for p in preds[node]:
                stack.append((p, length + 1))
    return best


@pytest.mark.parametrize("seed", range(20))
def test_levels_brute_force_longest_path(seed):
    n = 12
    m = small_random_lower(n, 0.35, seed)
    rp = m.rowptr.astype(np.int64)
    deps = {i: m.colidx[rp[i]:rp[i + 1] - 1].tolist() for i in range(n)}
    lev, mm = O.levels(m.rowptr, m.colidx)
    assert lev.tolist() == brute_levels(n, deps)
    assert mm == max(brute_levels(n, deps)) + 1


def test_levels_networkx_critical_path():
    nx = pytest.importorskip("networkx")
    m = small_random_lower(200, 0.05, 11)
    rp = m.rowptr.astype(np.int64)
    g = nx.DiGraph()
    g.add_nodes_from(range(m.n))
    for i in range(m.n):
        for j in m.colidx[rp[i]:rp[i + 1] - 1]:
            g.add_edge(int(j), i)
    _, mm = O.levels(m.rowptr, m.colidx)
    assert mm == nx.dag_longest_path_length(g) + 1


@pytest.mark.parametrize("side", [1, 2, 5, 17, 64])
def test_levels_laplacian_closed_form(side):
    m = S.gen_laplacian(side)
    lev, mm = O.levels(m.rowptr, m.colidx)
    r, c = np.divmod(np.arange(m.n), side)
    assert np.array_equal(lev, r + c)
    assert mm == 2 * side - 1
    st = O.level_stats(m.rowptr, lev, mm)
    ell = np.arange(mm)
    assert np.array_equal(st["rows"], np.minimum(ell + 1, 2 * side - 1 - ell))
    # cost of a level is 2 * sum(nnz) - rows (Section III)
    assert st["cost"].sum() == 2 * m.nnz - m.n


def test_levels_redblack_two_levels():
    m = S.gen_redblack(16)
    lev, mm = O.levels(m.rowptr, m.colidx)
    assert mm == 2 and (lev == 0).sum() == 128


def test_levels_layered():
    m = S.gen_layered(5, 300, 2)
    lev, mm = O.levels(m.rowptr, m.colidx)
    assert mm == 5 and np.array_equal(lev, np.arange(m.n) // 300)


# ---------------------------------------------------------------------------------
# rewriting (Section II.B)
# ---------------------------------------------------------------------------------

def fig2_matrix(seed=0):
    g = json.load(open(os.path.join(GOLD, "fig2_worked_example.json")))
    n = g["n"]
    counts = np.array([len(g["deps"][str(i)]) for i in range(n)])
    cols = np.array([c for i in range(n) for c in g["deps"][str(i)]], dtype=np.int64)
    rng = np.random.default_rng(seed)
    off = rng.uniform(-2, 2, cols.size)
    diag = rng.uniform(0.5, 2.0, n)
    return g, S.gen_from_deps(n, counts, cols, None, offdiag=off, diag=diag)


@pytest.mark.parametrize("seed", range(5))
def test_rewrite_worked_example_closed_form(seed):
    g, m = fig2_matrix(seed)
    lev, mm = O.levels(m.rowptr, m.colidx)
    assert lev.tolist() == g["levels_before"]
    L = m.to_dense()
    b = np.random.default_rng(seed + 9).uniform(-1, 1, 4)
    # twice: x3 = (b3 - L31 * ((b1 - L10 * (b0 / L00)) / L11)) / L33
    tgt = lev.copy()
    tgt[3] = g["rewrite_twice"]["target_level"]
    sy = O.rewrite(m.rowptr, m.colidx, m.vals, lev, tgt)
    assert sy.ccol[sy.cptr[3]:sy.cptr[4]].tolist() == g["rewrite_twice"]["deps_after"]
    x3 = (b[3] - L[3, 1] * ((b[1] - L[1, 0] * (b[0] / L[0, 0])) / L[1, 1])) / L[3, 3]
    assert sy.solve(b)[3] == pytest.approx(x3, rel=1e-14, abs=1e-15)
    # rearranged: b'_3 = sum_m e_3m b_m with the constants folded; dval = 1 (no division)
    e = dict(zip(sy.ecol[sy.eptr[3]:sy.eptr[4]].tolist(), sy.eval[sy.eptr[3]:sy.eptr[4]].tolist()))
    assert sy.dval[3] == 1.0
    assert e[3] == pytest.approx(1 / L[3, 3], rel=1e-15)
    assert e[1] == pytest.approx(-L[3, 1] / (L[1, 1] * L[3, 3]), rel=1e-14)
    assert e[0] == pytest.approx(L[3, 1] * L[1, 0] / (L[0, 0] * L[1, 1] * L[3, 3]), rel=1e-14)
    # once (middle graph of Fig. 2): row 3 now depends on row 0
    tgt = lev.copy()
    tgt[3] = g["rewrite_once"]["target_level"]
    sy1 = O.rewrite(m.rowptr, m.colidx, m.vals, lev, tgt)
    assert sy1.ccol[sy1.cptr[3]:sy1.cptr[4]].tolist() == g["rewrite_once"]["deps_after"]
    c30 = sy1.cval[sy1.cptr[3]]
    # x3 = (b3 - L31 (b1 - L10 x0) / L11) / L33  ->  coefficient of x0 is -L31 L10 / (L11 L33)
    assert -c30 == pytest.approx(L[3, 1] * L[1, 0] / (L[1, 1] * L[3, 3]), rel=1e-14)
    l2, m2 = sy1.levels()
    assert l2[3] == 1 and m2 == 2


def dense_system(sy: O.System, n):
    """Rows of the rewritten equations as dense [A | F] with A x = F b."""
    A = np.zeros((n, n))
    F = np.zeros((n, n))
    for r in range(n):
        A[r, r] = sy.dval[r]
        A[r, sy.ccol[sy.cptr[r]:sy.cptr[r + 1]]] += sy.cval[sy.cptr[r]:sy.cptr[r + 1]]
        if sy.moved[r]:
            F[r, sy.ecol[sy.eptr[r]:sy.eptr[r + 1]]] = sy.eval[sy.eptr[r]:sy.eptr[r + 1]]
        else:
            F[r, r] = 1.0
    return A, F


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("kind,k", [(O.DEPTH, 1), (O.DEPTH, 3), (O.NAIVE, 0)])
def test_rewrite_is_elimination_E_times_L(seed, kind, k):
    """Every rewritten row is a combination of original rows: A = F L, where the columns
    the rewrite removed become (numerically) zero."""
    m = small_random_lower(60, 0.08, seed)
    lev, mm = O.levels(m.rowptr, m.colidx)
    check_elimination(m, lev, mm, O.plan(m.rowptr, m.colidx, lev, mm, kind, k=k), seed)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("kind", ["manual", "chosen", "chosen_thin", "rowcap", "rowcap_cap"])
def test_rewrite_is_elimination_for_every_planner(seed, kind):
    """The same identities for the other planners: MANUAL, per-target depths (all levels or
    thin levels only) and ROWCAP, with and without the nnz cap."""
    m = small_random_lower(80, 0.06, seed + 100)
    lev, mm = O.levels(m.rowptr, m.colidx)
    dot = np.random.default_rng(seed).integers(0, 6, mm).astype(np.int32)
    p = {"manual": lambda: O.plan(m.rowptr, m.colidx, lev, mm, O.MANUAL, k=3),
         "chosen": lambda: O.plan(m.rowptr, m.colidx, lev, mm, O.CHOSEN, depth_of_target=dot),
         "chosen_thin": lambda: O.plan(m.rowptr, m.colidx, lev, mm, O.CHOSEN_THIN, depth_of_target=dot),
         "rowcap": lambda: O.plan(m.rowptr, m.colidx, lev, mm, O.ROWCAP, k=6),
         "rowcap_cap": lambda: O.plan(m.rowptr, m.colidx, lev, mm, O.ROWCAP, k=6, cap=1.2)}[kind]()
    check_elimination(m, lev, mm, p, seed)
    if kind == "rowcap_cap":
        assert p.stored_nnz <= 1.2 * p.nnz_l


def check_elimination(m, lev, mm, p, seed):
    L = m.to_dense()
    sy = O.rewrite(m.rowptr, m.colidx, m.vals, lev, p.target)
    A, F = dense_system(sy, m.n)
    assert np.allclose(F @ L, A, rtol=0, atol=1e-13)
    # no dependency on a row of the same or a later level after re-levelling
    l2, m2 = sy.levels()
    for r in range(m.n):
        deps = sy.ccol[sy.cptr[r]:sy.cptr[r + 1]]
        assert np.all(l2[deps] < l2[r])
        if sy.moved[r]:
            assert np.all(p.target[deps] < p.target[r])
    assert m2 <= p.levels_after <= mm
    b = np.random.default_rng(seed).uniform(-1, 1, (2, m.n))
    assert np.allclose(sy.solve(b), O.forward_subst(m.rowptr, m.colidx, m.vals, b), rtol=0, atol=1e-13)
    # dominant input: rearranged coefficients stay below one in magnitude
    assert np.abs(sy.cval[np.repeat(sy.moved.astype(bool), np.diff(sy.cptr))]).max(initial=0) < 1
    assert np.abs(sy.eval).max(initial=0) <= 1


@pytest.mark.parametrize("k", [1, 2, 4])
def test_rewrite_laplacian_binomial_closed_form(k):
    """Grid rows at depth d inside a group: x = sum over the cone of b with weight
    C(e, a) / 4^(e+1) at distance e, minus the d+2 points one level above the target with
    weight C(d+1, a) / 4^(d+1) (each step back goes up or left with weight 1/4)."""
    side = 14
    m = S.gen_laplacian(side)
    lev, mm = O.levels(m.rowptr, m.colidx)
    p = O.plan(m.rowptr, m.colidx, lev, mm, O.DEPTH, k=k)
    sy = O.rewrite(m.rowptr, m.colidx, m.vals, lev, p.target)
    checked = 0
    for idx in range(m.n):
        r, c = divmod(idx, side)
        d = lev[idx] - p.target[idx]
        if d == 0 or r < d + 2 or c < d + 2:
            continue  # unmoved or touching the boundary
        cdict = dict(zip(sy.ccol[sy.cptr[idx]:sy.cptr[idx + 1]].tolist(),
                         sy.cval[sy.cptr[idx]:sy.cptr[idx + 1]].tolist()))
        want_c = {(r - a) * side + (c - (d + 1 - a)): -math.comb(d + 1, a) / 4 ** (d + 1) for a in range(d + 2)}
        assert set(cdict) == set(want_c)
        for key, v in want_c.items():
            assert cdict[key] == pytest.approx(v, rel=1e-14)
        edict = dict(zip(sy.ecol[sy.eptr[idx]:sy.eptr[idx + 1]].tolist(),
                         sy.eval[sy.eptr[idx]:sy.eptr[idx + 1]].tolist()))
        want_e = {}
        for e in range(d + 1):
            for a in range(e + 1):
                want_e[(r - a) * side + (c - (e - a))] = math.comb(e, a) / 4 ** (e + 1)
        assert set(edict) == set(want_e)
        for key, v in want_e.items():
            assert edict[key] == pytest.approx(v, rel=1e-14)
        checked += 1
    assert checked > 20


def test_rewrite_far_with_tiny_pivots_blows_up():
    """Fig. 3: rewriting far over rows with small pivots produces huge constants."""
    n = 12
    counts = np.array([0] + [1] * (n - 1))
    cols = np.arange(n - 1)
    m = S.gen_from_deps(n, counts, cols, None, offdiag=1.0, diag=1e-3)
    lev, mm = O.levels(m.rowptr, m.colidx)
    tgt = np.zeros(n, np.int32)
    sy = O.rewrite(m.rowptr, m.colidx, m.vals, lev, tgt)
    assert np.abs(sy.eval).max() > 1e30


# ---------------------------------------------------------------------------------
# the planner (Section III)
# ---------------------------------------------------------------------------------

def test_planner_costmap_example():
    g = json.load(open(os.path.join(GOLD, "costmap_example.json")))
    # structure giving the example's levels and original costs (2 nnz -> 3, 3 nnz -> 5)
    deps = {0: [], 1: [], 2: [0], 3: [1], 4: [2], 5: [2, 3], 6: [4], 7: [5]}
    n = 8
    counts = np.array([len(deps[i]) for i in range(n)])
    cols = np.array([c for i in range(n) for c in deps[i]], dtype=np.int64)
    m = S.gen_from_deps(n, counts, cols, S.rng_for(0))
    lev, mm = O.levels(m.rowptr, m.colidx)
    assert [sorted(np.nonzero(lev == l)[0].tolist()) for l in range(mm)] == g["levels"]
    st = O.level_stats(m.rowptr, lev, mm)
    oc = g["original_row_cost"]
    assert [int(v) for v in st["cost"]] == [sum(oc[str(r)] for r in rows) for rows in g["levels"]]
    inj = np.array([g["cost_on_target"].get(str(i), g["original_row_cost"][str(i)]) for i in range(n)])
    p = O.plan(m.rowptr, m.colidx, lev, mm, O.NAIVE, avg=g["avg_level_cost"], injected_cost=inj)
    assert p.target.tolist() == [g["expected_target"][str(i)] for i in range(n)]
    for lvl, cost in g["expected_level_cost"].items():
        assert int(p.row_cost[p.target == int(lvl)].sum()) == cost
    assert mm - p.levels_after == g["expected_levels_removed"]


def test_planner_naive_fat_level_breaks_run_and_avg_is_fixed():
    # chain of single rows with one very wide level in the middle
    n_chain = 6
    counts, cols = [], []
    for i in range(n_chain):
        counts.append(1 if i else 0)
        cols.extend([i - 1] if i else [])
    wide = 40
    for w in range(wide):
        counts.append(1)
        cols.append(n_chain - 1)
    base = n_chain + wide
    for i in range(base, base + n_chain):
        counts.append(1)
        cols.append(i - 1 if i > base else n_chain + wide - 1)
    n = base + n_chain
    m = S.gen_from_deps(n, np.array(counts), np.array(cols, dtype=np.int64), S.rng_for(1))
    lev, mm = O.levels(m.rowptr, m.colidx)
    p = O.plan(m.rowptr, m.colidx, lev, mm, O.NAIVE)
    st = O.level_stats(m.rowptr, lev, mm)
    assert p.avg == pytest.approx(st["cost"].sum() / mm, abs=1e-6)
    wide_level = lev[n_chain]
    assert np.all(p.target[n_chain:base] == wide_level)  # fat level keeps its rows
    assert np.all(p.target[:n_chain] < wide_level)
    assert np.all(p.target[base:] > wide_level)
    assert p.levels_after < mm


def test_planner_depth_k_group_counts():
    m = S.gen_laplacian(32)
    lev, mm = O.levels(m.rowptr, m.colidx)
    for k in (1, 2, 4):
        p = O.plan(m.rowptr, m.colidx, lev, mm, O.DEPTH, k=k)
        assert p.levels_after == math.ceil(mm / (k + 1))
        assert np.array_equal(p.target, lev - lev % (k + 1))


def test_planner_nnz_cap_is_respected():
    m, b, _ = S.gen_config("c1", scale=0.01)
    lev, mm = O.levels(m.rowptr, m.colidx)
    for cap in (1.05, 1.2, 1.5):
        p = O.plan(m.rowptr, m.colidx, lev, mm, O.NAIVE, cap=cap)
        assert p.stored_nnz <= math.floor(cap * p.nnz_l)
        sy = O.rewrite(m.rowptr, m.colidx, m.vals, lev, p.target)
        stored = int(sy.cptr[-1]) + m.n + int(sy.eptr[-1])
        assert stored == p.stored_nnz  # planner bookkeeping equals the rewrite's structure


def test_planner_chosen_depths_equal_depth_k():
    m = S.gen_laplacian(20)
    lev, mm = O.levels(m.rowptr, m.colidx)
    p1 = O.plan(m.rowptr, m.colidx, lev, mm, O.DEPTH, k=3)
    p2 = O.plan(m.rowptr, m.colidx, lev, mm, O.CHOSEN, depth_of_target=np.full(mm, 3))
    assert np.array_equal(p1.target, p2.target)
    p0 = O.plan(m.rowptr, m.colidx, lev, mm, O.CHOSEN, depth_of_target=np.zeros(mm))
    assert np.array_equal(p0.target, lev)


@pytest.mark.parametrize("seed", range(4))
def test_backward_subst_matches_library(seed):
    """Upper-triangular solve (the second half of an ILU preconditioner, Section I)."""
    n = 40
    m = small_random_lower(n, 0.2, seed)
    Lt = m.to_dense().T.copy()  # an upper-triangular matrix
    rp, ci, va = [0], [], []
    for i in range(n):
        cols = np.nonzero(Lt[i])[0]
        cols = np.concatenate([[i], cols[cols > i]])
        ci.extend(cols.tolist())
        va.extend(Lt[i, cols].tolist())
        rp.append(len(ci))
    b = np.random.default_rng(seed).uniform(-1, 1, n)
    x = O.backward_subst(np.array(rp), np.array(ci), np.array(va), b)
    assert np.allclose(x, scipy.linalg.solve_triangular(Lt, b, lower=False), rtol=1e-12, atol=1e-14)


def test_planner_manual_is_depth_over_thin_levels():
    """MANUAL (Section IV: every 9 thin levels into the 10th) equals DEPTH on a matrix
    whose levels are all thin, and leaves fat levels alone."""
    n = 400
    chain = S.gen_from_deps(n, np.array([0] + [1] * (n - 1)), np.arange(n - 1), S.rng_for(2))
    lev, mm = O.levels(chain.rowptr, chain.colidx)
    # a uniform chain: cost 3 on every level but the first (cost 1) -> all but level 0 equal the average or above;
    # use an explicit average above every level so that every level is thin
    p1 = O.plan(chain.rowptr, chain.colidx, lev, mm, O.MANUAL, k=9, avg=100.0)
    p2 = O.plan(chain.rowptr, chain.colidx, lev, mm, O.DEPTH, k=9)
    assert np.array_equal(p1.target, p2.target)
    m = S.gen_torso2_like()
    lev, mm = O.levels(m.rowptr, m.colidx)
    st = O.level_stats(m.rowptr, lev, mm)
    p = O.plan(m.rowptr, m.colidx, lev, mm, O.MANUAL, k=9)
    fat = st["cost"] >= p.avg
    assert np.all(p.target[fat[lev]] == lev[fat[lev]])
    assert p.levels_after < mm


def test_planner_chosen_thin_follows_per_target_depths_on_thin_levels():
    """CHOSEN_THIN (the learned strategy's plan): thin levels only, as in the Section III
    rule, each target taking the next depth_of_target[t] levels.  On a chain whose levels
    are all thin the partition follows from the depths alone; with one depth k everywhere
    it is the MANUAL plan with k, fat levels left alone."""
    n = 60
    chain = S.gen_from_deps(n, np.array([0] + [1] * (n - 1)), np.arange(n - 1), S.rng_for(4))
    lev, mm = O.levels(chain.rowptr, chain.colidx)
    dot = S.rng_for(5).integers(0, 5, mm).astype(np.int32)
    p = O.plan(chain.rowptr, chain.colidx, lev, mm, O.CHOSEN_THIN, avg=100.0, depth_of_target=dot)
    exp = np.empty(mm, np.int64)
    t = -1
    for lv_ in range(mm):
        if t < 0 or lv_ - t > dot[t]:
            t = lv_
        exp[lv_] = t
    assert np.array_equal(p.target, exp[lev])
    m = S.gen_torso2_like(scale=0.25)
    lev, mm = O.levels(m.rowptr, m.colidx)
    for k in (3, 9):
        p1 = O.plan(m.rowptr, m.colidx, lev, mm, O.CHOSEN_THIN, depth_of_target=np.full(mm, k, np.int32))
        p2 = O.plan(m.rowptr, m.colidx, lev, mm, O.MANUAL, k=k)
        assert np.array_equal(p1.target, p2.target) and p1.moved == p2.moved > 0


def test_planner_rowcap_counts_rows_on_thin_levels():
    """ROWCAP: the Section III walk with a row count in place of avgLevelCost.  On a chain of
    one-row thin levels a target of k rows takes the next k-1 levels (the MANUAL plan with
    k-1); on general inputs no target ends with more than k rows, fat levels keep theirs."""
    n = 300
    chain = S.gen_from_deps(n, np.array([0] + [1] * (n - 1)), np.arange(n - 1), S.rng_for(6))
    lev, mm = O.levels(chain.rowptr, chain.colidx)
    for k in (2, 7, 16):
        p1 = O.plan(chain.rowptr, chain.colidx, lev, mm, O.ROWCAP, k=k, avg=100.0)
        p2 = O.plan(chain.rowptr, chain.colidx, lev, mm, O.MANUAL, k=k - 1, avg=100.0)
        assert np.array_equal(p1.target, p2.target)
    for m in (S.gen_torso2_like(scale=0.25), S.gen_config("c0")[0], S.gen_skewed(20000, 3, head=10000)):
        lev, mm = O.levels(m.rowptr, m.colidx)
        st = O.level_stats(m.rowptr, lev, mm)
        for k in (8, 32):
            p = O.plan(m.rowptr, m.colidx, lev, mm, O.ROWCAP, k=k, cap=1.5)
            moved = p.target != lev
            assert moved.any()
            got = np.bincount(p.target, minlength=mm)
            assert got[np.unique(p.target[moved])].max() <= k
            fat = st["cost"] >= p.avg
            assert np.all(p.target[fat[lev]] == lev[fat[lev]])


@pytest.mark.parametrize("alpha,beta", [(3, 0), (0, 40), (4, 100), (1, 0)])
def test_planner_per_row_rules(alpha, beta):
    """Section III.A rules: every rewritten row keeps fewer than alpha dependencies and a
    dependency spread below beta; huge limits are the same as no rules."""
    m, _, _ = S.gen_config("c0", seed=3)
    lev, mm = O.levels(m.rowptr, m.colidx)
    for kind, k in ((O.NAIVE, 0), (O.DEPTH, 3)):
        p = O.plan(m.rowptr, m.colidx, lev, mm, kind, k=k, alpha=alpha, beta=beta)
        sy = O.rewrite(m.rowptr, m.colidx, m.vals, lev, p.target)
        for r in np.nonzero(sy.moved)[0]:
            deps = sy.ccol[sy.cptr[r]:sy.cptr[r + 1]]
            if alpha:
                assert deps.size < alpha
            if beta and deps.size > 1:
                assert deps.max() - deps.min() < beta
        free = O.plan(m.rowptr, m.colidx, lev, mm, kind, k=k)
        loose = O.plan(m.rowptr, m.colidx, lev, mm, kind, k=k, alpha=10**6, beta=10**9)
        assert np.array_equal(free.target, loose.target)
        assert p.moved <= free.moved or kind == O.NAIVE


# ---------------------------------------------------------------------------------
# the cost of a rewritten row (Section III row cost, Section IV: division folded in)
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["equality", "over", "zero"])
def test_planner_naive_rewritten_row_cost_hand_derived(name):
    """NAIVE plans worked out by hand (tests/naive_cost_cases.py) with no injected cost and no
    avg override: the planner's own cost of a rewritten row, 2 |D'|, decides them.  Charging
    2 |D'| + 1 changes the plan of EQUALITY and ZERO, 2 |D'| - 1 that of OVER."""
    from tests.naive_cost_cases import CASES, csr_arrays, expected_row_cost, expected_target
    case = CASES[name]
    n, counts, cols = csr_arrays(case)
    m = S.gen_from_deps(n, np.array(counts), np.array(cols, dtype=np.int64), S.rng_for(3))
    lev, mm = O.levels(m.rowptr, m.colidx)
    st = O.level_stats(m.rowptr, lev, mm)
    assert [int(c) for c in st["cost"]] == case["level_cost"]
    p = O.plan(m.rowptr, m.colidx, lev, mm, O.NAIVE)
    assert p.avg == pytest.approx(case["avg"], abs=1e-9)
    assert p.target.tolist() == expected_target(case)
    assert p.row_cost.tolist() == expected_row_cost(case)
    assert p.levels_after == case["levels_after"]
    for lvl, cost in case["target_level_cost"].items():
        assert int(p.row_cost[p.target == lvl].sum()) == cost
    # the dependency counts the costs were derived from are those of the rewritten equations
    sy = O.rewrite(m.rowptr, m.colidx, m.vals, lev, p.target)
    for r, d in case["deps_after"].items():
        assert int(sy.cptr[r + 1] - sy.cptr[r]) == d
        assert p.row_cost[r] == 2 * d


# ---------------------------------------------------------------------------------
# the walk started at several places (Section III: also from the end of the graph)
# ---------------------------------------------------------------------------------

def _chain(n, seed=0):
    return S.gen_from_deps(n, np.array([0] + [1] * (n - 1)), np.arange(n - 1), S.rng_for(seed))


def test_planner_parts_depth_chain_hand_derived():
    """DEPTH k = 2 on a chain of 10 one-row levels.  One walk: targets every third level.  With
    P ranges every range [w*10/P, (w+1)*10/P) starts its own groups of three."""
    m = _chain(10)
    lev, mm = O.levels(m.rowptr, m.colidx)
    want = {1: [0, 0, 0, 3, 3, 3, 6, 6, 6, 9],
            2: [0, 0, 0, 3, 3, 5, 5, 5, 8, 8],       # ranges [0,5), [5,10)
            3: [0, 0, 0, 3, 3, 3, 6, 6, 6, 9],       # ranges [0,3), [3,6), [6,10): the same as one walk
            4: [0, 0, 2, 2, 2, 5, 5, 7, 7, 7]}       # ranges [0,2), [2,5), [5,7), [7,10)
    for parts, tgt in want.items():
        p = O.plan(m.rowptr, m.colidx, lev, mm, O.DEPTH, k=2, parts=parts)
        assert p.target.tolist() == tgt, parts
    # more ranges than levels: every level starts a range, nothing moves
    p = O.plan(m.rowptr, m.colidx, lev, mm, O.DEPTH, k=2, parts=25)
    assert p.target.tolist() == list(range(10)) and p.moved == 0


def test_planner_parts_cap_share_hand_derived():
    """DEPTH k = 8 on a chain of 9 one-row levels with the nnz cap 2.0: nnz(L) = 17, allowance 17.
    Moving row i into level 0 adds i entries (its E row grows by one substitution per row above).
    One walk takes rows 1..5 (15), rejects row 6 (21 > 17): level 6 is a target; row 7 joins it
    (+2, 17), row 8 does not (+3): level 8 is a target.  Two ranges, levels [0,4) with 7 entries and
    [4,9) with 10: shares 17*7/17 = 7 and 17*10/17 = 10; range 0 moves rows 1..3 (1+2+3 = 6); range 1
    starts a target at 4 and moves rows 5, 6, 7 (+2, +3, +4 = 9) but not 8 (+5 > 10)."""
    m = _chain(9)
    lev, mm = O.levels(m.rowptr, m.colidx)
    p1 = O.plan(m.rowptr, m.colidx, lev, mm, O.DEPTH, k=8, cap=2.0)
    assert p1.target.tolist() == [0, 0, 0, 0, 0, 0, 6, 6, 8]
    assert p1.stored_nnz == 17 + 15 + 2
    p2 = O.plan(m.rowptr, m.colidx, lev, mm, O.DEPTH, k=8, cap=2.0, parts=2)
    assert p2.target.tolist() == [0, 0, 0, 0, 4, 4, 4, 4, 8]
    assert p2.stored_nnz == 17 + 6 + 9


@pytest.mark.parametrize("kind,k", [(O.NAIVE, 0), (O.ROWCAP, 32), (O.MANUAL, 9), (O.DEPTH, 3)])
@pytest.mark.parametrize("parts", [2, 5])
def test_planner_parts_invariants(kind, k, parts):
    """Rows never move across a range start; the first eligible level of every range keeps its rows;
    the rewrite of the plan is still the elimination E L, and with the cap each range stays within
    its share."""
    m = S.gen_mixture(6000, 10_555)
    lev, mm = O.levels(m.rowptr, m.colidx)
    for cap in (0.0, 1.3):
        p = O.plan(m.rowptr, m.colidx, lev, mm, kind, k=k, cap=cap, parts=parts)
        starts = [mm * w // parts for w in range(parts)]
        rng_of = np.searchsorted(starts, lev, side="right") - 1
        assert np.all(p.target >= np.array(starts)[rng_of])
        for s0 in starts:
            assert np.all(p.target[lev == s0] == s0)
        if cap:
            assert p.stored_nnz <= math.floor(cap * p.nnz_l)
        sy = O.rewrite(m.rowptr, m.colidx, m.vals, lev, p.target)
        stored = int(sy.cptr[-1]) + m.n + int(sy.eptr[-1])
        assert stored == p.stored_nnz
        b = S.rhs_uniform(m.n, 1, 2)[0]
        assert np.allclose(sy.solve(b), O.forward_subst(m.rowptr, m.colidx, m.vals, b), rtol=1e-9, atol=1e-12)
