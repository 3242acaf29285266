"""GPU parity of analysis and the plain level-set solve against the CPU oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S
from tests.gpu_util import TOL_F32, TOL_F64, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def check_levels(m):
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    ex = lv.export()
    lev, mm = O.levels(m.rowptr, m.colidx)
    assert lv.m == mm
    assert np.array_equal(ex["level"], lev)
    st = O.level_stats(m.rowptr, lev, mm)
    assert np.array_equal(ex["rows"], st["rows"])
    assert np.array_equal(ex["nnz"], st["nnz"])
    assert np.array_equal(ex["cost"], st["cost"])
    # rows of each level, ascending row index inside the level
    order = np.lexsort((np.arange(m.n), lev))
    assert np.array_equal(ex["level_rows"], order)
    assert np.array_equal(ex["level_ptr"], np.concatenate([[0], np.cumsum(st["rows"])]))
    return M, lv


@pytest.mark.parametrize("seed", range(4))
def test_levels_small_random(seed):
    torch_cuda()
    m = S.gen_banded_random(3000 + 37 * seed, seed, k=4, band=50 + 30 * seed)
    check_levels(m)


@pytest.mark.parametrize("name", ["c0", "c2"])
def test_levels_configs(name):
    torch_cuda()
    m, _, _ = S.gen_config(name, scale=1.0 if name == "c0" else 0.05)
    check_levels(m)


def test_levels_skewed_full_size():
    torch_cuda()
    m, _, _ = S.gen_config("c1")
    check_levels(m)


def test_levels_edge_cases():
    torch_cuda()
    # single row, diagonal only, a pure chain (one row per level), all independent
    for n, counts, cols in [
        (1, [0], []),
        (100, [0] * 100, []),
        (1000, [0] + [1] * 999, list(range(999))),
    ]:
        m = S.gen_from_deps(n, np.array(counts), np.array(cols, dtype=np.int64), S.rng_for(1))
        check_levels(m)


def solve_and_compare(m, b, tol, system_kw=None, tune=None):
    torch = torch_cuda()
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    sysm = B.System(M, lv, **(system_kw or {}))
    if tune:
        sysm.tune(**tune)
    vt = torch.float64 if M.dtype == B.F64 else torch.float32
    bt = torch.from_numpy(np.ascontiguousarray(b)).to("cuda", dtype=vt)
    x = sysm.solve(bt, check_status=True).cpu().numpy()
    ref = O.forward_subst(m.rowptr, m.colidx, m.vals, b)
    err = rel_l2(x, ref)
    assert err <= tol, err
    return sysm, x, ref


@pytest.mark.parametrize("seed", range(6))
def test_plain_solve_config0_seeds(seed):
    m, b, xt = S.gen_config("c0", seed=seed)
    _, x, _ = solve_and_compare(m, b, TOL_F64)
    assert rel_l2(x, xt) < 1e-12


@pytest.mark.parametrize("nrhs", [1, 2, 3, 5, 16, 32])
def test_plain_solve_multi_rhs(nrhs):
    m = S.gen_banded_random(5000, 3, k=6, band=300)
    b = S.rhs_uniform(m.n, nrhs, 4)
    solve_and_compare(m, b, TOL_F64)


@pytest.mark.parametrize("run_width", [-1, 8, 0, 100000])
@pytest.mark.parametrize("lpr", [1, 4, 32])
def test_plain_solve_schedule_variants(run_width, lpr):
    """Every schedule shape (no runs, short runs, default, everything in one CTA) and
    lanes-per-row split gives the same solution."""
    m = S.gen_skewed(20000, 5, head=15000)
    _, b = S.rhs_from_xtrue(m, 1, 2)
    solve_and_compare(m, b, TOL_F64, tune=dict(run_width=run_width, lanes_per_row=lpr))


@pytest.mark.parametrize("nrhs", [2, 5, 16, 17, 29, 32])
@pytest.mark.parametrize("lpr", [1, 2])
@pytest.mark.parametrize("f32", [False, True])
def test_fast_thin_levels_several_rhs(nrhs, lpr, f32):
    """Thin levels with several right-hand sides in the fast executor (one lane per row,
    right-hand side and coefficient lane; two right-hand sides per lane above 16, the last
    lane of an odd count holding one), plain and rewritten, against the oracle; the
    dependencies older than the ring window are folded for every right-hand side."""
    m = S.gen_skewed(30000, 8, head=12000)
    if f32:
        m = m.astype(np.float32)
    b = S.rhs_uniform(m.n, nrhs, 9)
    if f32:
        b = b.astype(np.float32)
    tol = TOL_F32 if f32 else TOL_F64
    for kw in ({}, dict(kind=B.NAIVE, cap=1.5), dict(kind=B.DEPTH_K, k=3)):
        solve_and_compare(m, b, tol, system_kw=kw, tune=dict(lanes_per_row=lpr))


def test_plain_solve_float32_values():
    m = S.gen_banded_random(4000, 9).astype(np.float32)
    b = S.rhs_uniform(m.n, 3, 1).astype(np.float32)
    solve_and_compare(m, b, TOL_F32)


@pytest.mark.parametrize("name", ["c1", "c2", "c2r16", "w1"])
def test_plain_solve_full_size(name):
    m, b, _ = S.gen_config(name)
    solve_and_compare(m, b, TOL_F64)


def test_plain_solve_repeat_is_deterministic():
    torch = torch_cuda()
    m, b, _ = S.gen_config("c1", scale=0.05)
    M = B.Matrix.from_host(m)
    sysm = B.System(M, B.Levels(M))
    bt = torch.from_numpy(b).cuda()
    x1 = sysm.solve(bt, check_status=True).cpu().numpy()
    for _ in range(3):
        x2 = sysm.solve(bt, check_status=True).cpu().numpy()
        assert np.array_equal(x1, x2)


def test_invalid_csr_is_rejected():
    torch_cuda()
    m = S.gen_banded_random(100, 0)
    bad = S.LowerCsr(m.n, m.rowptr, m.colidx.copy(), m.vals.copy())
    bad.vals[m.rowptr[10] - 1] = 0.0  # zero diagonal of row 9
    M = B.Matrix.from_host(bad)
    with pytest.raises(B.SptrsvError) as e:
        B.Levels(M)
    assert e.value.code == B.ERR_INVALID and "row 9" in str(e.value)
    bad2 = S.LowerCsr(m.n, m.rowptr, m.colidx.copy(), m.vals.copy())
    bad2.colidx[m.rowptr[20] - 1] = 5  # diagonal of row 19 missing
    with pytest.raises(B.SptrsvError):
        B.Matrix.from_host(bad2).validate()


def test_bounded_wait_times_out_without_faulting():
    """A withheld completion flag makes the waiting CTAs give up after the short limit;
    the status comes back as TIMEOUT and the context stays usable."""
    torch = torch_cuda()
    m = S.gen_layered(4, 20000, 3)
    _, b = S.rhs_from_xtrue(m, 1, 2)
    M = B.Matrix.from_host(m)
    sysm = B.System(M, B.Levels(M))
    bt = torch.from_numpy(b).cuda()
    sysm.solve(bt, check_status=True)
    assert sysm.refresh()["segments"] >= 2
    sysm.debug_set_wait(withhold_segment=1, timeout_ns=50_000_000)
    sysm.solve(bt)
    with pytest.raises(B.SptrsvError) as e:
        sysm.status()
    assert e.value.code == B.ERR_TIMEOUT
    sysm.debug_set_wait(-1, 0)
    x = sysm.solve(bt, check_status=True).cpu().numpy()
    assert rel_l2(x, O.forward_subst(m.rowptr, m.colidx, m.vals, b)) < TOL_F64


def test_autotune_keeps_the_solution():
    torch = torch_cuda()
    m = S.gen_skewed(40000, 12, head=30000)
    _, b = S.rhs_from_xtrue(m, 1, 3)
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    ref = O.forward_subst(m.rowptr, m.colidx, m.vals, b)
    for kw in ({}, dict(kind=B.NAIVE, cap=1.5)):
        s = B.System(M, lv, **kw)
        us = s.autotune(1)
        assert us > 0
        x = s.solve(torch.from_numpy(b).cuda(), check_status=True).cpu().numpy()
        assert rel_l2(x, ref) <= TOL_F64
        assert s.autotune(1) == us  # cached by signature


@pytest.mark.parametrize("nrhs", [1, 3])
def test_per_level_launch_mode(nrhs):
    """One launch per level (run width -2) gives the same solution."""
    m = S.gen_layered(6, 30000, 9)
    b = S.rhs_uniform(m.n, nrhs, 2)
    solve_and_compare(m, b, TOL_F64, tune=dict(run_width=-2))
    m2, b2, _ = S.gen_config("c0")
    solve_and_compare(m2, b2, TOL_F64, system_kw=dict(kind=B.NAIVE, cap=1.5), tune=dict(run_width=-2))


@pytest.mark.parametrize("k", [3, 5, 8, 11, 17])
def test_wide_only_schedules(k):
    """Schedules of wide levels only (no single-CTA runs) run the kernel variant without shared
    memory, whose rows load their coefficients eight at a time: rows of 3..17 coefficients
    (aligned and unaligned, shorter and longer than eight), plain and after a depth-1 rewrite
    (rewritten rows with E entries in wide levels)."""
    m = S.gen_layered(6, 30_000, 21, k=k)
    _, b = S.rhs_from_xtrue(m, 1, 3)
    for kw in ({}, dict(kind=B.DEPTH_K, k=1)):
        s, x, ref = solve_and_compare(m, b, TOL_F64, system_kw=kw, tune=dict(lanes_per_row=1))
        info = s.refresh()
        assert info["run_levels"] == 0 and info["cluster_levels"] == 0
