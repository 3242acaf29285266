"""GPU parity of schedules with CLUSTER segments: mid-width levels run on the CTAs of one
thread-block cluster with a cluster barrier per level, inside regions that also hold
single-CTA runs, between WIDE levels that use the device-wide completion flags.  Every
solution is compared with the CPU oracle's forward substitution."""
import numpy as np
import pytest

import oracle as O
from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S
from tests.gpu_util import TOL_F32, TOL_F64, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def solve_cluster(m, b, cluster, cluster_rows=0, run_width=0, lpr=0, system_kw=None, stamps=False, shared_x=0):
    torch = torch_cuda()
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    s = B.System(M, lv, **(system_kw or {}))
    if run_width or lpr:
        s.tune(run_width=run_width, lanes_per_row=lpr)
    s.tune_cluster(cluster, cluster_rows, shared_x=shared_x)
    vt = torch.float64 if M.dtype == B.F64 else torch.float32
    bt = torch.from_numpy(np.ascontiguousarray(b)).to("cuda", dtype=vt)
    st = torch.zeros(max(s.m, 1), dtype=torch.int64, device="cuda") if stamps else None
    x = s.solve(bt, stamps=st, check_status=True).cpu().numpy()
    ref = O.forward_subst(m.rowptr, m.colidx, m.vals, b)
    return s, x, ref, st


def layered_profile(widths, deps, seed):
    """Levels of the given widths; every row of a level reads `deps` distinct rows of the level
    before it (so the level structure is exactly the profile)."""
    rng = S.rng_for(seed)
    counts, cols = [], []
    start_prev, start = 0, 0
    for li, w in enumerate(widths):
        for _ in range(w):
            if li == 0:
                counts.append(0)
            else:
                c = np.sort(rng.choice(widths[li - 1], size=min(deps, widths[li - 1]), replace=False)) + start_prev
                counts.append(len(c))
                cols.extend(c.tolist())
        start_prev, start = start, start + w
    n = sum(widths)
    return S.gen_from_deps(n, np.array(counts), np.array(cols, dtype=np.int64), rng)


@pytest.mark.parametrize("cluster", [2, 8, 16])
@pytest.mark.parametrize("nrhs", [1, 4])
def test_cluster_grid_runs_and_cluster_levels(cluster, nrhs):
    """A 300 x 300 grid (levels of 1..300 rows): levels up to 64 rows in single-CTA runs, the
    wider ones on the cluster, all in one region."""
    m = S.gen_laplacian(300)
    b = S.rhs_uniform(m.n, nrhs, 3)
    s, x, ref, st = solve_cluster(m, b, cluster, run_width=64, stamps=(nrhs == 1))
    info = s.refresh()
    assert info["cluster"] == cluster and info["cluster_levels"] > 0
    assert rel_l2(x, ref) <= TOL_F64
    if st is not None:
        t = st.cpu().numpy()[:s.m]
        assert (t > 0).all() and (np.diff(t) >= 0).all()  # every level stamped, in order


@pytest.mark.parametrize("cluster_rows", [2000, 16384])
@pytest.mark.parametrize("rewrite", [False, True])
def test_cluster_mixture_with_wide_levels(cluster_rows, rewrite):
    """A mixture of skewed-head, chain and grid blocks: WIDE levels, CLUSTER levels and thin runs
    interleave, so regions are entered and left through the completion flags many times."""
    m = S.gen_mixture(120_000, 10_077)
    _, b = S.rhs_from_xtrue(m, 1, 4)
    kw = dict(kind=B.NAIVE, cap=1.5) if rewrite else {}
    s, x, ref, _ = solve_cluster(m, b, 16, cluster_rows=cluster_rows, system_kw=kw)
    assert s.refresh()["cluster_levels"] > 0
    assert rel_l2(x, ref) <= TOL_F64


def test_cluster_profile_wide_cluster_wide():
    """WIDE (20,000 rows), three CLUSTER levels (5,000 rows), WIDE again, thin levels, CLUSTER."""
    m = layered_profile([20000, 5000, 5000, 5000, 20000, 8, 8, 8, 8, 8, 3000, 3000], 4, 11)
    b = S.rhs_uniform(m.n, 2, 5)
    for cl in (4, 16):
        s, x, ref, _ = solve_cluster(m, b, cl, cluster_rows=10000)
        assert s.refresh()["cluster"] == cl
        assert rel_l2(x, ref) <= TOL_F64


def test_cluster_float32_and_two_lanes_per_row():
    m = S.gen_laplacian(200).astype(np.float32)
    b = S.rhs_uniform(m.n, 1, 6).astype(np.float32)
    for lpr in (1, 2):
        s, x, ref, _ = solve_cluster(m, b, 8, run_width=32, lpr=lpr)
        assert s.refresh()["cluster_levels"] > 0
        assert rel_l2(x, ref) <= TOL_F32


def test_cluster_off_matches_cluster_on():
    torch = torch_cuda()
    m = S.gen_laplacian(256)
    b = S.rhs_uniform(m.n, 1, 8)
    _, x_on, ref, _ = solve_cluster(m, b, 16, run_width=64)
    s_off, x_off, _, _ = solve_cluster(m, b, 1, run_width=64)
    assert s_off.refresh()["cluster"] == 1 and s_off.refresh()["cluster_levels"] == 0
    assert rel_l2(x_on, ref) <= TOL_F64 and rel_l2(x_off, ref) <= TOL_F64


@pytest.mark.parametrize("withhold", [0, 1])
def test_cluster_bounded_wait_times_out_without_faulting(withhold):
    """A withheld completion flag in front of a cluster region (segment 0) or after it (segment 1):
    the waiting CTAs give up after the short limit, every CTA of the cluster keeps taking the
    cluster barriers, the status reads TIMEOUT and the next solve is correct."""
    torch = torch_cuda()
    m = layered_profile([20000, 5000, 5000, 5000, 20000], 3, 13)
    _, b = S.rhs_from_xtrue(m, 1, 2)
    M = B.Matrix.from_host(m)
    s = B.System(M, B.Levels(M))
    s.tune_cluster(16, 10000)
    bt = torch.from_numpy(b).cuda()
    s.solve(bt, check_status=True)
    info = s.refresh()
    assert info["segments"] == 3 and info["cluster_levels"] == 3  # WIDE, CLUSTER (3 levels), WIDE
    assert info["shared_x_levels"] == 3  # x of the cluster levels through shared memory
    s.debug_set_wait(withhold_segment=withhold, timeout_ns=50_000_000)
    s.solve(bt)
    with pytest.raises(B.SptrsvError) as e:
        s.status()
    assert e.value.code == B.ERR_TIMEOUT
    s.debug_set_wait(-1, 0)
    x = s.solve(bt, check_status=True).cpu().numpy()
    assert rel_l2(x, O.forward_subst(m.rowptr, m.colidx, m.vals, b)) < TOL_F64


@pytest.mark.parametrize("cluster", [2, 8, 16])
def test_shared_x_grid_ragged_shares(cluster):
    """One right-hand side: CLUSTER levels read the previous level's x from the shared memory of the
    CTA that computed it.  Grid levels of 65..300 rows split over 2, 8 or 16 CTAs leave ragged last
    shares (and CTAs with no rows); the solution matches the oracle and the same schedule without
    the shared-memory exchange."""
    m = S.gen_laplacian(300)
    b = S.rhs_uniform(m.n, 1, 3)
    s, x, ref, st = solve_cluster(m, b, cluster, run_width=64, stamps=True)
    info = s.refresh()
    assert info["shared_x_levels"] == info["cluster_levels"] > 0
    assert rel_l2(x, ref) <= TOL_F64
    t = st.cpu().numpy()[:s.m]
    assert (t > 0).all() and (np.diff(t) >= 0).all()
    s1, x1, _, _ = solve_cluster(m, b, cluster, run_width=64, shared_x=1)
    assert s1.refresh()["shared_x_levels"] == 0 and s1.refresh()["cluster_levels"] == info["cluster_levels"]
    assert rel_l2(x1, ref) <= TOL_F64


@pytest.mark.parametrize("rewrite", [None, "naive", "depth4"])
def test_shared_x_mixture_and_rewritten_rows(rewrite):
    """Mixtures with WIDE, CLUSTER and thin levels; rewritten systems put rows with E entries (b-parts
    computed up front) and long substituted rows into the CLUSTER levels."""
    m = S.gen_mixture(150_000, 10_091)
    _, b = S.rhs_from_xtrue(m, 1, 4)
    kw = {None: {}, "naive": dict(kind=B.NAIVE, cap=1.5), "depth4": dict(kind=B.DEPTH_K, k=4)}[rewrite]
    s, x, ref, _ = solve_cluster(m, b, 16, system_kw=kw)
    assert s.refresh()["shared_x_levels"] > 0
    assert rel_l2(x, ref) <= TOL_F64


def test_shared_x_float32_profile():
    """float32 values; CLUSTER segments after WIDE levels and after thin runs, with levels of 1,000
    to 9,000 rows (shares of up to 563 rows: two rows for some threads)."""
    m = layered_profile([20000, 9000, 1000, 7001, 8, 8, 8, 8, 8, 3001, 9000, 20000, 5000], 5, 17)
    m32 = m.astype(np.float32)
    b = S.rhs_uniform(m.n, 1, 5).astype(np.float32)
    s, x, ref, _ = solve_cluster(m32, b, 16, cluster_rows=10000)
    assert s.refresh()["shared_x_levels"] >= 5
    assert rel_l2(x, ref) <= TOL_F32


def test_shared_x_full_size_grid():
    """The 2048 x 2048 grid (4,194,304 rows, 4,095 levels of up to 2,048 rows) at full size, plain and
    rewritten to depth 4."""
    m, b, _ = S.gen_config("c2")
    for kw in ({}, dict(kind=B.DEPTH_K, k=4)):
        s, x, ref, _ = solve_cluster(m, b, 16, system_kw=kw)
        assert s.refresh()["shared_x_levels"] > 0
        assert rel_l2(x, ref) <= TOL_F64


def test_profile_launch_switch_keeps_cluster_shape():
    """SPTRSV_PROFILE_LAUNCH=1 (read once per process, so in a child process): launches with clusters
    go out without the cooperative attribute; the shared-x cluster solve still runs on its clusters
    (the kernel checks its cluster shape on entry) and matches the oracle."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import numpy as np, torch\n"
        "import oracle as O\n"
        "from paper_2206_05843_gb300 import binding as B, synth as S\n"
        "m = S.gen_laplacian(300); b = S.rhs_uniform(m.n, 1, 3)\n"
        "M = B.Matrix.from_host(m); s = B.System(M, B.Levels(M)); s.tune(run_width=64); s.tune_cluster(16, 0)\n"
        "x = s.solve(torch.from_numpy(b).cuda(), check_status=True).cpu().numpy()\n"
        "ref = O.forward_subst(m.rowptr, m.colidx, m.vals, b)\n"
        "info = s.refresh()\n"
        "print(info['cluster'], info['shared_x_levels'], float(np.linalg.norm(x - ref) / np.linalg.norm(ref)))\n")
    env = dict(os.environ, SPTRSV_PROFILE_LAUNCH="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    cl, shared, err = r.stdout.split()[-3:]
    assert int(cl) == 16 and int(shared) > 0 and float(err) <= TOL_F64
