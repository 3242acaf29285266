"""GPU parity of wide levels whose coefficients stream through shared-memory tiles (bulk copies on
an mbarrier, two buffers): solutions against the CPU oracle for several tile sizes, float32
values, rewritten rows (E entries) inside wide levels, and a timed-out wait with tile copies in
flight."""
import numpy as np
import pytest

import oracle as O
from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S
from tests.gpu_util import TOL_F32, TOL_F64, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def solve(m, b, tiles, system_kw=None, lpr=0):
    torch = torch_cuda()
    M = B.Matrix.from_host(m)
    s = B.System(M, B.Levels(M), **(system_kw or {}))
    s.tune_cluster(1, 0, tiles)
    if lpr:
        s.tune(lanes_per_row=lpr)
    vt = torch.float64 if M.dtype == B.F64 else torch.float32
    bt = torch.from_numpy(np.ascontiguousarray(b)).to("cuda", dtype=vt)
    x = s.solve(bt, check_status=True).cpu().numpy()
    return s, x, O.forward_subst(m.rowptr, m.colidx, m.vals, b)


@pytest.mark.parametrize("deps", [3, 8, 20, 60])
def test_tiled_layered_levels(deps):
    """8 layers of 100,000 rows, `deps` dependencies per row: with 60 per row the tile shrinks to
    128 rows (or the level is not tiled); the solution is the oracle's either way."""
    m = S.gen_layered(8, 100_000, 5, k=deps)
    _, b = S.rhs_from_xtrue(m, 1, 1)
    s, x, ref = solve(m, b, 0, lpr=1)  # tiles run one lane per row
    if deps <= 20:  # 512-row tiles up to 8 per row, 128-row tiles at 20 per row
        assert s.refresh()["tiled_levels"] >= 7
    assert rel_l2(x, ref) <= TOL_F64
    s_off, x_off, _ = solve(m, b, 1, lpr=1)
    assert s_off.refresh()["tiled_levels"] == 0
    assert rel_l2(x_off, ref) <= TOL_F64


def test_tiled_float32_and_rewritten_rows():
    m = S.gen_layered(8, 60_000, 9)
    _, b = S.rhs_from_xtrue(m, 1, 2)
    # float32 values
    m32 = m.astype(np.float32)
    s, x, ref = solve(m32, b.astype(np.float32), 0, lpr=1)
    assert s.refresh()["tiled_levels"] > 0
    assert rel_l2(x, ref) <= TOL_F32
    # depth-1 rewrite: every other layer moves into the one before it, so wide levels hold
    # rewritten rows with E entries (3 dependencies per row keep the rewritten rows short)
    m = S.gen_layered(8, 60_000, 9, k=3)
    _, b = S.rhs_from_xtrue(m, 1, 2)
    s2, x2, ref2 = solve(m, b, 0, system_kw=dict(kind=B.DEPTH_K, k=1), lpr=1)
    info = s2.refresh()
    assert info["rows_moved"] > 0 and info["tiled_levels"] > 0
    assert rel_l2(x2, ref2) <= TOL_F64


def test_tiled_full_size_wide_level_matrix():
    m, b, xt = S.gen_config("w2")
    s, x, ref = solve(m, b, 0, lpr=1)
    assert s.refresh()["tiled_levels"] >= 7
    assert rel_l2(x, ref) <= TOL_F64 and rel_l2(x, xt) < 1e-12


def test_tiled_bounded_wait_times_out_without_faulting():
    """A withheld completion flag: the CTAs of the next level give up after the short limit with
    their first tile copies in flight, wait for those copies, and the status reads TIMEOUT; the
    next solve is correct."""
    torch = torch_cuda()
    m = S.gen_layered(4, 200_000, 3)
    _, b = S.rhs_from_xtrue(m, 1, 2)
    M = B.Matrix.from_host(m)
    s = B.System(M, B.Levels(M))
    s.tune_cluster(1, 0, 0)
    bt = torch.from_numpy(b).cuda()
    s.solve(bt, check_status=True)
    assert s.refresh()["tiled_levels"] >= 3
    s.debug_set_wait(withhold_segment=1, timeout_ns=50_000_000)
    s.solve(bt)
    with pytest.raises(B.SptrsvError) as e:
        s.status()
    assert e.value.code == B.ERR_TIMEOUT
    s.debug_set_wait(-1, 0)
    x = s.solve(bt, check_status=True).cpu().numpy()
    assert rel_l2(x, O.forward_subst(m.rowptr, m.colidx, m.vals, b)) < TOL_F64
