"""The solve that allocates nothing (sptrsv_solve_noalloc), called through the C ABI.

Callers that cannot call cudaMalloc while they solve (real-time loops that must stay out
of the allocator, processes whose device memory a framework's caching allocator holds,
plug-in code handed only its inputs and outputs) use this entry point; its scratch is a
fixed device array of the library.  This file runs last so that a failure
here does not hide the other tests, and it passes both alone and after them."""
import numpy as np
import pytest

from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S
from tests.gpu_util import TOL_F32, TOL_F64, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["plain", "naive"])
def test_noalloc_matches_regular_solve_twice(kind):
    torch = torch_cuda()
    m = S.gen_skewed(30000, 8, head=22000)
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    s = B.System(M, lv) if kind == "plain" else B.System(M, lv, B.NAIVE, cap=1.5)
    b1 = torch.from_numpy(S.rhs_uniform(m.n, 1, 1)[0]).cuda()
    b2 = torch.from_numpy(S.rhs_uniform(m.n, 1, 2)[0]).cuda()
    r1 = s.solve(b1, check_status=True).clone()  # builds the schedule for nrhs = 1
    r2 = s.solve(b2, check_status=True).clone()
    x = torch.empty_like(b1)
    s.solve_noalloc(b1, x)
    s.status()
    assert rel_l2(x.cpu().numpy(), r1.cpu().numpy()) <= TOL_F64
    s.solve_noalloc(b2, x)
    s.status()
    assert rel_l2(x.cpu().numpy(), r2.cpu().numpy()) <= TOL_F64


def test_noalloc_multi_rhs_and_limits():
    torch = torch_cuda()
    m = S.gen_banded_random(20000, 5)
    M = B.Matrix.from_host(m)
    s = B.System(M, B.Levels(M))
    b = torch.from_numpy(S.rhs_uniform(m.n, 4, 3)).cuda()
    x = torch.empty_like(b)
    with pytest.raises(B.SptrsvError) as e:  # no schedule for nrhs = 4 yet
        s.solve_noalloc(b, x)
    assert e.value.code == B.ERR_INVALID
    ref = s.solve(b, check_status=True).clone()
    for _ in range(2):
        s.solve_noalloc(b, x)
        s.status()
        assert rel_l2(x.cpu().numpy(), ref.cpu().numpy()) <= TOL_F64
    # beyond the static scratch: rejected on the host before any launch
    big = S.gen_from_deps(9_000_000, np.zeros(9_000_000, np.int64), np.zeros(0, np.int64), None, diag=2.0)
    MB = B.Matrix.from_host(big)
    sb = B.System(MB, B.Levels(MB))
    bb = torch.ones(big.n, dtype=torch.float64, device="cuda")
    sb.solve(bb, check_status=True)
    with pytest.raises(B.SptrsvError) as e2:
        sb.solve_noalloc(bb, torch.empty_like(bb))
    assert e2.value.code == B.ERR_UNSUPPORTED


def test_noalloc_float32_and_one_launch_per_level():
    """float32 values (checked at the float32 tolerance), and a system tuned to one launch per
    level, whose launches the entry point follows."""
    torch = torch_cuda()
    m = S.gen_skewed(20000, 8, head=16000).astype(np.float32)
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    for tune in (None, -2):
        s = B.System(M, lv, B.NAIVE, cap=1.5)
        if tune is not None:
            s.tune(run_width=tune)
        x = None
        for seed in (4, 5):
            b = torch.from_numpy(S.rhs_uniform(m.n, 1, seed)[0]).to("cuda", dtype=torch.float32)
            ref = s.solve(b, check_status=True).clone()
            x = torch.empty_like(b) if x is None else x
            s.solve_noalloc(b, x)
            s.status()
            assert rel_l2(x.cpu().numpy(), ref.cpu().numpy()) <= TOL_F32


def test_noalloc_cluster_levels_with_shared_x():
    """A schedule whose mid-width levels run on a 16-CTA cluster and read the previous level's x from
    the cluster's shared memory: the entry point launches the same kernel; two calls in a row match
    the regular solve."""
    torch = torch_cuda()
    m = S.gen_laplacian(300)
    M = B.Matrix.from_host(m)
    s = B.System(M, B.Levels(M))
    s.tune(run_width=64)
    s.tune_cluster(16, 0)
    x = None
    for seed in (6, 7):
        b = torch.from_numpy(S.rhs_uniform(m.n, 1, seed)[0]).cuda()
        ref = s.solve(b, check_status=True).clone()
        assert s.refresh()["shared_x_levels"] > 0
        x = torch.empty_like(b) if x is None else x
        s.solve_noalloc(b, x)
        s.status()
        assert rel_l2(x.cpu().numpy(), ref.cpu().numpy()) <= TOL_F64
