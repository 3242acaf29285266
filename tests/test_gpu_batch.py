"""GPU parity of the batched solve: every matrix of the batch is checked against the CPU
oracle individually, and the captured graph is replayed with new right-hand sides."""
import numpy as np
import pytest

import oracle as O
from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S
from tests.gpu_util import TOL_F32, TOL_F64, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def make_batch(items, rewrite_every=0):
    torch = torch_cuda()
    mats, systems, keep = [], [], []
    for idx, it in enumerate(items):
        m = it.matrix.astype(np.float32) if it.fp32 else it.matrix
        M = B.Matrix.from_host(m)
        lv = B.Levels(M)
        if rewrite_every and idx % rewrite_every == 0:
            s = B.System(M, lv, B.DEPTH_K, k=2)
        else:
            s = B.System(M, lv)
        mats.append(m)
        systems.append(s)
        keep.append((M, lv))
    bt = B.Batch(systems, [it.nrhs for it in items])
    return bt, mats, systems, keep


def check(items, mats, xs, bs_host):
    for it, m, x, b in zip(items, mats, xs, bs_host):
        ref = O.forward_subst(m.rowptr, m.colidx, m.vals, b)
        err = rel_l2(x.cpu().numpy(), ref)
        assert err <= (TOL_F32 if it.fp32 else TOL_F64), (m.name, it.nrhs, it.fp32, err)


@pytest.mark.parametrize("rewrite_every", [0, 3])
def test_batch_small_mixed(rewrite_every):
    torch = torch_cuda()
    items = S.gen_batch(count=24, base_seed=77, n_lo=500, n_hi=6000, rhs_hi=32)
    bt, mats, systems, keep = make_batch(items, rewrite_every)
    assert bt.info["graph"] == 1
    for rep in range(3):  # graph replays with new right-hand sides
        bs_host = [S.rhs_uniform(it.matrix.n, it.nrhs, 1000 * rep + i) for i, it in enumerate(items)]
        bs = [torch.from_numpy(b).to("cuda", dtype=torch.float32 if it.fp32 else torch.float64)
              for b, it in zip(bs_host, items)]
        xs = bt.solve(bs)
        torch.cuda.synchronize()
        bs_used = [b.astype(np.float32).astype(np.float64) if it.fp32 else b for b, it in zip(bs_host, items)]
        check(items, mats, xs, bs_used)


def test_batch_full_config3():
    torch = torch_cuda()
    items = S.gen_batch()
    bt, mats, systems, keep = make_batch(items)
    bs = [torch.from_numpy(it.b).to("cuda", dtype=torch.float32 if it.fp32 else torch.float64) for it in items]
    xs = bt.solve(bs)
    torch.cuda.synchronize()
    bs_used = [it.b.astype(np.float32).astype(np.float64) if it.fp32 else it.b for it in items]
    check(items, mats, xs, bs_used)
    # float64 matrices generated from x_true recover it
    for it, x in zip(items, xs):
        if not it.fp32 and it.x_true is not None:
            assert rel_l2(x.cpu().numpy(), it.x_true) < 1e-12


def test_batch_single_matrix_wide_levels():
    """A level far wider than the staging area is split over blocks."""
    torch = torch_cuda()
    m = S.gen_layered(3, 5000, 4)
    _, b = S.rhs_from_xtrue(m, 3, 2)
    M = B.Matrix.from_host(m)
    s = B.System(M, B.Levels(M))
    bt = B.Batch([s], [3])
    xs = bt.solve([torch.from_numpy(b).cuda()])
    torch.cuda.synchronize()
    assert rel_l2(xs[0].cpu().numpy(), O.forward_subst(m.rowptr, m.colidx, m.vals, b)) < TOL_F64


def test_batch_splits_heavy_right_hand_sides():
    """A banded matrix of 60,000 rows with 32 right-hand sides among small ones: its float64 work
    outweighs its critical path, so its right-hand sides split into parts that run on several
    CTAs (more work items than systems); every system and right-hand side matches the oracle, on
    two graph replays."""
    torch = torch_cuda()
    items = S.gen_batch(count=10, base_seed=91, n_lo=1000, n_hi=6000, rhs_hi=3)
    heavy = S.gen_banded_random(60_000, 5)
    xt, b = S.rhs_from_xtrue(heavy, 32, 6)
    items.insert(3, S.BatchItem(heavy, b, xt, 32, False, 0))
    bt, mats, systems, keep = make_batch(items)
    assert bt.info["items"] > bt.info["count"] == len(items)
    for rep in range(2):
        bs_host = [S.rhs_uniform(it.matrix.n, it.nrhs, 500 * rep + i) for i, it in enumerate(items)]
        bs = [torch.from_numpy(b).to("cuda", dtype=torch.float32 if it.fp32 else torch.float64)
              for b, it in zip(bs_host, items)]
        xs = bt.solve(bs)
        torch.cuda.synchronize()
        bs_used = [b.astype(np.float32).astype(np.float64) if it.fp32 else b for b, it in zip(bs_host, items)]
        check(items, mats, xs, bs_used)
