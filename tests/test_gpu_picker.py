"""GPU parity of the learned picker: features against the feature oracle, inference and
gradients against the float64 MLP oracle, one Adam step, save/load, and the learned
rewrite path against the CPU oracle."""
import numpy as np
import pytest

import oracle as O
from oracle import features as OF
from oracle import mlp as OM
from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S
from tests.gpu_util import TOL_F64, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
DEPTHS = [1, 2, 4, 8, 16, 32, -3, -16, -64]  # depths and row budgets


@pytest.mark.parametrize("which", ["c0", "skewed", "grid", "mixture"])
def test_features_match_oracle(which):
    torch_cuda()
    m = {"c0": lambda: S.gen_config("c0")[0], "skewed": lambda: S.gen_skewed(5000, 3, head=3000),
         "grid": lambda: S.gen_laplacian(40), "mixture": lambda: S.gen_mixture(8000, 10002)}[which]()
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    f = B.features(M, lv, DEPTHS).cpu().numpy()
    ref = OF.features(m.rowptr, m.colidx, DEPTHS)
    assert f.shape == ref.shape
    assert np.allclose(f, ref, rtol=2e-6, atol=1e-6)


def random_batch(n, seed):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((n, 12)) * 2 + 1).astype(np.float32)
    t = (X[:, :3].sum(axis=1) - 0.5 * X[:, 5] + 0.1 * rng.standard_normal(n)).astype(np.float32)
    return X, t


@pytest.mark.parametrize("bf16", [False, True])
def test_inference_matches_oracle(bf16):
    torch = torch_cuda()
    pk = B.Picker(seed=5)
    mean, std = np.linspace(-0.5, 0.5, 12), np.linspace(0.5, 2.0, 12)
    pk.set_norm(mean, std, 3.0)
    X, _ = random_batch(5000, 1)
    y = pk.infer(torch.from_numpy(X).cuda(), bf16=bf16).cpu().numpy()
    ref = OM.forward(pk.get_params(), X, mean.astype(np.float32), std.astype(np.float32), bf16=bf16)
    assert rel_l2(y, ref) < 1e-5


@pytest.mark.parametrize("bf16", [False, True])
def test_gradient_matches_oracle(bf16):
    torch = torch_cuda()
    pk = B.Picker(seed=7)
    mean, std = np.zeros(12), np.full(12, 1.5)
    pk.set_norm(mean, std, 2.0)
    X, t = random_batch(3000, 2)
    g, loss = pk.grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), bf16=bf16)
    lref, gref = OM.loss_and_grad(pk.get_params(), X, t, mean, std.astype(np.float32), target_scale=2.0, bf16=bf16)
    assert rel_l2(g.cpu().numpy(), gref) < (1e-4 if not bf16 else 1e-3)
    assert abs(float(loss.item()) - lref) <= 1e-5 * max(1.0, lref)


def test_adam_step_and_training_reduce_loss():
    torch = torch_cuda()
    pk = B.Picker(seed=11)
    X, t = random_batch(4096, 3)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    mean, std = X.mean(axis=0), X.std(axis=0)
    pk.set_norm(mean, std, float(t.std()))
    p0 = pk.get_params()
    # one step against the oracle's Adam (gradient through the bfloat16 weights)
    _, g = OM.loss_and_grad(p0, X, t, mean, std, float(np.float32(t.std())), bf16=True)
    p1_ref, _, _ = OM.adam_step(p0.astype(np.float64), np.zeros_like(g), np.zeros_like(g), g, 1, 1e-3)
    pk.train_step(Xd, td, 1e-3)
    assert rel_l2(pk.get_params(), p1_ref) < 1e-5
    losses = [float(pk.train_step(Xd, td, 2e-3).item()) for _ in range(300)]
    assert losses[-1] < 0.3 * losses[0]


def test_save_load_roundtrip(tmp_path):
    torch = torch_cuda()
    pk = B.Picker(seed=3)
    pk.set_norm(np.arange(12), np.ones(12) * 2, 5.0)
    path = str(tmp_path / "p.bin")
    pk.save(path)
    q = B.Picker.load(path)
    assert np.array_equal(q.get_params(), pk.get_params())
    X, _ = random_batch(100, 4)
    Xd = torch.from_numpy(X).cuda()
    assert torch.equal(pk.infer(Xd), q.infer(Xd))


def constant_picker(value):
    pk = B.Picker(seed=0)
    p = np.zeros(B.PICKER_PARAMS, np.float32)
    p[-1] = value  # output bias only: every candidate predicts `value`
    pk.set_params(p)
    return pk


def test_learned_rewrite_extremes_match_oracle_plans():
    torch = torch_cuda()
    m = S.gen_skewed(20000, 4, head=15000)
    _, b = S.rhs_from_xtrue(m, 1, 5)
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    lev, mm = O.levels(m.rowptr, m.colidx)
    bt = torch.from_numpy(b).cuda()
    ref = O.forward_subst(m.rowptr, m.colidx, m.vals, b)
    # predictions all positive: no candidate helps, nothing is rewritten
    s0 = B.System(M, lv, B.LEARNED, cap=1.5, picker=constant_picker(1.0), model_only=True)
    assert s0.info["rows_moved"] == 0 and s0.m == mm
    # all negative and equal: the first depth with the lowest prediction (the smallest), on thin levels
    s1 = B.System(M, lv, B.LEARNED, cap=1.5, picker=constant_picker(-1.0), depths=[4, 8], model_only=True)
    p = O.plan(m.rowptr, m.colidx, lev, mm, O.CHOSEN_THIN, cap=1.5, depth_of_target=np.full(mm, 4))
    assert np.array_equal(s1.export()["target"], p.target)
    for s in (s0, s1):
        x = s.solve(bt, check_status=True).cpu().numpy()
        assert rel_l2(x, ref) < TOL_F64


def test_learned_without_picker_falls_back_to_naive():
    torch_cuda()
    m, _, _ = S.gen_config("c0")
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    a = B.System(M, lv, B.LEARNED, cap=1.5).export()["target"]
    b = B.System(M, lv, B.NAIVE, cap=1.5).export()["target"]
    assert np.array_equal(a, b)


def test_learned_keeps_the_faster_of_model_and_naive():
    """The paper's strategy and no rewrite are the fallbacks: with a model that rewrites
    nothing, the measured solve time keeps the naive plan (or the plain system) on a
    chain-heavy matrix; the solution is right whichever is kept."""
    torch = torch_cuda()
    m = S.gen_skewed(60000, 13, head=30000)
    _, b = S.rhs_from_xtrue(m, 1, 5)
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    s = B.System(M, lv, B.LEARNED, cap=1.5, picker=constant_picker(1.0))
    # the kept plan is the candidate with the lowest measured time (model, naive, ROWCAP, plain)
    cand = s.info["candidate_us"]
    assert all(c > 0 for c in cand)
    kinds = [B.CHOSEN, B.NAIVE, B.ROWCAP, B.NONE]
    assert s.info["strategy_used"] == kinds[int(np.argmin(cand))], cand
    naive = B.System(M, lv, B.NAIVE, cap=1.5)
    if s.info["strategy_used"] == B.NAIVE:
        assert np.array_equal(s.export()["target"], naive.export()["target"])
    if s.info["strategy_used"] in (B.NONE, B.CHOSEN):  # the model predicts no gain: its plan rewrites nothing
        assert s.info["rows_moved"] == 0 and s.m == lv.m
    x = s.solve(torch.from_numpy(b).cuda(), check_status=True).cpu().numpy()
    assert rel_l2(x, O.forward_subst(m.rowptr, m.colidx, m.vals, b)) < TOL_F64
