"""Pins for the picker oracles (MLP and features): finite differences, closed forms,
and a library bfloat16 conversion as a second opinion."""
import math

import numpy as np
import pytest

from oracle import features as OF
from oracle import mlp as OM
from paper_2206_05843_gb300 import synth as S


def test_bf16_rounding_known_values_and_torch():
    one = 1.0
    vals = np.array([one, one + 2 ** -8, one + 3 * 2 ** -8, -2.5, 3.14159, 1e-3, 65504.0], dtype=np.float32)
    r = OM.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                 # tie -> even mantissa
    assert r[2] == 1.0 + 2 ** -6       # tie -> even mantissa (upwards)
    assert r[3] == -2.5
    torch = pytest.importorskip("torch")
    ref = torch.tensor(vals).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(r, ref)
    rnd = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 100
    assert np.array_equal(OM.bf16_round(rnd), torch.tensor(rnd).to(torch.bfloat16).to(torch.float64).numpy())


def test_forward_closed_form_identity_network():
    p = np.zeros(OM.NPARAM)
    W1, b1, W2, b2, W3, b3, W4, b4 = OM.unpack(p)
    W1[:12, :12] = np.eye(12)
    W2[:] = np.eye(64)
    W3[:] = np.eye(64)
    W4[:] = 1.0
    b4[:] = 0.5
    X = np.random.default_rng(1).standard_normal((20, 12))
    y = OM.forward(p, X)
    assert np.allclose(y, np.maximum(X, 0).sum(axis=1) + 0.5, rtol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    p = OM.init_params(seed).astype(np.float64) + rng.uniform(-0.05, 0.05, OM.NPARAM)
    X = rng.standard_normal((16, 12))
    t = rng.standard_normal(16)
    mean, std = rng.standard_normal(12) * 0.1, rng.uniform(0.5, 2.0, 12)
    loss, g = OM.loss_and_grad(p, X, t, mean, std, target_scale=2.0)
    idx = rng.choice(OM.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (OM.loss_and_grad(pp, X, t, mean, std, 2.0)[0] - OM.loss_and_grad(pm, X, t, mean, std, 2.0)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adam_first_step_is_sign_step():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p, m, v = OM.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, lr=0.01)
    assert np.allclose(p[:3], -0.01 * np.sign(g[:3]), rtol=1e-5)
    assert p[3] == 0.0


def test_training_reduces_loss_on_a_linear_target():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((256, 12))
    t = X @ rng.standard_normal(12)
    p = OM.init_params(1).astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = OM.loss_and_grad(p, X, t)[0]
    for step in range(1, 201):
        _, g = OM.loss_and_grad(p, X, t)
        p, m, v = OM.adam_step(p, m, v, g, step, 1e-3)
    assert OM.loss_and_grad(p, X, t)[0] < 0.1 * l0


def test_features_chain_closed_form():
    """A chain: one row per level, in-degree 1 (row 0: 0); cost 1 then 3 per level."""
    n = 50
    m = S.gen_from_deps(n, np.array([0] + [1] * (n - 1)), np.arange(n - 1), S.rng_for(0))
    depths = [1, 4, 8]
    F = OF.features(m.rowptr, m.colidx, depths).reshape(n, len(depths), 12)
    avg = (1 + 3 * (n - 1)) / n
    for t in (0, 5, 45, 49):
        for d, g in enumerate(depths):
            te = min(t + g, n - 1)
            f = F[t, d]
            assert f[0] == pytest.approx(math.log2(1 + g))
            assert f[1] == pytest.approx(math.log2(1 + te - t + 1))
            nnzW = sum(1 if l == 0 else 2 for l in range(t, te + 1))
            assert f[2] == pytest.approx(math.log2(1 + nnzW))
            if te > t:
                assert f[3] == pytest.approx(1.0)      # log2(1 + 1)
                assert f[4] == pytest.approx(1.0)
                assert f[5] == 1
                twohop = sum(1 if l >= 2 else 0 for l in range(t + 1, te + 1))
                assert f[6] == pytest.approx(math.log2(1 + twohop))
            else:
                assert f[3] == 0 and f[5] == 0
            assert f[7] == pytest.approx(1.0)
            assert f[8] == pytest.approx(1.0 if t > 0 else 0.0)
            assert f[9] == pytest.approx(1.0 if te + 1 < n else 0.0)
            costW = sum(1 if l == 0 else 3 for l in range(t, te + 1))
            assert f[10] == pytest.approx(costW / avg, rel=1e-6)
            thin = sum(1 for l in range(t, te + 1) if (1 if l == 0 else 3) < avg)
            assert f[11] == pytest.approx(thin / (te - t + 1))


def test_features_grid_widths():
    side = 9
    m = S.gen_laplacian(side)
    F = OF.features(m.rowptr, m.colidx, [2]).reshape(-1, 12)
    mm = 2 * side - 1
    width = [min(l + 1, mm - l) for l in range(mm)]
    for t in range(mm):
        te = min(t + 2, mm - 1)
        assert F[t, 7] == pytest.approx(math.log2(1 + width[t]))
        assert F[t, 1] == pytest.approx(math.log2(1 + sum(width[t:te + 1])))


def test_row_capped_candidates_closed_forms():
    """A row budget -r: on a chain (one row per level) the window holds r levels, g = r - 1 (cut at
    the last level); on the 9 x 9 grid (widths 1, 2, ..., 9, ..., 1) the depths follow the widths;
    the candidate's features are those of the fixed depth it resolves to."""
    n = 40
    chain = S.gen_from_deps(n, np.array([0] + [1] * (n - 1)), np.arange(n - 1), S.rng_for(0))
    rows = np.ones(n, np.int64)
    for t in (0, 10, 35, 39):
        assert OF.candidate_depth(rows, t, -8) == min(7, n - 1 - t)
        assert OF.candidate_depth(rows, t, -1) == 0
    F = OF.features(chain.rowptr, chain.colidx, [-8, 7, 3]).reshape(n, 3, 12)
    assert np.array_equal(F[10, 0], F[10, 1])  # -8 resolves to depth 7 at t = 10
    assert np.array_equal(F[36, 0], F[36, 2])  # and to depth 3 at t = 36 (3 levels left)
    side = 9
    grid = S.gen_laplacian(side)
    width = np.array([min(l + 1, 2 * side - 1 - l) for l in range(2 * side - 1)])
    # widths 1,2,3,4,... : a budget of 10 rows takes levels 0..3 from t = 0 (1+2+3+4 = 10)
    assert OF.candidate_depth(width, 0, -10) == 3
    assert OF.candidate_depth(width, 0, -9) == 2
    assert OF.candidate_depth(width, 8, -9) == 0    # level 8 alone holds 9 rows
    assert OF.candidate_depth(width, 8, -8) == 0    # more than the budget: no rewrite
    assert OF.candidate_depth(width, 13, -9) == 2   # widths 4, 3, 2 = 9
    assert OF.candidate_depth(width, 16, -100) == 0  # the last level has nothing after it
