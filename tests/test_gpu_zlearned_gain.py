"""The learned gain of the committed trained picker on held-out mixtures (timed on the GPU;
after the parity files, so that a slow or noisy box cannot hide them)."""
import os

import numpy as np
import pytest

from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S
from tests.gpu_util import TOL_F64, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def _median_solve_us(sysm, bt, reps=9):
    torch = torch_cuda()
    x = torch.empty_like(bt)
    for _ in range(2):
        sysm.solve(bt, x)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sysm.solve(bt, x)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e3)
    sysm.status()
    return float(np.median(ts)), x


def test_trained_picker_gain_on_held_out_mixtures():
    """The learned gain with the committed trained picker, on the first three held-out mixtures
    (seeds 20,000+, sizes drawn as in the evaluation): the learned strategy is at least as fast as
    the paper's naive strategy (10% timing tolerance), clearly faster than the plain solve on each
    matrix and by 1.3x in geometric mean, and exact to 1e-10."""
    torch = torch_cuda()
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2206_05843_gb300",
                        "picker_trained.bin")
    pk = B.Picker.load(path)
    erng = S.rng_for(54321)
    gains = []
    for i in range(3):
        n = int(round(np.exp(erng.uniform(np.log(100_000), np.log(1_000_000)))))
        m = S.gen_mixture(n, 20_000 + i)
        xt, b = S.rhs_from_xtrue(m, 1, 7)
        M = B.Matrix.from_host(m)
        lv = B.Levels(M)
        bt = torch.from_numpy(b[0]).cuda()
        t_plain, _ = _median_solve_us(B.System(M, lv), bt)
        t_naive, _ = _median_solve_us(B.System(M, lv, B.NAIVE, cap=1.5), bt)
        learned = B.System(M, lv, B.LEARNED, cap=1.5, picker=pk)
        t_learned, x = _median_solve_us(learned, bt)
        assert rel_l2(x.cpu().numpy(), xt[0]) < TOL_F64
        assert t_learned <= 1.10 * t_naive, (i, t_learned, t_naive, learned.info["strategy_used"])
        assert t_plain / t_learned >= 1.15, (i, t_plain, t_learned)
        gains.append(t_plain / t_learned)
    assert float(np.exp(np.mean(np.log(gains)))) >= 1.3, gains


def test_bench_configuration_full_size_matches_oracle():
    """The configuration bench.py times, at full size: the skewed n = 1,000,000 matrix, the
    learned strategy with the trained picker under the 1.5 nnz cap, the autotuned schedule;
    the solution against the oracle's forward substitution of the original system."""
    import oracle as O
    torch = torch_cuda()
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2206_05843_gb300",
                        "picker_trained.bin")
    m, b, xt = S.gen_config("c1")
    M = B.Matrix.from_host(m)
    lv = B.Levels(M)
    s = B.System(M, lv, B.LEARNED, cap=1.5, picker=B.Picker.load(path))
    s.autotune(1)
    assert s.info["stored_nnz"] <= 1.5 * s.info["nnz_l"]
    x = s.solve(torch.from_numpy(b).cuda(), check_status=True).cpu().numpy()
    assert rel_l2(x, O.forward_subst(m.rowptr, m.colidx, m.vals, b)) < TOL_F64
    assert rel_l2(x, xt) < 1e-12


def test_trained_network_own_plan_on_held_out_mixtures():
    """What the trained network itself gains: its own plan (the learned strategy with model_only,
    no fallback) against the paper's naive strategy on the first three held-out mixtures, in
    geometric mean; and the learned strategy's measured choice with the network against the same
    choice without it (naive, ROWCAP, no rewrite).  Solutions exact to 1e-10."""
    torch = torch_cuda()
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2206_05843_gb300",
                        "picker_trained.bin")
    pk = B.Picker.load(path)
    erng = S.rng_for(54321)
    own, with_vs_without = [], []
    for i in range(3):
        n = int(round(np.exp(erng.uniform(np.log(100_000), np.log(1_000_000)))))
        m = S.gen_mixture(n, 20_000 + i)
        xt, b = S.rhs_from_xtrue(m, 1, 7)
        M = B.Matrix.from_host(m)
        lv = B.Levels(M)
        bt = torch.from_numpy(b[0]).cuda()
        t = {}
        for name, kw in (("none", {}), ("naive", dict(kind=B.NAIVE, cap=1.5)),
                         ("rowcap", dict(kind=B.ROWCAP, k=32, cap=1.5)),
                         ("model", dict(kind=B.LEARNED, cap=1.5, picker=pk, model_only=True))):
            sysm = B.System(M, lv, **kw)
            t[name], x = _median_solve_us(sysm, bt)
            assert rel_l2(x.cpu().numpy(), xt[0]) < TOL_F64, name
        own.append(t["naive"] / t["model"])
        without = min(t["naive"], t["rowcap"], t["none"])
        with_vs_without.append(without / min(without, t["model"]))
    g_own = float(np.exp(np.mean(np.log(own))))
    g_choice = float(np.exp(np.mean(np.log(with_vs_without))))
    print(f"network's plan over naive: {own} (geomean {g_own:.3f}); "
          f"choice with / without the network: {with_vs_without} (geomean {g_choice:.3f})")
    assert g_own >= 1.0, own
    # the network's plan is the fastest of all four candidates on at least one of the matrices
    assert max(with_vs_without) > 1.0, with_vs_without
