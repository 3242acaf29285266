"""Host-side arithmetic of bench.py on CPU: the dependent-FP64 chain floor and the algorithmic
bytes of a solve, against hand counts on small systems."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class FakeSystem:
    """What chain_floor reads: the level count and the exported level / row pointer arrays."""

    def __init__(self, level, cptr):
        self.m = int(max(level) + 1) if len(level) else 0
        self._ex = {"level": np.asarray(level, np.int32), "cptr": np.asarray(cptr, np.int64)}

    def export(self):
        return self._ex


def test_chain_floor_counts_product_and_add_tree():
    # level 0: two rows without dependencies (1 op); level 1: rows with 1 and 3 coefficients
    # (longest 3 -> 1 + ceil(log2 3) = 3 ops); level 2: one row with 4 (1 + 2 = 3 ops)
    level = [0, 0, 1, 1, 2]
    cptr = [0, 0, 0, 1, 4, 8]
    out = bench.chain_floor(FakeSystem(level, cptr), 1000.0)
    assert out["levels"] == 3
    assert out["dependent_fp64_ops"] == 1 + 3 + 3
    assert abs(out["floor_us"] - 7 * bench.FP64_LATENCY_CYCLES / 1000.0) < 0.11


def test_alg_bytes_plain_and_rewritten():
    n, nnz_c = 10, 20
    plain = {"nnz_c": nnz_c, "nnz_e": 0, "rows_moved": 0, "rewritten": 0}
    # 4(n+1) + (4+v)(nnz_c + n) + 2 v n r
    assert bench.alg_bytes(plain, n, 1) == 4 * 11 + 12 * 30 + 2 * 8 * 10
    assert bench.alg_bytes(plain, n, 3, v=4) == 4 * 11 + 8 * 30 + 2 * 4 * 10 * 3
    rw = {"nnz_c": nnz_c, "nnz_e": 7, "rows_moved": 4, "rewritten": 1}
    # plus 4(n_rw + 1) + (4+v) nnz_e for the E rows
    assert bench.alg_bytes(rw, n, 1) == bench.alg_bytes(plain, n, 1) + 4 * 5 + 12 * 7


def test_rel_residual_of_an_exact_and_a_perturbed_solution():
    from paper_2206_05843_gb300 import synth as S
    m = S.gen_banded_random(300, 2)
    xt, b = S.rhs_from_xtrue(m, 2, 3)
    assert bench.rel_residual(m, xt, b) < 1e-14
    x = xt.copy()
    x[1, 7] += 1.0
    # the perturbation shows up as column 7 of L in the second right-hand side
    col7 = np.zeros(m.n)
    rp = m.rowptr.astype(np.int64)
    for i in range(m.n):
        for q in range(rp[i], rp[i + 1]):
            if m.colidx[q] == 7:
                col7[i] = m.vals[q]
    assert abs(bench.rel_residual(m, x, b) - np.linalg.norm(col7) / np.linalg.norm(b[1])) < 1e-12


def test_flat_extras_keeps_time_and_fraction_or_the_error():
    ex = {"w2": {"us": 200.0, "hbm_frac": 0.5, "gbs": 3000.0}, "c3": {"error": "RuntimeError: x"},
          "w1r16": {"us": 955.0, "hbm_frac": 0.19, "fp64_frac": 0.56}}
    assert bench.flat_extras(ex) == {"w2_us": 200.0, "w2_hbm_frac": 0.5, "c3_error": "RuntimeError: x",
                                     "w1r16_us": 955.0, "w1r16_hbm_frac": 0.19, "w1r16_fp64_frac": 0.56}


def test_fp64_issue_bound_of_a_known_workload():
    """float64 operations per solve and the full-issue rate: n = 4,194,304 rows with 4 off-diagonal
    entries in all but 8,192 rows and 16 right-hand sides need about 335 M operations, 533 us at
    152 SMs x 2 operations a cycle at 2,070 MHz."""
    n = 2048 * 2048
    nnz_c = 4 * n - 4 * 2048
    ops = bench.fp64_ops({"nnz_c": nnz_c, "nnz_e": 0, "n": n}, 16)
    assert ops == (nnz_c + n) * 16
    peak = bench.fp64_peak(152, 2070.0)
    assert peak == 152 * 2 * 2070e6
    assert 520e-6 < ops / peak < 540e-6


def test_cpu_oracle_preprocessing_times_every_step():
    """The bench's CPU preprocessing baseline times the oracle's level analysis and the naive and
    row-capped plans and rewrites on the workload it is given (a small skewed matrix here)."""
    from paper_2206_05843_gb300 import synth as S
    m, _, _ = S.gen_config("c1", scale=0.01)
    out = bench.cpu_oracle_preprocessing(m)
    assert set(out) == {"oracle_cpu_levels_ms", "oracle_cpu_plan_naive_ms", "oracle_cpu_rewrite_naive_ms",
                        "oracle_cpu_plan_rowcap_ms", "oracle_cpu_rewrite_rowcap_ms"}
    assert all(isinstance(v, float) and v >= 0 for v in out.values())
