"""Upper-triangular solves U x = b (index reversal onto the lower-triangular path)
against the CPU oracle's backward substitution."""
import numpy as np
import pytest

import oracle as O
from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S
from tests.gpu_util import TOL_F64, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def upper_from_lower(m):
    """U = L^T in CSR with the diagonal first (numpy, input construction only)."""
    rp = m.rowptr.astype(np.int64)
    rows = np.repeat(np.arange(m.n), np.diff(rp))
    order = np.lexsort((rows, m.colidx))  # by column of L = row of U, then by row of L
    urow = m.colidx[order].astype(np.int64)
    ucol = rows[order].astype(np.int32)
    uval = m.vals[order]
    urp = np.zeros(m.n + 1, np.int64)
    np.add.at(urp, urow + 1, 1)
    return S.LowerCsr(m.n, np.cumsum(urp).astype(np.int32), ucol, uval)


@pytest.mark.parametrize("kind", [B.NONE, B.NAIVE, B.DEPTH_K])
def test_upper_solve_matches_backward_substitution(kind):
    torch = torch_cuda()
    L = S.gen_skewed(30000, 6, head=20000)
    U = upper_from_lower(L)
    b = S.rhs_uniform(U.n, 2, 4)
    ref = O.backward_subst(U.rowptr, U.colidx, U.vals, b)
    kw = {"k": 3} if kind == B.DEPTH_K else ({"cap": 1.5} if kind == B.NAIVE else {})
    x, s, _ = B.solve_upper(B.Matrix.from_host(U), torch.from_numpy(b).cuda(), kind, **kw)
    assert rel_l2(x.cpu().numpy(), ref) <= TOL_F64


def test_upper_to_lower_structure():
    torch = torch_cuda()
    L = S.gen_banded_random(500, 2)
    U = upper_from_lower(L)
    R = B.upper_to_lower(B.Matrix.from_host(U))
    n = U.n
    Ud = np.zeros((n, n))
    for i in range(n):
        Ud[i, U.colidx[U.rowptr[i]:U.rowptr[i + 1]]] = U.vals[U.rowptr[i]:U.rowptr[i + 1]]
    Rd = np.zeros((n, n))
    rp, ci, va = R.rowptr.cpu().numpy(), R.colidx.cpu().numpy(), R.vals.cpu().numpy()
    for i in range(n):
        Rd[i, ci[rp[i]:rp[i + 1]]] = va[rp[i]:rp[i + 1]]
    assert np.array_equal(Rd, Ud[::-1, ::-1])
    R.validate()
