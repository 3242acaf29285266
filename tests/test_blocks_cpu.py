"""The host block cutter of the single-CTA executor, on CPU through its test hook: blocks
partition the positions in order; fast blocks hold whole levels within the warp's lanes and the
record capacity, with one K per block; other blocks respect the staging limits; no level that
qualifies for a fast block starts inside another block."""
import numpy as np
import pytest

import oracle as O
from paper_2206_05843_gb300 import binding as B
from paper_2206_05843_gb300 import synth as S

NARROW, FAST, KSHIFT, NLMASK = 1 << 30, 1 << 29, 26, (1 << 26) - 1


def stored_order(m):
    """Level pointer and coefficient row pointer of the plain system in level order."""
    lev, mm = O.levels(m.rowptr, m.colidx)
    order = np.lexsort((np.arange(m.n), lev))
    lp = np.concatenate([[0], np.cumsum(np.bincount(lev, minlength=mm))]).astype(np.int32)
    length = (np.diff(m.rowptr) - 1)[order]
    cptr = np.concatenate([[0], np.cumsum(length)]).astype(np.int32)
    return lp, cptr


def check_blocks(lp, cptr, nrhs, lpr, vb):
    blocks, g = B.run_blocks(lp, cptr, nrhs=nrhs, lanes_per_row=lpr, value_bytes=vb)
    n, m = int(lp[-1]), lp.size - 1
    r2 = 1
    while r2 < nrhs:
        r2 <<= 1
    r2 //= 2 if nrhs > 16 else 1
    fast_on = nrhs <= 32 and (lpr in (1, 2) or (lpr == 4 and nrhs == 1))
    level_of = np.repeat(np.arange(m), np.diff(lp))

    def k_of(level):
        rows = lp[level + 1] - lp[level]
        if not fast_on or rows * lpr * r2 > 32:
            return 0
        mx = int((cptr[lp[level] + 1:lp[level + 1] + 1] - cptr[lp[level]:lp[level + 1]]).max())
        k = max(1, -(-mx // lpr))
        return k if k <= 4 else 0

    assert blocks[0, 0] == 0 and blocks[-1, 1] == n
    assert np.array_equal(blocks[1:, 0], blocks[:-1, 1])
    for p0, p1, l0, w in blocks:
        nl = w & NLMASK
        assert p1 > p0 and l0 == level_of[p0] and nl == level_of[p1 - 1] - l0 + 1
        if w & FAST:
            assert w & NARROW
            assert p0 == lp[l0] and p1 == lp[l0 + nl]  # whole levels
            ks = [k_of(l) for l in range(l0, l0 + nl)]
            assert min(ks) > 0
            kb = (w >> KSHIFT) & 7
            assert kb == max(ks)
            assert kb * lpr * (p1 - p0) <= g["fast_records"] and p1 - p0 <= g["stage_rows"]
        else:
            rows, ents = p1 - p0, cptr[p1] - cptr[p0]
            if nl > 1:
                assert rows <= g["stage_rows"] and ents <= g["stage_entries"]
            # a level qualifying for a fast block never starts inside this block
            for l in range(l0 + 1, l0 + nl):
                assert k_of(l) == 0
            if p0 == lp[l0]:
                assert k_of(l0) == 0
    return blocks, g


@pytest.mark.parametrize("nrhs,lpr", [(1, 1), (1, 2), (1, 4), (3, 1), (17, 1), (32, 2), (64, 1)])
@pytest.mark.parametrize("vb", [8, 4])
def test_block_cutter_invariants(nrhs, lpr, vb):
    for m in (S.gen_skewed(30000, 3, head=20000), S.gen_config("c0")[0], S.gen_mixture(20000, 10007)):
        lp, cptr = stored_order(m)
        blocks, g = check_blocks(lp, cptr, nrhs, lpr, vb)
        assert g["ring_rows"] >= 2 * g["stage_rows"]
        if nrhs == 1 and lpr == 1 and m.name.startswith("skewed"):
            assert (blocks[:, 3] & FAST).any()


def test_block_cutter_splits_a_level_too_large_for_the_stage():
    # one level of 5,000 independent rows after a root: split by rows, never fast
    n = 5001
    lp = np.array([0, 1, n], np.int32)
    cptr = np.concatenate([[0, 0], np.arange(1, n)]).astype(np.int32)  # every row depends on the root
    blocks, g = check_blocks(lp, cptr, 1, 1, 8)
    assert len(blocks) >= 2 and not (blocks[1:, 3] & FAST).any()
    assert (blocks[:, 1] - blocks[:, 0]).max() <= g["stage_rows"]


def test_block_cutter_random_structures():
    """Random level widths (1..70 rows) and row lengths (0..20 coefficients): the invariants hold
    for every lanes / right-hand-side choice the executor supports."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=60, deadline=None)
    @hyp.given(widths=st.lists(st.integers(1, 70), min_size=1, max_size=120),
               seed=st.integers(0, 2**31 - 1),
               cfg=st.sampled_from([(1, 1, 8), (1, 2, 8), (1, 4, 8), (2, 1, 8), (20, 2, 8), (1, 1, 4), (7, 2, 4)]))
    def run(widths, seed, cfg):
        rng = np.random.default_rng(seed)
        n = int(sum(widths))
        lp = np.concatenate([[0], np.cumsum(widths)]).astype(np.int32)
        length = rng.integers(0, 21, n)
        length[: widths[0]] = 0  # the first level has no dependencies
        cptr = np.concatenate([[0], np.cumsum(length)]).astype(np.int32)
        check_blocks(lp, cptr, *cfg)

    run()
