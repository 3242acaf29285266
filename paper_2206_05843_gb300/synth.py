"""Seeded synthetic inputs: sparse lower-triangular CSR matrices and right-hand sides.

This module draws inputs only; it holds none of the solver's arithmetic (no forward
substitution, no level sets, no rewriting).  Both the CPU oracle tests and the CUDA
path consume the arrays it returns, so parity compares the two on identical data.

Conventions shared by every generator (the problem statement of Section II.A and the
CSR layout of Algorithm 1): row i of L holds its off-diagonal columns in ascending
order followed by the diagonal entry, which is the last entry of the row.  Column
indices and row pointers are int32, values float64.  Generators draw with numpy's
PCG64, which gives the same stream on x86-64 and aarch64.

Workload recipes (the paper's lung2 / torso2 matrices are not available, so these
shapes stand in for its long chains of thin levels and its triangular level profile):

* ``gen_banded_random``  n rows, min(k, window) distinct columns uniform in
  [max(0, i-band), i), off-diagonals U[-1, 1], diagonal 1 + sum|off|.
* ``gen_skewed``         head rows with min(8, i) distinct columns uniform over [0, i)
  (few wide levels), tail rows with 3 distinct columns of [i-4, i) (a near-serial chain).
* ``gen_laplacian``      lower triangle of the 5-point Laplacian on an s x s grid in
  natural order: diagonal 4, neighbours (r-1, c) and (r, c-1) with value -1.
* ``gen_redblack``       the same grid in red-black order: two levels.
* ``gen_layered``        L layers of equal size; each row of layer >= 1 has k distinct
  dependencies uniform over all earlier layers, at least one in the previous layer.
* ``gen_batch``          many matrices of log-uniform size drawn from the first three.
* ``gen_mixture``        concatenated head / tail / grid blocks with random proportions.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "LowerCsr", "rng_for", "gen_banded_random", "gen_skewed", "gen_laplacian",
    "gen_redblack", "gen_layered", "gen_from_deps", "rhs_uniform", "rhs_from_xtrue",
    "gen_config", "gen_batch", "gen_mixture", "BatchItem",
]


@dataclass
class LowerCsr:
    """A lower-triangular CSR matrix with the diagonal stored last in each row."""

    n: int
    rowptr: np.ndarray  # int32[n+1]
    colidx: np.ndarray  # int32[nnz]
    vals: np.ndarray  # float64[nnz]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def astype(self, dtype) -> "LowerCsr":
        return LowerCsr(self.n, self.rowptr, self.colidx, self.vals.astype(dtype),
                        self.name, dict(self.meta))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=np.float64)
        for i in range(self.n):
            a, b = int(self.rowptr[i]), int(self.rowptr[i + 1])
            d[i, self.colidx[a:b]] = self.vals[a:b]
        return d


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# ----------------------------------------------------------------------------------
# assembly helpers
# ----------------------------------------------------------------------------------

def gen_from_deps(n: int, counts: np.ndarray, cols: np.ndarray, rng: np.random.Generator | None,
                  offdiag: np.ndarray | float | None = None, diag: np.ndarray | float | None = None,
                  name: str = "") -> LowerCsr:
    """Assemble CSR from per-row sorted dependency columns (flattened in row order).

    Off-diagonal values are U[-1, 1] unless given; the diagonal defaults to
    1 + sum of |off-diagonals| of the row (strict diagonal dominance).
    """
    counts = np.asarray(counts, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    assert counts.shape == (n,) and cols.size == int(counts.sum())
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(counts + 1)
    nnz = int(rowptr[-1])
    if nnz >= 2**31:
        raise ValueError("nnz does not fit int32 row pointers")
    diag_pos = rowptr[1:] - 1
    is_off = np.ones(nnz, dtype=bool)
    is_off[diag_pos] = False
    colidx = np.empty(nnz, dtype=np.int32)
    colidx[is_off] = cols
    colidx[diag_pos] = np.arange(n, dtype=np.int32)
    if offdiag is None:
        off = rng.uniform(-1.0, 1.0, size=cols.size) if cols.size else np.zeros(0)
    else:
        off = np.broadcast_to(np.asarray(offdiag, dtype=np.float64), (cols.size,))
    vals = np.empty(nnz, dtype=np.float64)
    vals[is_off] = off
    if diag is None:
        rowid = np.repeat(np.arange(n), counts)
        vals[diag_pos] = 1.0 + np.bincount(rowid, weights=np.abs(off), minlength=n)
    else:
        vals[diag_pos] = np.broadcast_to(np.asarray(diag, dtype=np.float64), (n,))
    return LowerCsr(n, rowptr.astype(np.int32), colidx, vals, name)


def _take_all(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Flattened ranges [lo_r, hi_r) for every row r."""
    w = hi - lo
    if w.sum() == 0:
        return np.zeros(0, dtype=np.int64)
    starts = np.repeat(lo - np.concatenate(([0], np.cumsum(w)[:-1])), w)
    return starts + np.arange(int(w.sum()))


def _distinct_uniform(rng: np.random.Generator, lo: np.ndarray, hi: np.ndarray,
                      k: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Per row r: k_r distinct integers uniform in [lo_r, hi_r), sorted ascending.

    Returns (counts, flat columns in row order).  k_r is clipped to the window size.
    """
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    w = hi - lo
    k = np.minimum(np.asarray(k, dtype=np.int64), w)
    n = lo.size
    rows_all = np.nonzero(k == w)[0]
    rows_rest = np.nonzero(k < w)[0]
    # exclude-one rows (k == w - 1): draw the excluded element
    ex = rows_rest[k[rows_rest] == w[rows_rest] - 1]
    small = rows_rest[(k[rows_rest] < w[rows_rest] - 1) & (w[rows_rest] <= 4 * k[rows_rest])]
    big = rows_rest[(k[rows_rest] < w[rows_rest] - 1) & (w[rows_rest] > 4 * k[rows_rest])]
    # assemble into a dense (n, kmax) array padded with -1, then flatten
    kmax = int(k.max()) if n else 0
    dense = np.full((n, max(kmax, 1)), -1, dtype=np.int64)
    if rows_all.size:
        flat = _take_all(lo[rows_all], hi[rows_all])
        pos = np.repeat(np.arange(rows_all.size), k[rows_all])
        within = np.arange(flat.size) - np.repeat(np.cumsum(k[rows_all]) - k[rows_all], k[rows_all])
        dense[rows_all[pos], within] = flat
    if ex.size:
        excl = lo[ex] + rng.integers(0, w[ex])
        for kval in np.unique(k[ex]):
            sel = ex[k[ex] == kval]
            e = excl[k[ex] == kval]
            base = lo[sel][:, None] + np.arange(kval + 1)[None, :]
            keep = base != e[:, None]
            dense[sel, :kval] = base[keep].reshape(sel.size, kval)
    for r in small:
        c = rng.choice(int(w[r]), size=int(k[r]), replace=False) + lo[r]
        dense[r, :k[r]] = np.sort(c)
    for kval in np.unique(k[big]) if big.size else []:
        pend = big[k[big] == kval]
        while pend.size:
            draw = lo[pend][:, None] + np.floor(rng.random((pend.size, kval)) * w[pend][:, None]).astype(np.int64)
            draw.sort(axis=1)
            dup = np.any(draw[:, 1:] == draw[:, :-1], axis=1) if kval > 1 else np.zeros(pend.size, bool)
            ok = ~dup
            dense[pend[ok], :kval] = draw[ok]
            pend = pend[dup]
    mask = np.arange(dense.shape[1])[None, :] < k[:, None]
    return k, dense[mask]


# ----------------------------------------------------------------------------------
# matrix generators
# ----------------------------------------------------------------------------------

def gen_banded_random(n: int, seed: int, k: int = 5, band: int = 200) -> LowerCsr:
    """min(k, window) distinct columns uniform in [max(0, i-band), i); dominant diagonal."""
    rng = rng_for(seed)
    i = np.arange(n, dtype=np.int64)
    lo = np.maximum(0, i - band)
    counts, cols = _distinct_uniform(rng, lo, i, np.full(n, k))
    m = gen_from_deps(n, counts, cols, rng, name=f"banded_random(n={n},k={k},band={band},seed={seed})")
    m.meta.update(kind="banded_random", seed=seed)
    return m


def gen_skewed(n: int, seed: int, head: int | None = None, k_head: int = 8, k_tail: int = 3,
               tail_window: int = 4) -> LowerCsr:
    """Head rows: min(k_head, i) distinct columns uniform over [0, i).  Tail rows:
    k_tail distinct columns of [i - tail_window, i).  Dominant diagonal."""
    rng = rng_for(seed)
    head = int(round(0.8 * n)) if head is None else int(head)
    i = np.arange(n, dtype=np.int64)
    lo = np.where(i < head, 0, np.maximum(0, i - tail_window))
    k = np.where(i < head, k_head, k_tail)
    counts, cols = _distinct_uniform(rng, lo, i, k)
    m = gen_from_deps(n, counts, cols, rng, name=f"skewed(n={n},head={head},seed={seed})")
    m.meta.update(kind="skewed", seed=seed, head=head)
    return m


def gen_laplacian(side: int) -> LowerCsr:
    """Lower triangle of the 5-point Laplacian on a side x side grid, natural order."""
    s = int(side)
    n = s * s
    idx = np.arange(n, dtype=np.int64)
    r, c = idx // s, idx % s
    has_up = r > 0
    has_left = c > 0
    counts = has_up.astype(np.int64) + has_left.astype(np.int64)
    # per row: (idx - s) then (idx - 1), ascending
    dense = np.full((n, 2), -1, dtype=np.int64)
    dense[:, 0] = np.where(has_up, idx - s, np.where(has_left, idx - 1, -1))
    dense[:, 1] = np.where(has_up & has_left, idx - 1, -1)
    mask = np.arange(2)[None, :] < counts[:, None]
    m = gen_from_deps(n, counts, dense[mask], None, offdiag=-1.0, diag=4.0,
                      name=f"laplacian({s}x{s})")
    m.meta.update(kind="laplacian", side=s)
    return m


def gen_redblack(side: int) -> LowerCsr:
    """5-point Laplacian on a side x side grid in red-black order (red: (r+c) even,
    first); lower triangle, so red rows are independent and black rows depend on
    their red neighbours."""
    s = int(side)
    n = s * s
    idx = np.arange(n, dtype=np.int64)
    r, c = idx // s, idx % s
    red = ((r + c) % 2) == 0
    newpos = np.empty(n, dtype=np.int64)
    nred = int(red.sum())
    newpos[red] = np.arange(nred)
    newpos[~red] = nred + np.arange(n - nred)
    # rows in new order
    order = np.argsort(newpos)
    ro, co = r[order], c[order]
    isred = red[order]
    nb = np.full((n, 4), -1, dtype=np.int64)
    for t, (dr, dc) in enumerate(((-1, 0), (0, -1), (0, 1), (1, 0))):
        rr, cc = ro + dr, co + dc
        ok = (rr >= 0) & (rr < s) & (cc >= 0) & (cc < s) & (~isred)
        nb[ok, t] = newpos[(rr * s + cc)[ok]]
    nb = np.where(nb < 0, np.iinfo(np.int64).max, nb)
    nb.sort(axis=1)
    counts = (nb != np.iinfo(np.int64).max).sum(axis=1)
    mask = np.arange(4)[None, :] < counts[:, None]
    m = gen_from_deps(n, counts, nb[mask], None, offdiag=-1.0, diag=4.0, name=f"redblack({s}x{s})")
    m.meta.update(kind="redblack", side=s)
    return m


def gen_layered(n_layers: int, layer_rows: int, seed: int, k: int = 8) -> LowerCsr:
    """Layered random DAG: rows of layer l >= 1 take one dependency uniform in layer
    l-1 and k-1 more distinct ones uniform over all earlier layers."""
    rng = rng_for(seed)
    n = n_layers * layer_rows
    idx = np.arange(n, dtype=np.int64)
    layer = idx // layer_rows
    counts = np.where(layer == 0, 0, k).astype(np.int64)
    dense = np.full((n, k), -1, dtype=np.int64)
    rows = np.nonzero(layer > 0)[0]
    L = layer[rows]
    first = (L - 1) * layer_rows + rng.integers(0, layer_rows, size=rows.size)
    pend = np.arange(rows.size)
    while pend.size:
        hi = L[pend] * layer_rows
        rest = np.floor(rng.random((pend.size, k - 1)) * hi[:, None]).astype(np.int64)
        allc = np.concatenate([first[pend][:, None], rest], axis=1)
        allc.sort(axis=1)
        dup = np.any(allc[:, 1:] == allc[:, :-1], axis=1)
        ok = ~dup
        dense[rows[pend[ok]]] = allc[ok]
        pend = pend[dup]
    mask = np.arange(k)[None, :] < counts[:, None]
    m = gen_from_deps(n, counts, dense[mask], rng, name=f"layered({n_layers}x{layer_rows},k={k},seed={seed})")
    m.meta.update(kind="layered", seed=seed)
    return m


# ----------------------------------------------------------------------------------
# right-hand sides
# ----------------------------------------------------------------------------------

def rhs_uniform(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Column-major right-hand sides: array of shape (nrhs, n), entries U[-1, 1]."""
    return rng_for(seed).uniform(-1.0, 1.0, size=(nrhs, n))


def rhs_from_xtrue(m: LowerCsr, nrhs: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """x_true U[-1, 1] (shape (nrhs, n)) and b = L x_true, column by column."""
    xt = rng_for(seed).uniform(-1.0, 1.0, size=(nrhs, m.n))
    rowid = np.repeat(np.arange(m.n), np.diff(m.rowptr.astype(np.int64)))
    b = np.empty_like(xt)
    for k in range(nrhs):
        b[k] = np.bincount(rowid, weights=m.vals.astype(np.float64) * xt[k][m.colidx], minlength=m.n)
    return xt, b


# ----------------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------------

def gen_config(name: str, seed: int = 0, scale: float = 1.0):
    """Named workloads.  Returns (matrix, b, x_true or None).

    c0  n=2,000 banded random (k=5, band 200), b = L x_true, 1 RHS
    c1  n=1,000,000 skewed (head 800,000), b = L x_true, 1 RHS
    c2  2048 x 2048 Laplacian, natural order, b U[-1, 1], 1 RHS (c2r16: 16 RHS)
    w1  2048 x 2048 Laplacian, red-black order, b = L x_true
    w2  8 layers x 524,288 rows, 8 deps, b = L x_true
    ``scale`` shrinks n for quick runs (1.0 = the full size).
    """
    if name == "c0":
        n = max(16, int(2000 * scale))
        m = gen_banded_random(n, seed)
        xt, b = rhs_from_xtrue(m, 1, seed + 1)
        return m, b, xt
    if name == "c1":
        n = max(64, int(1_000_000 * scale))
        m = gen_skewed(n, seed, head=int(round(0.8 * n)))
        xt, b = rhs_from_xtrue(m, 1, seed + 1)
        return m, b, xt
    if name in ("c2", "c2r16"):
        side = max(4, int(2048 * np.sqrt(scale)))
        m = gen_laplacian(side)
        b = rhs_uniform(m.n, 16 if name == "c2r16" else 1, seed + 1)
        return m, b, None
    if name == "w1":
        side = max(4, int(2048 * np.sqrt(scale)))
        m = gen_redblack(side)
        xt, b = rhs_from_xtrue(m, 1, seed + 1)
        return m, b, xt
    if name == "w2":
        rows = max(8, int(524_288 * scale))
        m = gen_layered(8, rows, 7 if seed == 0 else seed)
        xt, b = rhs_from_xtrue(m, 1, seed + 1)
        return m, b, xt
    raise KeyError(name)


@dataclass
class BatchItem:
    matrix: LowerCsr
    b: np.ndarray  # (nrhs, n)
    x_true: np.ndarray | None
    nrhs: int
    fp32: bool
    kind: int


def gen_batch(count: int = 256, base_seed: int = 1000, n_lo: int = 1000, n_hi: int = 65536,
              rhs_hi: int = 32) -> list[BatchItem]:
    """Matrices of log-uniform size from the banded / skewed / grid generators, each
    with 1..rhs_hi right-hand sides; even items float64 values, odd items float32."""
    top = rng_for(base_seed)
    items = []
    for idx in range(count):
        n = int(round(np.exp(top.uniform(np.log(n_lo), np.log(n_hi)))))
        kind = int(top.integers(0, 3))
        nrhs = int(top.integers(1, rhs_hi + 1))
        seed = base_seed + idx
        if kind == 0:
            m = gen_banded_random(n, seed)
        elif kind == 1:
            m = gen_skewed(n, seed, head=int(round(0.8 * n)))
        else:
            m = gen_laplacian(max(2, int(np.sqrt(n))))
        if kind == 2:
            xt, b = None, rhs_uniform(m.n, nrhs, seed + 7)
        else:
            xt, b = rhs_from_xtrue(m, nrhs, seed + 7)
        fp32 = (idx % 2) == 1
        items.append(BatchItem(m, b, xt, nrhs, fp32, kind))
    return items


def gen_mixture(n: int, seed: int) -> LowerCsr:
    """Concatenated blocks of the skewed head, the skewed tail and the grid, in random
    order with random proportions.  Head rows draw 8 columns inside their block; tail
    rows 3 of the previous 4 rows; grid rows follow the natural-order Laplacian of a
    square block.  The first row of every block after the first depends on the row
    just before it, so the blocks form one dependency chain."""
    rng = rng_for(seed)
    props = rng.dirichlet(np.ones(3))
    order = rng.permutation(3)
    sizes = np.maximum(16, np.round(props * n).astype(np.int64))
    counts_all, cols_all = [], []
    start = 0
    for b in order:
        rows = int(sizes[b])
        if b == 2:
            side = max(2, int(np.sqrt(rows)))
            rows = side * side
            g = gen_laplacian(side)
            cnt = np.diff(g.rowptr.astype(np.int64)) - 1
            off = np.ones(g.nnz, dtype=bool)
            off[g.rowptr[1:].astype(np.int64) - 1] = False
            cols = g.colidx[off].astype(np.int64) + start
        else:
            i = np.arange(start, start + rows, dtype=np.int64)
            if b == 0:
                lo = np.full(rows, start, dtype=np.int64)
                k = np.full(rows, 8)
            else:
                lo = np.maximum(0, i - 4)
                k = np.full(rows, 3)
            cnt, cols = _distinct_uniform(rng, lo, i, k)
        cnt = np.asarray(cnt, dtype=np.int64).copy()
        if start > 0 and b != 1 and cnt[0] == 0:
            cnt[0] = 1
            cols = np.concatenate([[start - 1], cols])
        counts_all.append(cnt)
        cols_all.append(np.asarray(cols, dtype=np.int64))
        start += rows
    counts = np.concatenate(counts_all)
    cols = np.concatenate(cols_all)
    m = gen_from_deps(start, counts, cols, rng, name=f"mixture(n={start},seed={seed})")
    m.meta.update(kind="mixture", seed=seed)
    return m


# ----------------------------------------------------------------------------------
# shapes of the paper's matrices (structure only; the matrices themselves are not
# available): level counts, level-width profiles and dependency densities as stated
# in Section IV and Table I
# ----------------------------------------------------------------------------------

def _from_level_widths(widths, deps_per_row: float, seed: int, window: int = 3, name: str = "") -> LowerCsr:
    """Rows in level order.  Every row of level l >= 1 takes one dependency in level l-1
    (so its level is exactly l) and, on average, deps_per_row - 1 more distinct ones
    uniform over the previous `window` levels."""
    rng = rng_for(seed)
    widths = np.asarray(widths, dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(widths)])
    n = int(starts[-1])
    counts = np.zeros(n, dtype=np.int64)
    cols = []
    for l in range(1, widths.size):
        a, b = int(starts[l]), int(starts[l + 1])
        lo = int(starts[max(0, l - window)])
        prev_a, prev_b = int(starts[l - 1]), int(starts[l])
        for r in range(a, b):
            d = {int(rng.integers(prev_a, prev_b))}
            extra = rng.poisson(max(0.0, deps_per_row - 1.0))
            span = prev_b - lo
            for _ in range(int(min(extra, span - 1))):
                d.add(int(rng.integers(lo, prev_b)))
            s = sorted(d)
            counts[r] = len(s)
            cols.extend(s)
    m = gen_from_deps(n, counts, np.asarray(cols, dtype=np.int64), rng, name=name)
    m.meta.update(kind=name, seed=seed)
    return m


def gen_lung2_like(seed: int = 0, scale: float = 1.0) -> LowerCsr:
    """109,460 rows in 479 levels, 453 of them two rows wide (Section IV), the other 26
    levels wide "bumps"; about 1.5 dependencies per row (Table I's total level cost
    437,834 = 2 nnz - n gives nnz = 273,647).  ``scale`` narrows the fat levels (same
    level count) for quick runs."""
    rng = rng_for(seed + 1)
    m_levels, n = 479, max(2 * 479, int(109_460 * scale))
    fat = np.sort(rng.choice(np.arange(1, m_levels), size=26, replace=False))
    widths = np.full(m_levels, 2, dtype=np.int64)
    rest = n - 2 * (m_levels - 26)
    share = rng.dirichlet(np.ones(26)) * rest
    w = np.floor(share).astype(np.int64)
    w[: rest - int(w.sum())] += 1
    widths[fat] = w
    return _from_level_widths(widths, 1.5, seed, window=2, name="lung2_like")


def gen_torso2_like(seed: int = 0, scale: float = 1.0) -> LowerCsr:
    """115,967 rows in 513 levels with a triangular width profile (Section IV); about
    3.96 dependencies per row (Table I: 1,035,484 = 2 nnz - n).  ``scale`` narrows the
    levels (same level count) for quick runs."""
    m_levels, n = 513, max(2 * 513, int(115_967 * scale))
    x = np.arange(m_levels)
    tri = np.minimum(x + 1, m_levels - x).astype(np.float64)
    widths = np.maximum(1, np.floor(tri / tri.sum() * n)).astype(np.int64)
    widths[m_levels // 2] += n - int(widths.sum())
    return _from_level_widths(widths, 3.96, seed, window=3, name="torso2_like")
