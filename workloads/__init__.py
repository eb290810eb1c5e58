"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and bench.py.

This module only draws random structures and values (numpy PCG64, fixed seeds).
It holds none of the contraction arithmetic: no semiring operation, no symbolic
or numeric phase, no shortest-path or centrality step.  Everything it returns is
plain host arrays in the CSR layout used on both sides of the boundary:

    rowptr  int64[nrows + 1]   (monotone, rowptr[0] == 0)
    col     int32[nnz]         (ascending and unique inside each row)
    val     typed array[nnz]   (or None for structure-only matrices)

Recipes (the shapes of the workloads the method is measured on):

* ``er_fixed_degree``   Erdos-Renyi digraph with exactly ``deg`` distinct uniform
                         columns per row (self-loops allowed).
* ``rmat``               R-MAT (Chakrabarti et al.) with quadrant probabilities
                         a/b/c/d, no noise, vertex labels not permuted, self-loops
                         and duplicate edges removed before any value is drawn.
* ``weights_unit01``     uniform (0,1] values as (m+1) * 2^-24, m ~ U[0, 2^24):
                         exactly representable in fp32 and fp64.
* ``weights_int``        uniform integers in [lo, hi].
* ``weights_normal``     N(0,1) rounded to fp32.
* ``powerlaw_batch``     many independent square matrices whose row counts follow
                         a truncated power law, with U{dmin..dmax} distinct
                         columns per row.
* ``banded``             banded matrices with a given half bandwidth and fill.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

TWO_M24 = 2.0 ** -24


@dataclass
class Csr:
    nrows: int
    ncols: int
    rowptr: np.ndarray  # int64[nrows+1]
    col: np.ndarray     # int32[nnz]
    val: Optional[np.ndarray] = None

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def with_val(self, val: np.ndarray) -> "Csr":
        assert val.shape[0] == self.nnz
        return Csr(self.nrows, self.ncols, self.rowptr, self.col, val)

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr)


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def sorted_unique(keys: np.ndarray) -> np.ndarray:
    """Ascending distinct values (sort, then drop repeats)."""
    k = np.sort(keys, kind="stable" if keys.size < 1024 else "quicksort")
    if k.size == 0:
        return k
    keep = np.empty(k.size, dtype=bool)
    keep[0] = True
    np.not_equal(k[1:], k[:-1], out=keep[1:])
    return k[keep]


def csr_from_sorted_keys(keys: np.ndarray, nrows: int, ncols: int) -> Csr:
    """Build a CSR structure from unique int64 keys row*ncols+col, sorted ascending."""
    rows = keys // ncols
    cols = (keys - rows * ncols).astype(np.int32)
    counts = np.bincount(rows, minlength=nrows).astype(np.int64)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return Csr(nrows, ncols, rowptr, cols)


def csr_from_coo(rows: np.ndarray, cols: np.ndarray, nrows: int, ncols: int,
                 drop_self_loops: bool = False) -> Csr:
    """Sort and de-duplicate a coordinate list into a CSR structure."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    if drop_self_loops:
        keep = rows != cols
        rows, cols = rows[keep], cols[keep]
    keys = sorted_unique(rows * ncols + cols)
    return csr_from_sorted_keys(keys, nrows, ncols)


def distinct_columns(rng: np.random.Generator, counts: np.ndarray, ncols: int) -> Csr:
    """Per row i draw counts[i] distinct columns uniformly from [0, ncols).

    Uniform sampling without replacement: candidates are drawn with replacement
    and the first ``counts[i]`` distinct ones (in draw order) are kept; rows that
    come up short are redrawn with more candidates.  Rows asking for more than
    half of the columns take a prefix of a random permutation instead.
    """
    counts = np.asarray(counts, dtype=np.int64)
    nrows = counts.shape[0]
    if np.any(counts > ncols):
        raise ValueError("more distinct columns requested than columns")
    out_keys = [np.zeros(0, np.int64)]
    todo = np.nonzero(counts > 0)[0].astype(np.int64)
    dense = counts[todo] * 2 > ncols
    for r in todo[dense].tolist():
        perm = rng.permutation(ncols)[: counts[r]]
        out_keys.append(r * ncols + perm.astype(np.int64))
    todo = todo[~dense]
    factor = 2
    while todo.size:
        c = counts[todo]
        m = c * factor + 4
        rowid = np.repeat(todo, m)
        cand = rng.integers(0, ncols, size=rowid.size, dtype=np.int64)
        key = rowid * ncols + cand
        _, first = np.unique(key, return_index=True)
        first.sort()                      # draw order; rows stay grouped
        krow = rowid[first]
        rank = np.arange(krow.size, dtype=np.int64) - np.searchsorted(krow, krow, side="left")
        pos = np.searchsorted(todo, krow)
        ok = np.bincount(pos, minlength=todo.size) >= c
        keep = ok[pos] & (rank < c[pos])
        out_keys.append(key[first][keep])
        todo = todo[~ok]
        factor *= 2
    keys = np.sort(np.concatenate(out_keys))
    return csr_from_sorted_keys(keys, nrows, ncols)


# ---------------------------------------------------------------- structures

def er_fixed_degree(n: int, deg: int, seed: int = 0) -> Csr:
    """n x n digraph, exactly ``deg`` distinct uniform random columns per row."""
    rng = _rng(seed)
    return distinct_columns(rng, np.full(n, deg, dtype=np.int64), n)


def random_csr(nrows: int, ncols: int, max_per_row: int, seed: int,
               empty_frac: float = 0.0) -> Csr:
    """Rows with U{0..max_per_row} distinct columns; a fraction forced empty."""
    rng = _rng(seed)
    counts = rng.integers(0, min(max_per_row, ncols) + 1, size=nrows)
    if empty_frac > 0:
        counts[rng.random(nrows) < empty_frac] = 0
    return distinct_columns(rng, counts, ncols)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 0, chunk: int = 1 << 23) -> Csr:
    """R-MAT digraph on 2^scale vertices with edge_factor * 2^scale draws.

    Each edge picks one quadrant per level (a: top-left, b: top-right,
    c: bottom-left, d: bottom-right); the high bit is decided first.  A level's
    choice compares a 16-bit uniform integer with the cumulative probabilities
    scaled to 2^16 (four levels per 64-bit random word).  No noise, no label
    permutation (vertex 0 is the largest hub).  Self-loops and duplicates are
    removed; the result is sorted by (row, col).
    """
    n = 1 << scale
    m = edge_factor * n
    rng = _rng(seed)
    t_ab = np.uint64(round((a + b) * 65536))
    t_a = np.uint64(round(a * 65536))
    t_abc = np.uint64(round((a + b + c) * 65536))
    mask = np.uint64(0xFFFF)
    keys_parts = []
    nwords = (scale + 3) // 4
    for s in range(0, m, chunk):
        cnt = min(chunk, m - s)
        u = np.zeros(cnt, dtype=np.uint64)
        v = np.zeros(cnt, dtype=np.uint64)
        level = 0
        for _ in range(nwords):
            word = rng.integers(0, 2 ** 64 - 1, size=cnt, dtype=np.uint64, endpoint=True)
            for q in range(4):
                if level == scale:
                    break
                r = (word >> np.uint64(16 * q)) & mask
                down = r >= t_ab                        # quadrants c or d: row bit set
                right = ((r >= t_a) & (r < t_ab)) | (r >= t_abc)  # quadrants b or d: col bit
                sh = np.uint64(scale - 1 - level)
                u |= down.astype(np.uint64) << sh
                v |= right.astype(np.uint64) << sh
                level += 1
        keep = u != v
        uu = u[keep].astype(np.int64)
        keys_parts.append(sorted_unique(uu * n + v[keep].astype(np.int64)))
    keys = sorted_unique(np.concatenate(keys_parts))
    return csr_from_sorted_keys(keys, n, n)


def banded(n: int, half_bw: int, fill: float, seed: int) -> Csr:
    """Each (i, j) with |i - j| <= half_bw kept with probability ``fill``."""
    rng = _rng(seed)
    offs = np.arange(-half_bw, half_bw + 1, dtype=np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), offs.size)
    cols = rows + np.tile(offs, n)
    keep = (cols >= 0) & (cols < n) & (rng.random(rows.size) < fill)
    keys = rows[keep] * n + cols[keep]
    return csr_from_sorted_keys(keys, n, n)


def powerlaw_sizes(count: int, lo: int, hi: int, exponent: float, seed: int) -> np.ndarray:
    """Integer sizes r = floor((lo^-e1 + u (hi^-e1 - lo^-e1))^(-1/e1)), e1 = exponent - 1."""
    rng = _rng(seed)
    e1 = exponent - 1.0
    u = rng.random(count)
    x = (lo ** -e1 + u * (hi ** -e1 - lo ** -e1)) ** (-1.0 / e1)
    return np.clip(np.floor(x).astype(np.int64), lo, hi)


def powerlaw_batch(nbatch: int, lo: int, hi: int, exponent: float, dmin: int, dmax: int,
                   seed: int):
    """``nbatch`` independent pairs (A_b, B_b), both r_b x r_b, N(0,1) fp32 values.

    Row counts follow ``powerlaw_sizes``; every row has U{dmin..dmax} distinct
    columns (capped at r_b).  Returns (sizes, [A_b], [B_b]).
    """
    sizes = powerlaw_sizes(nbatch, lo, hi, exponent, seed)
    rng = _rng(seed + 1)
    As, Bs = [], []
    for r in sizes.tolist():
        pair = []
        for _ in range(2):
            counts = np.minimum(rng.integers(dmin, dmax + 1, size=r), r)
            m = distinct_columns(rng, counts, r)
            m.val = rng.standard_normal(m.nnz).astype(np.float32)
            pair.append(m)
        As.append(pair[0])
        Bs.append(pair[1])
    return sizes, As, Bs


# ---------------------------------------------------------------- values

def weights_unit01(nnz: int, seed: int) -> np.ndarray:
    """Uniform (0,1] as (m+1) * 2^-24, returned as float64 (exact in fp32 too)."""
    rng = _rng(seed)
    m = rng.integers(0, 1 << 24, size=nnz, dtype=np.int64)
    return (m + 1).astype(np.float64) * TWO_M24


def weights_int(nnz: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = _rng(seed)
    return rng.integers(lo, hi + 1, size=nnz, dtype=np.int64).astype(np.int32)


def weights_normal(nnz: int, seed: int) -> np.ndarray:
    rng = _rng(seed)
    return rng.standard_normal(nnz).astype(np.float32)


def sample_sources(g: Csr, count: int, seed: int) -> np.ndarray:
    """``count`` distinct vertices with out-degree >= 1, uniform, sorted ascending."""
    rng = _rng(seed)
    cand = np.nonzero(np.diff(g.rowptr) > 0)[0]
    count = min(count, cand.size)
    pick = rng.choice(cand.size, size=count, replace=False)
    return np.sort(cand[pick]).astype(np.int32)


def multpath_values(nnz: int, dmax: int, smax: int, seed: int) -> np.ndarray:
    """Structured (int32 distance, fp64 multiplicity) entries for test operands."""
    rng = _rng(seed)
    out = np.zeros(nnz, dtype=MULTPATH_DTYPE)
    out["d"] = rng.integers(0, dmax + 1, size=nnz).astype(np.int32)
    out["s"] = rng.integers(1, smax + 1, size=nnz).astype(np.float64)
    return out


# (distance, multiplicity) element layout: int32 d, 4 bytes padding, fp64 sigma.
MULTPATH_DTYPE = np.dtype({"names": ["d", "pad", "s"], "formats": [np.int32, np.int32, np.float64],
                           "offsets": [0, 4, 8], "itemsize": 16})
