"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *generates input data* (matrices and start vectors).  It holds
none of the truncated-SVD arithmetic: no products with A, no orthogonalisation,
no small SVD.  Both the CPU oracle (``oracle/``) and the CUDA path read the
arrays produced here, so a parity test feeds both sides identical bytes.

Workload shapes follow the sparse and dense test families of the svds-C paper
(Sec. 3.1: random sparse matrices with a few nonzeros per row, tall sparse
real-world matrices with skewed row lengths, and dense matrices with a
prescribed singular-value decay), scaled to the sizes used here.

All matrices are returned in 0-based, 3-array CSR (``row_ptr`` int64 of length
m+1, ``col_idx`` int32, ``values`` float64 or float32), or as a column-major
(Fortran-ordered) dense float64 array.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# Base seed of the named workloads (an arbitrary fixed number); workload c uses
# BASE_SEED + c.
BASE_SEED = 240518966

# Row-length scaling for the Zipf workload: X ~ Zipf(1.5) truncated to
# [1, 2000], L = clamp(ceil(ZIPF_SCALE * X), 1, 2000).  With this constant the
# expected row length is 20.00 nnz/row (computed from the exact pmf), 38.9 % of
# rows hold one nonzero and the longest possible row holds 1,139.
ZIPF_SCALE = 0.56905


@dataclass
class CSR:
    m: int
    n: int
    row_ptr: np.ndarray  # int64, m+1
    col_idx: np.ndarray  # int32, nnz
    values: np.ndarray   # float64 or float32, nnz
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        """Column-major dense copy (only for small matrices in tests)."""
        a = np.zeros((self.m, self.n), dtype=np.float64, order="F")
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        a[rows, self.col_idx] = self.values
        return a


@dataclass
class Dense:
    m: int
    n: int
    a: np.ndarray  # float64, shape (m, n), Fortran order (column-major, ld = m)
    name: str = ""
    # Optional exact factors for matrices built as Q1 diag(s) Q2^T.
    s: Optional[np.ndarray] = None
    left_reflectors: list = field(default_factory=list)
    right_reflectors: list = field(default_factory=list)


def _fill_rows(rng: np.random.Generator, m: int, n: int, lengths: np.ndarray):
    """Uniform distinct column indices for each row, sorted within the row."""
    lengths = lengths.astype(np.int64)
    if np.any(lengths > n):
        raise ValueError("row length exceeds the number of columns")
    nnz = int(lengths.sum())
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    rows = np.repeat(np.arange(m, dtype=np.int64), lengths)
    cols = rng.integers(0, n, size=nnz, dtype=np.int64)
    key = rows * n + cols
    # Resample the duplicates inside a row until every row's columns are
    # distinct (rows are contiguous in `key`, so sorting keeps them grouped).
    while True:
        key.sort(kind="stable")
        dup = np.nonzero(key[1:] == key[:-1])[0] + 1
        if dup.size == 0:
            break
        key[dup] = rows_of(key[dup], n) * n + rng.integers(0, n, size=dup.size, dtype=np.int64)
    col_idx = (key % n).astype(np.int32)
    return row_ptr, col_idx


def rows_of(key: np.ndarray, n: int) -> np.ndarray:
    return key // n


def csr_uniform(m: int, n: int, density: float, seed: int, dtype=np.float64, name="") -> CSR:
    """Exactly round(density*m*n) positions drawn uniformly without replacement
    over the m x n grid; values N(0,1)."""
    rng = np.random.default_rng(seed)
    nnz = int(round(density * m * n))
    pos = np.sort(rng.choice(m * n, size=nnz, replace=False))
    rows = pos // n
    cols = (pos % n).astype(np.int32)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    vals = rng.standard_normal(nnz)
    if dtype == np.float32:
        vals = vals.astype(np.float32)
    return CSR(m, n, row_ptr, cols, vals, name)


def zipf_row_lengths(rng: np.random.Generator, m: int, alpha: float = 1.5, cap: int = 2000,
                     scale: float = ZIPF_SCALE) -> np.ndarray:
    """Row lengths L = clamp(ceil(scale*X), 1, cap), X ~ Zipf(alpha) truncated to [1, cap]."""
    x = np.arange(1, cap + 1, dtype=np.float64)
    pmf = x ** (-alpha)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    u = rng.random(m)
    xs = np.searchsorted(cdf, u, side="right") + 1
    xs = np.minimum(xs, cap)
    return np.clip(np.ceil(scale * xs), 1, cap).astype(np.int64)


def csr_zipf(m: int, n: int, seed: int, alpha: float = 1.5, cap: int = 2000,
             scale: float = ZIPF_SCALE, dtype=np.float64, name="") -> CSR:
    """Tall sparse matrix with heavy-tailed (Zipf) row lengths, uniform columns,
    values N(0,1)."""
    rng = np.random.default_rng(seed)
    lengths = zipf_row_lengths(rng, m, alpha, min(cap, n), scale)
    row_ptr, col_idx = _fill_rows(rng, m, n, lengths)
    vals = rng.standard_normal(int(row_ptr[-1]))
    if dtype == np.float32:
        vals = vals.astype(np.float32)
    return CSR(m, n, row_ptr, col_idx, vals, name)


def csr_uniform_rows(m: int, n: int, lo: int, hi: int, seed: int, dtype=np.float32, name="") -> CSR:
    """Each row's length uniform in [lo, hi], columns uniform and distinct, values N(0,1)."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(lo, hi + 1, size=m)
    lengths = np.minimum(lengths, n)
    row_ptr, col_idx = _fill_rows(rng, m, n, lengths)
    vals = rng.standard_normal(int(row_ptr[-1]))
    if dtype == np.float32:
        vals = vals.astype(np.float32)
    return CSR(m, n, row_ptr, col_idx, vals, name)


def householder_vectors(rng: np.random.Generator, dim: int, count: int) -> list:
    return [rng.standard_normal(dim) for _ in range(count)]


def dense_prescribed(m: int, n: int, s: np.ndarray, seed: int, nrefl: int = 4, name="") -> Dense:
    """A = H_1...H_q [diag(s); 0] (G_1...G_q)^T with H_j = I - 2 w w^T/(w^T w)
    (w ~ N(0, I_m)) and G_j likewise in R^n.  The singular values of A are |s|
    exactly (up to rounding of the construction), the left singular vector i is
    H_1...H_q e_i and the right one G_1...G_q e_i."""
    assert m >= n and s.shape == (n,)
    rng = np.random.default_rng(seed)
    hs = householder_vectors(rng, m, nrefl)
    gs = householder_vectors(rng, n, nrefl)
    # B = diag(s) (G_1...G_q)^T = diag(s) G_q ... G_1 : apply G_q first from the right.
    b = np.zeros((n, n), dtype=np.float64, order="F")
    b[np.arange(n), np.arange(n)] = s
    for g in reversed(gs):          # right-multiply by G_q, ..., G_1 in turn
        coef = 2.0 / np.dot(g, g)
        bg = b @ g
        b -= coef * np.outer(bg, g)
    a = np.zeros((m, n), dtype=np.float64, order="F")
    a[:n, :] = b
    try:
        from scipy.linalg.blas import dger
    except Exception:  # pragma: no cover - scipy missing
        dger = None
    for h in reversed(hs):          # left-multiply by H_q first, H_1 last
        coef = 2.0 / np.dot(h, h)
        ht_a = h @ a                 # row vector h^T A
        if dger is not None:
            a = dger(-coef, h, ht_a, a=a, overwrite_a=True)
        else:
            a -= coef * np.outer(h, ht_a)
    return Dense(m, n, a, name, s=np.asarray(s, dtype=np.float64).copy(),
                 left_reflectors=hs, right_reflectors=gs)


def apply_reflectors(vecs: list, x: np.ndarray) -> np.ndarray:
    """Q x for Q = H_1 ... H_q given the reflector vectors [w_1..w_q] (x: vector or matrix)."""
    y = np.array(x, dtype=np.float64, copy=True)
    for w in reversed(vecs):
        coef = 2.0 / np.dot(w, w)
        if y.ndim == 1:
            y -= coef * w * np.dot(w, y)
        else:
            y -= coef * np.outer(w, w @ y)
    return y


def start_vector(n: int, seed: int) -> np.ndarray:
    """An explicit N(0,1) start vector (input data, used when a test passes v0)."""
    return np.random.default_rng(seed ^ 0x5EED).standard_normal(n)


# ---------------------------------------------------------------------------
# Named workloads.  Sizes are the ones the solver is benchmarked and tested on;
# `scale` shrinks the large ones proportionally for quick tests.

def workload_sparse_small(seed_offset: int = 1) -> CSR:
    """2,000 x 1,000 CSR, 1 % uniform density (20,000 nnz), N(0,1) values, FP64."""
    return csr_uniform(2000, 1000, 0.01, BASE_SEED + seed_offset, name="sparse-2000x1000-1pct")


def workload_sparse_zipf(scale: float = 1.0) -> CSR:
    """1,000,000 x 500,000 CSR with Zipf(1.5) row lengths (mean 20, cap 2,000), FP64."""
    m = max(1, int(round(1_000_000 * scale)))
    n = max(1, int(round(500_000 * scale)))
    return csr_zipf(m, n, BASE_SEED + 2, name=f"sparse-zipf-{m}x{n}")


def decay_095(n: int) -> np.ndarray:
    return 0.95 ** np.arange(n, dtype=np.float64)


def workload_dense(scale: float = 1.0) -> Dense:
    """50,000 x 5,000 dense, A = Q1 diag(0.95^i) Q2^T with 4+4 Householder reflectors."""
    m = max(2, int(round(50_000 * scale)))
    n = max(2, int(round(5_000 * scale)))
    return dense_prescribed(m, n, decay_095(n), BASE_SEED + 3, name=f"dense-{m}x{n}-0.95^i")


def decay1(n: int) -> np.ndarray:
    """Decay1 of Eq. 16: sigma_i = 10^(-4 (i-1)/19) for i = 1..20, then 1e-4 / (i-20)^0.1."""
    i = np.arange(1, n + 1, dtype=np.float64)
    head = 10.0 ** (-4.0 * (i - 1.0) / 19.0)
    tail = 1e-4 / np.maximum(i - 20.0, 1.0) ** 0.1
    return np.where(i <= 20, head, tail)


def decay2(n: int) -> np.ndarray:
    """Decay2 of Eq. 16: sigma_i = i^-2."""
    return np.arange(1, n + 1, dtype=np.float64) ** -2.0


def decay3(n: int) -> np.ndarray:
    """Decay3 of Eq. 16: sigma_i = i^-3."""
    return np.arange(1, n + 1, dtype=np.float64) ** -3.0


DECAYS = {1: decay1, 2: decay2, 3: decay3}


def workload_dense_decay(which: int, scale: float = 1.0) -> Dense:
    """DenseN of Sec. 5 (N = 1, 2, 3): 10,000 x 10,000 dense FP64 with the DecayN
    spectrum of Eq. 16.  The paper does not say how its singular vectors are
    drawn; here they are products of 4 + 4 random Householder reflectors, so the
    exact singular values (and vectors) are known."""
    n = max(2, int(round(10_000 * scale)))
    return dense_prescribed(n, n, DECAYS[which](n), BASE_SEED + 10 + which,
                            name=f"dense{which}-{n}x{n}-decay{which}")


def repeated_spectrum(n: int) -> np.ndarray:
    """A spectrum with exactly repeated singular values (clusters of sizes 3, 2,
    4, 2 at the top, then a geometric tail), the kind of input on which Sec. 5
    reports other solvers returning wrong values (many multiple singular values)."""
    head = [3.0] * 3 + [2.0] * 2 + [1.5] * 4 + [1.25] * 2
    tail = 1.0 * 0.97 ** np.arange(max(0, n - len(head)), dtype=np.float64)
    return np.concatenate([np.array(head[:n]), tail])[:n]


def workload_sparse_small_fp32() -> CSR:
    """The 2,000 x 1,000 matrix with values rounded to FP32 (exact in both precisions)."""
    a = workload_sparse_small()
    a.values = a.values.astype(np.float32).astype(np.float64)
    a.name = "sparse-2000x1000-1pct-fp32exact"
    return a


@dataclass
class BatchItem:
    a: CSR
    k: int
    p: int


def workload_batch(count: int = 256, seed: int = BASE_SEED + 5, size_scale: float = 1.0,
                   only=None) -> list:
    """`count` CSR matrices: m ~ U{2000..60000}, n ~ U{1000..30000}, row lengths
    ~ U{5..50}, values N(0,1) FP32; k ~ U{5..40}, p = k (sizes multiplied by
    `size_scale` for quick tests).  `only` (indices): build just those items
    of the same batch (the shape and seed draws of the others are still taken,
    so item i is identical either way); returns them in the order given."""
    rng = np.random.default_rng(seed)
    want = None if only is None else set(int(i) for i in only)
    items = {}
    for b in range(count):
        m = int(rng.integers(2000, 60001) * size_scale)
        n = int(rng.integers(1000, 30001) * size_scale)
        k = int(rng.integers(5, 41))
        m = max(m, 2 * k + 2)
        n = max(n, 2 * k + 2)
        mseed = int(rng.integers(0, 2**62))
        if want is not None and b not in want:
            continue
        a = csr_uniform_rows(m, n, 5, 50, mseed, dtype=np.float32, name=f"batch{b}-{m}x{n}")
        items[b] = BatchItem(a, k, k)
    if only is None:
        return [items[b] for b in range(count)]
    return [items[int(i)] for i in only]


def workload_batch_shapes(count: int = 256, seed: int = BASE_SEED + 5, size_scale: float = 1.0) -> list:
    """(m, n, k) of every item of workload_batch, without building the matrices."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(2000, 60001) * size_scale)
        n = int(rng.integers(1000, 30001) * size_scale)
        k = int(rng.integers(5, 41))
        rng.integers(0, 2**62)
        out.append((max(m, 2 * k + 2), max(n, 2 * k + 2), k))
    return out
