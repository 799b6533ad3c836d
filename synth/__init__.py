"""Seeded synthetic inputs for ANLS-NMF, shared by the tests, the benchmark and
the smoke check.

This module draws random numbers and assembles test matrices from them. It holds
none of the factorisation's arithmetic: no Gram matrix, no product with a factor,
no least-squares solve and no objective.

Generator
---------
Every value is a pure function of ``(seed, tensor_id, element index)``, so any
crop of any tensor can be regenerated on the host without materialising the rest.
The bits come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output number ``e`` of a stream
whose state starts at ``s`` is ``mix64(s + (e + 1) * GOLDEN)``, where ``mix64`` is
the stafford-13 finaliser and ``GOLDEN`` the 64-bit golden-ratio increment.
A stream's start state is ``mix64(seed * GOLDEN ^ (tensor_id << 32))``.

Uniforms in [0, 1) take the top 53 bits (``u >> 11`` times 2^-53); uniforms in
(0, 1] add one ulp of 2^-53 first. Normals use the Box-Muller transform (Box and
Muller 1958) on two uniforms drawn from two sibling streams.

Workload recipes (the paper's synthetic sets, Section 6.1.1)
-----------------------------------------------------------
* ``dense_planted``: A = W0 H0 + |N(0, sigma^2)|, W0 (m x k) and H0 (k x n)
  uniform [0, 1), formed in FP64 and stored FP32 row-major. Shape family of DSYN
  (uniform random matrix plus Gaussian noise); the absolute value keeps A >= 0.
* ``csr_uniform``: nnz positions uniform over the m x n grid (Erdos-Renyi style,
  as SSYN), values uniform (0, 1]; duplicate positions keep the entry drawn
  first. CSR with int64 row pointers and int32 column indices, columns sorted.
* ``init_factors``: the non-negative starting point of Algorithm 1, uniform
  [0, 1) for both W (m x k) and H (stored as H^T, n x k). The same seed gives the
  same start on every path (Section 6.1.3).
* ``stress_factor``: the factor of the batched-BPP stress recipe, uniform
  [0, 1) with each entry zeroed with probability ``zero_frac`` (its own
  stream), and ``normal_matrix`` for the right-hand-side draws of that recipe.
* ``mlp_init``: starting weights of the passive-set proposal network (3k -> h
  -> h -> k), one flat FP32 array [W1 (h x 3k), b1, W2 (h x h), b2, W3 (k x h),
  b3]; each weight matrix uniform in +-sqrt(6 / (fan_in + fan_out)) (Glorot and
  Bengio 2010), biases zero.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Fixed tensor ids: one independent stream per tensor of a recipe.
TID_W0 = 1
TID_H0 = 2
TID_NOISE_U1 = 3
TID_NOISE_U2 = 4
TID_W_INIT = 5
TID_H_INIT = 6
TID_CSR_ROW = 7
TID_CSR_COL = 8
TID_CSR_VAL = 9
TID_NLS_C = 10
TID_NLS_B = 11
TID_STRESS_W = 12
TID_STRESS_ZERO = 13
TID_STRESS_A = 14
TID_MLP_INIT = 15
TID_MLP_BATCH = 16

DEFAULT_SEED = 1509


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_state(seed: int, tensor_id: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.uint64(seed) * GOLDEN ^ (np.uint64(tensor_id) << np.uint64(32))
    return _mix64(np.array([s], dtype=np.uint64))[0]


def bits(seed: int, tensor_id: int, idx: np.ndarray) -> np.ndarray:
    """Raw 64-bit outputs number ``idx`` (any integer array) of one stream."""
    s = stream_state(seed, tensor_id)
    e = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(s + (e + np.uint64(1)) * GOLDEN)


def uniform01(seed: int, tensor_id: int, idx: np.ndarray) -> np.ndarray:
    """Uniform [0, 1) in float64 for element indices ``idx``."""
    return (bits(seed, tensor_id, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_open0(seed: int, tensor_id: int, idx: np.ndarray) -> np.ndarray:
    """Uniform (0, 1] in float64."""
    return ((bits(seed, tensor_id, idx) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normal(seed: int, tensor_pair: tuple[int, int], idx: np.ndarray) -> np.ndarray:
    """Standard normals by Box-Muller from two sibling uniform streams."""
    u1 = uniform_open0(seed, tensor_pair[0], idx)
    u2 = uniform01(seed, tensor_pair[1], idx)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _grid_idx(rows: np.ndarray, cols: np.ndarray, ncols_full: int) -> np.ndarray:
    return rows.astype(np.uint64)[:, None] * np.uint64(ncols_full) + cols.astype(np.uint64)[None, :]


def uniform_matrix(seed: int, tensor_id: int, rows: int, cols: int,
                   row0: int = 0, col0: int = 0, ncols_full: int | None = None) -> np.ndarray:
    """Block [row0:row0+rows, col0:col0+cols] of a uniform [0,1) matrix whose
    full width is ``ncols_full`` (default: ``col0 + cols``)."""
    ncols_full = col0 + cols if ncols_full is None else ncols_full
    idx = _grid_idx(np.arange(row0, row0 + rows), np.arange(col0, col0 + cols), ncols_full)
    return uniform01(seed, tensor_id, idx)


def dense_planted(m: int, n: int, k: int, sigma: float, seed: int = DEFAULT_SEED,
                  row0: int = 0, col0: int = 0, m_full: int | None = None,
                  n_full: int | None = None, return_factors: bool = False):
    """A = W0 H0 + |sigma * N(0,1)| as float32, m x n row-major (a crop of the
    m_full x n_full matrix when row0/col0/m_full/n_full are given)."""
    n_full = col0 + n if n_full is None else n_full
    W0 = uniform_matrix(seed, TID_W0, m, k, row0, 0, k)
    H0 = uniform_matrix(seed, TID_H0, k, n, 0, col0, n_full)
    A = W0 @ H0
    if sigma:
        idx = _grid_idx(np.arange(row0, row0 + m), np.arange(col0, col0 + n), n_full)
        A += np.abs(sigma * normal(seed, (TID_NOISE_U1, TID_NOISE_U2), idx))
    A32 = np.ascontiguousarray(A.astype(np.float32))
    if return_factors:
        return A32, W0, H0
    return A32


def init_factors(m: int, n: int, k: int, seed: int = DEFAULT_SEED):
    """Starting point of Algorithm 1: W (m x k) and H^T (n x k), uniform [0,1),
    float32 (the precision both paths start from)."""
    W = uniform_matrix(seed, TID_W_INIT, m, k).astype(np.float32)
    Ht = uniform_matrix(seed, TID_H_INIT, n, k).astype(np.float32)
    return np.ascontiguousarray(W), np.ascontiguousarray(Ht)


def csr_uniform(m: int, n: int, nnz_draws: int, seed: int = DEFAULT_SEED):
    """CSR matrix with ``nnz_draws`` uniformly placed draws (duplicates merged by
    keeping the first draw), values uniform (0, 1].

    Returns (rowptr int64[m+1], colidx int32[nnz], vals float32[nnz])."""
    e = np.arange(nnz_draws, dtype=np.uint64)
    rows = (bits(seed, TID_CSR_ROW, e) % np.uint64(m)).astype(np.int64)
    cols = (bits(seed, TID_CSR_COL, e) % np.uint64(n)).astype(np.int64)
    vals = uniform_open0(seed, TID_CSR_VAL, e).astype(np.float32)
    key = rows * np.int64(n) + cols
    ukey, first = np.unique(key, return_index=True)   # sorted by (row, col)
    r = ukey // n
    c = (ukey % n).astype(np.int32)
    v = vals[first]
    rowptr = np.zeros(m + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(np.bincount(r, minlength=m))
    return rowptr, np.ascontiguousarray(c), np.ascontiguousarray(v)


def csr_to_dense(rowptr, colidx, vals, m, n) -> np.ndarray:
    D = np.zeros((m, n), dtype=np.float32)
    for i in range(m):
        s, e = rowptr[i], rowptr[i + 1]
        D[i, colidx[s:e]] = vals[s:e]
    return D


def nls_batch(k: int, nrhs: int, rows_c: int | None = None, seed: int = DEFAULT_SEED,
              cond_boost: float = 0.0, signed_rhs: bool = True):
    """A batch of NLS problems in normal-equations form, sharing one matrix.

    C is rows_c x k uniform [0,1) (plus ``cond_boost`` times a common column
    added to every column, which raises cond(C^T C)); the Gram is returned as
    Gram = C^T C computed here in FP64 only to *define* the test input. Each RHS
    b_j is C^T d_j with d_j uniform [-0.5, 1) (``signed_rhs``) or [0,1), so the
    solutions have mixed active sets. Returns (G float64 k x k, B float64
    nrhs x k)."""
    rows_c = 4 * k if rows_c is None else rows_c
    C = uniform_matrix(seed, TID_NLS_C, rows_c, k)
    if cond_boost:
        C = C + cond_boost * C[:, :1]
    D = uniform_matrix(seed, TID_NLS_B, nrhs, rows_c)
    if signed_rhs:
        D = 1.5 * D - 0.5
    G = C.T @ C
    B = D @ C
    return np.ascontiguousarray(G), np.ascontiguousarray(B)


def mlp_param_sizes(k: int, hidden: int) -> list[tuple[int, int]]:
    """(rows, cols) of the proposal network's tensors in flat order; biases have
    cols = 1."""
    return [(hidden, 3 * k), (hidden, 1), (hidden, hidden), (hidden, 1), (k, hidden), (k, 1)]


def mlp_init(k: int, hidden: int = 256, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Flat FP32 starting weights of the proposal network (see the module notes)."""
    parts = []
    off = 0
    for rows, cols in mlp_param_sizes(k, hidden):
        n = rows * cols
        if cols == 1:
            parts.append(np.zeros(n, dtype=np.float64))
        else:
            a = np.sqrt(6.0 / (rows + cols))
            u = uniform01(seed, TID_MLP_INIT, np.arange(off, off + n, dtype=np.uint64))
            parts.append((2.0 * u - 1.0) * a)
        off += n
    return np.concatenate(parts).astype(np.float32)


def batch_order(n: int, epoch: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """A seeded permutation of range(n) for one training epoch (sort of uniform keys)."""
    u = uniform01(seed + epoch, TID_MLP_BATCH, np.arange(n, dtype=np.uint64))
    return np.argsort(u, kind="stable").astype(np.int64)


def stress_factor(rows: int, k: int, zero_frac: float = 0.3, seed: int = DEFAULT_SEED) -> np.ndarray:
    """rows x k float32: uniform [0, 1), each entry zeroed with probability zero_frac."""
    W = uniform_matrix(seed, TID_STRESS_W, rows, k)
    Z = uniform_matrix(seed, TID_STRESS_ZERO, rows, k)
    return np.where(Z < zero_frac, 0.0, W).astype(np.float32)


def normal_matrix(seed: int, tensor_pair: tuple[int, int], rows: int, cols: int,
                  row0: int = 0) -> np.ndarray:
    """rows x cols standard normals (Box-Muller on the pair of streams), rows
    row0.. of a matrix with `cols` columns."""
    r = np.arange(row0, row0 + rows, dtype=np.uint64)[:, None]
    c = np.arange(cols, dtype=np.uint64)[None, :]
    return normal(seed, tensor_pair, r * np.uint64(cols) + c)
