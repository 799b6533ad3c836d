"""Python binding of the sm_103a ANLS-NMF library (``libnmf_gb300.so``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/nmf_gb300.h``; PyTorch supplies
device memory and streams. The functions carry the C names. Importing this
module loads the library and raises ImportError if it has not been built
(``python -c "import __graft_entry__ as g; g.build()"``); there is no CPU path.

Method: ANLS-NMF with block principal pivoting (Kannan, Ballard, Park,
arXiv 1509.09313): minimise ||A - W H||_F^2 over W, H >= 0 (Eq. 1) by
alternating exact NLS updates of W and H (Eq. 2, Alg. 1), each row solved by
BPP (Sec. 4.2). H is passed and stored as H^T (n x k).
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnmf_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")

_lib = ctypes.CDLL(LIB_PATH)

NMF_OK = 0
NMF_ERR_INVALID_ARG = 1
NMF_ERR_CUDA = 2
NMF_ERR_OOM = 3
NMF_ERR_NOT_CONVERGED = 4
NMF_ERR_SINGULAR_GRAM = 5
NMF_ERR_NONFINITE = 6

NMF_PREC_FP32 = 0
NMF_PREC_BF16X3 = 1
NMF_INPUT_DENSE = 0
NMF_INPUT_CSR = 1
NMF_START_COLD = 0
NMF_START_WARM = 1
NMF_MAX_K = 128
NMF_PROPOSAL_OFF = 0
NMF_PROPOSAL_TRAIN = 1
NMF_PROPOSAL_USE = 2
NMF_SOLVER_BPP = 0
NMF_SOLVER_MU = 1
NMF_SOLVER_HALS = 2

SOLVERS = {"bpp": NMF_SOLVER_BPP, "mu": NMF_SOLVER_MU, "hals": NMF_SOLVER_HALS}

PRECISIONS = {"fp32": NMF_PREC_FP32, "bf16x3": NMF_PREC_BF16X3}


class NMFError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {nmf_status_str(status)}")


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32


class nmf_nls_desc(ctypes.Structure):
    _fields_ = [("k", _I32), ("nrhs", _I64), ("G", _P), ("B", _P), ("X", _P),
                ("passive_in", _P), ("passive_out", _P), ("rounds_out", _P),
                ("status_out", _P), ("max_rounds", _I32)]


class nmf_config(ctypes.Structure):
    _fields_ = [("m", _I64), ("n", _I64), ("k", _I32), ("input_kind", _I32),
                ("precision", _I32), ("start_mode", _I32), ("max_bpp_rounds", _I32),
                ("objective_every", _I32), ("solver", _I32), ("no_split_copies", _I32),
                ("no_fused_products", _I32)]


class nmf_matrix(ctypes.Structure):
    _fields_ = [("dense", _P), ("lda", _I64), ("rowptr", _P), ("colidx", _P), ("vals", _P),
                ("nnz", _I64)]


class nmf_stats(ctypes.Structure):
    _fields_ = [("iterations", _I64), ("bpp_rhs", _I64), ("bpp_rounds", _I64),
                ("bpp_max_rounds", _I64), ("bpp_fp64_solves", _I64), ("bpp_fp64_halfsteps", _I64),
                ("bpp_not_converged", _I64), ("bpp_singular", _I64),
                ("ms_gram", ctypes.c_double), ("ms_mm", ctypes.c_double),
                ("ms_nls", ctypes.c_double), ("ms_objective", ctypes.c_double),
                ("kernel_launches", _I64), ("ms_proposal", ctypes.c_double),
                ("graph_launches", _I64), ("mm_splits_max", _I64)]


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_lib.nmf_status_str.argtypes = [ctypes.c_int]
_lib.nmf_status_str.restype = ctypes.c_char_p
_c_gram = _sig("nmf_gram", [_P, _I64, _I32, _P, _P])
_c_update_mu = _sig("nmf_update_mu", [_I32, _I64, _P, _P, _P, _P])
_c_update_hals = _sig("nmf_update_hals", [_I32, _I64, _P, _P, _P, _P])
_c_pgrad_sq = _sig("nmf_pgrad_sq", [_I32, _I64, _P, _P, _P, ctypes.POINTER(ctypes.c_double), _P])
_c_set_pgrad = _sig("nmf_set_pgrad", [_P, _I32])
_c_pgrad_history = _sig("nmf_pgrad_history", [_P, _P, _I64, ctypes.POINTER(_I64)])
_c_iterate_until = _sig("nmf_iterate_until", [_P, _I32, ctypes.c_double, ctypes.POINTER(_I32),
                                              ctypes.POINTER(ctypes.c_double)])
_c_mm_dense = _sig("nmf_mm_dense", [_P, _I64, _I64, _I64, _P, _I32, _I32, _I32, _P, _P])
_c_mm_csr = _sig("nmf_mm_csr", [_P, _P, _P, _I64, _I64, _P, _I32, _P, _P])
_c_csr_transpose = _sig("nmf_csr_transpose", [_P, _P, _P, _I64, _I64, _I64, _P, _P, _P, _P])
_c_nls_bpp = _sig("nmf_nls_bpp", [ctypes.POINTER(nmf_nls_desc), _P])
_c_nls_bpp_noalloc = _sig("nmf_nls_bpp_noalloc", [ctypes.POINTER(nmf_nls_desc), _P])
_c_nls_bpp_tune = _sig("nmf_nls_bpp_tune", [ctypes.POINTER(nmf_nls_desc), _P,
                                            ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                            ctypes.POINTER(_I32)])
_c_nls_bpp_set_shape = _sig("nmf_nls_bpp_set_shape", [_I32, _I32, _I32, _I32])
_c_kernel_launches = _sig("nmf_kernel_launches", [], _I64)
_c_probe_fp32_fma = _sig("nmf_probe_fp32_fma", [_I32, _I32, ctypes.POINTER(ctypes.c_double), _P])
_c_nls_bpp_get_shape = _sig("nmf_nls_bpp_get_shape", [_I32, ctypes.POINTER(_I32),
                                                      ctypes.POINTER(_I32), ctypes.POINTER(_I32)])
_c_objective_dense = _sig("nmf_objective_dense",
                          [_P, _I64, _I64, _I64, _P, _P, _I32, _I32,
                           ctypes.POINTER(ctypes.c_double), _P])
_c_init = _sig("nmf_init", [ctypes.POINTER(_P), ctypes.POINTER(nmf_config),
                            ctypes.POINTER(nmf_matrix), _P, _P, _P])
_c_iterate = _sig("nmf_iterate", [_P, _I32])
_c_sync = _sig("nmf_sync", [_P])
_c_objective = _sig("nmf_objective", [_P, ctypes.POINTER(ctypes.c_double)])
_c_history = _sig("nmf_objective_history", [_P, _P, _I64, ctypes.POINTER(_I64)])
_c_get_factors = _sig("nmf_get_factors", [_P, _P, _P])
_c_set_factors = _sig("nmf_set_factors", [_P, _P, _P])
_c_get_passive = _sig("nmf_get_passive", [_P, _P, _P])
_c_get_stats = _sig("nmf_get_stats", [_P, ctypes.POINTER(nmf_stats)])
_c_set_timing = _sig("nmf_set_timing", [_P, _I32])
_c_set_graph = _sig("nmf_set_graph", [_P, _I32])
_lib.nmf_destroy.argtypes = [_P]
_lib.nmf_destroy.restype = None
_c_mlp_param_count = _sig("nmf_mlp_param_count", [_I32, _I32], _I64)
_c_mlp_create = _sig("nmf_mlp_create", [ctypes.POINTER(_P), _I32, _I32, _P, _P])
_c_mlp_get_params = _sig("nmf_mlp_get_params", [_P, _P, _P])
_lib.nmf_mlp_destroy.argtypes = [_P]
_lib.nmf_mlp_destroy.restype = None
_c_mlp_features = _sig("nmf_mlp_features", [_P, _P, _P, _I64, _I32, _P, _P])
_c_mlp_forward = _sig("nmf_mlp_forward", [_P, _P, _I64, _P, _P])
_c_mlp_propose = _sig("nmf_mlp_propose", [_P, _P, _I64, _P, _P])
_c_mlp_gradient = _sig("nmf_mlp_gradient", [_P, _P, _P, _I64, _P, _P, _P])
_c_mlp_train = _sig("nmf_mlp_train", [_P, _P, _P, _I64, _I64, ctypes.c_float, _P, _P])
_c_set_proposal = _sig("nmf_set_proposal", [_P, _P, _I32, _I32, _I64, ctypes.c_float])

EXPORTED = ["nmf_status_str", "nmf_kernel_launches", "nmf_probe_fp32_fma", "nmf_gram", "nmf_mm_dense", "nmf_mm_csr",
            "nmf_csr_transpose", "nmf_nls_bpp", "nmf_nls_bpp_noalloc", "nmf_nls_bpp_tune", "nmf_nls_bpp_set_shape",
            "nmf_nls_bpp_get_shape", "nmf_objective_dense", "nmf_init", "nmf_iterate", "nmf_sync",
            "nmf_objective", "nmf_objective_history", "nmf_get_factors", "nmf_set_factors",
            "nmf_get_passive", "nmf_get_stats", "nmf_set_timing", "nmf_set_graph", "nmf_destroy",
            "nmf_mlp_param_count", "nmf_mlp_create", "nmf_mlp_get_params", "nmf_mlp_destroy",
            "nmf_mlp_features", "nmf_mlp_forward", "nmf_mlp_propose", "nmf_mlp_gradient",
            "nmf_mlp_train", "nmf_set_proposal", "nmf_update_mu", "nmf_update_hals",
            "nmf_pgrad_sq", "nmf_set_pgrad", "nmf_pgrad_history", "nmf_iterate_until"]


def nmf_status_str(status: int) -> str:
    return _lib.nmf_status_str(int(status)).decode()


def nmf_kernel_launches() -> int:
    """CUDA kernels this process has launched through the library so far."""
    return int(_c_kernel_launches())


def nmf_probe_fp32_fma(packed: bool = True, launches: int = 200, stream=None) -> float:
    """Measured FP32 FMA throughput of the current GPU in flop/s (scalar FFMA
    or packed FFMA2 chains on every SM; synchronises the stream)."""
    out = ctypes.c_double(0.0)
    _check(_c_probe_fp32_fma(int(bool(packed)), int(launches), ctypes.byref(out),
                             _stream(stream)), "nmf_probe_fp32_fma")
    return out.value


def _check(status: int, what: str):
    if status != NMF_OK:
        raise NMFError(status, what)


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None):
    return None if t is None else t.data_ptr()


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _shape(t: torch.Tensor, shape: tuple, name: str) -> torch.Tensor:
    """Exact shape check before any pointer reaches the library (a wrongly
    sized buffer would otherwise be read or written out of bounds)."""
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def _out(out, rows: int, k: int, ref: torch.Tensor, name: str = "out") -> torch.Tensor:
    """A caller's output buffer: contiguous float32 (rows x k) on ref's device;
    allocated when None."""
    if out is None:
        return torch.empty((rows, k), dtype=torch.float32, device=ref.device)
    _dev(out, torch.float32, name)
    if out.device != ref.device:
        raise ValueError(f"{name} must be on {ref.device}")
    return _shape(out, (rows, k), name)


def _matrix(t: torch.Tensor, name: str) -> torch.Tensor:
    if t.dim() != 2:
        raise ValueError(f"{name} must be a 2-D matrix")
    return t


def _prec(precision) -> int:
    return PRECISIONS[precision] if isinstance(precision, str) else int(precision)


def nmf_gram(X: torch.Tensor, stream=None) -> torch.Tensor:
    """G = X^T X (k x k, float64) for X (rows x k, float32)."""
    _matrix(_dev(X, torch.float32, "X"), "X")
    rows, k = X.shape
    G = torch.empty((k, k), dtype=torch.float64, device=X.device)
    _check(_c_gram(_ptr(X), rows, k, _ptr(G), _stream(stream)), "nmf_gram")
    return G


def _local_update(fn, name, G, R, X, stream):
    _dev(G, torch.float64, "G")
    _dev(R, torch.float32, "R")
    _matrix(_dev(X, torch.float32, "X"), "X")
    rows, k = X.shape
    if tuple(G.shape) != (k, k) or tuple(R.shape) != (rows, k):
        raise ValueError("G must be k x k and R rows x k")
    _check(fn(k, rows, _ptr(G), _ptr(R), _ptr(X), _stream(stream)), name)
    return X


def nmf_update_mu(G: torch.Tensor, R: torch.Tensor, X: torch.Tensor, stream=None) -> torch.Tensor:
    """One MU step (Eq. 5) of the rows of X (rows x k float32, updated in place)
    with Gram G (k x k float64) and right-hand sides R (rows x k float32)."""
    return _local_update(_c_update_mu, "nmf_update_mu", G, R, X, stream)


def nmf_update_hals(G: torch.Tensor, R: torch.Tensor, X: torch.Tensor,
                    stream=None) -> torch.Tensor:
    """One HALS sweep (Eq. 6) of the rows of X in place; arguments as nmf_update_mu."""
    return _local_update(_c_update_hals, "nmf_update_hals", G, R, X, stream)


def nmf_pgrad_sq(G: torch.Tensor, R: torch.Tensor, X: torch.Tensor, stream=None) -> float:
    """|P[X G - R]|_F^2: the squared projected-gradient norm of the rows of X
    (entries with x = 0 count only where the gradient is negative)."""
    _dev(G, torch.float64, "G")
    _dev(R, torch.float32, "R")
    _matrix(_dev(X, torch.float32, "X"), "X")
    rows, k = X.shape
    if tuple(G.shape) != (k, k) or tuple(R.shape) != (rows, k):
        raise ValueError("G must be k x k and R rows x k")
    out = ctypes.c_double(0.0)
    _check(_c_pgrad_sq(k, rows, _ptr(G), _ptr(R), _ptr(X), ctypes.byref(out), _stream(stream)),
           "nmf_pgrad_sq")
    return out.value


def nmf_mm_dense(A: torch.Tensor, F: torch.Tensor, trans: bool, precision="fp32",
                 out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """trans=False: A @ F with F = H^T (n x k) -> m x k.  trans=True: A^T @ F with
    F = W (m x k) -> n x k. A may have a row stride > n (2-D view)."""
    if A.dtype != torch.float32 or not A.is_cuda or A.dim() != 2 or A.stride(1) != 1:
        raise TypeError("A must be a row-major float32 CUDA matrix")
    _matrix(_dev(F, torch.float32, "F"), "F")
    m, n = A.shape
    k = F.shape[1]
    rows = n if trans else m
    _shape(F, (m if trans else n, k), "F")
    if F.device != A.device:
        raise ValueError("A and F must be on the same device")
    out = _out(out, rows, k, A)
    _check(_c_mm_dense(_ptr(A), m, n, A.stride(0), _ptr(F), k, int(trans), _prec(precision),
                       _ptr(out), _stream(stream)), "nmf_mm_dense")
    return out


def nmf_mm_csr(rowptr, colidx, vals, cols: int, F: torch.Tensor, out=None,
               stream=None) -> torch.Tensor:
    """out (rows x k) = S F for S in CSR (int64 rowptr, int32 colidx, float32 vals)."""
    _dev(rowptr, torch.int64, "rowptr")
    _dev(colidx, torch.int32, "colidx")
    _dev(vals, torch.float32, "vals")
    _matrix(_dev(F, torch.float32, "F"), "F")
    rows = rowptr.numel() - 1
    k = F.shape[1]
    _shape(F, (cols, k), "F")
    if colidx.numel() != vals.numel():
        raise ValueError("colidx and vals must have the same length")
    out = _out(out, rows, k, F)
    _check(_c_mm_csr(_ptr(rowptr), _ptr(colidx), _ptr(vals), rows, cols, _ptr(F), k, _ptr(out),
                     _stream(stream)), "nmf_mm_csr")
    return out


def nmf_csr_transpose(rowptr, colidx, vals, m: int, n: int, stream=None):
    _dev(rowptr, torch.int64, "rowptr")
    _dev(colidx, torch.int32, "colidx")
    _dev(vals, torch.float32, "vals")
    nnz = colidx.numel()
    if rowptr.numel() != m + 1 or vals.numel() != nnz:
        raise ValueError("rowptr must have m + 1 entries and vals as many as colidx")
    dev = rowptr.device
    t_rowptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    t_colidx = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)[:nnz]
    t_vals = torch.empty(max(nnz, 1), dtype=torch.float32, device=dev)[:nnz]
    _check(_c_csr_transpose(_ptr(rowptr), _ptr(colidx), _ptr(vals), m, n, nnz, _ptr(t_rowptr),
                            _ptr(t_colidx), _ptr(t_vals), _stream(stream)), "nmf_csr_transpose")
    return t_rowptr, t_colidx, t_vals


def nmf_nls_bpp(G: torch.Tensor, B: torch.Tensor, passive_in: torch.Tensor | None = None,
                max_rounds: int = 100, outputs: bool = True, stream=None):
    """Batched BPP: each row b of B gives argmin_{x>=0} 0.5 x^T G x - b^T x.

    G: k x k float64 (CUDA); B: nrhs x k float32. passive_in: nrhs x ceil(k/64)
    int64 bitmasks (warm start) or None (cold). Returns dict(X, passive, rounds,
    status (per RHS), worst (aggregate status))."""
    return _nls_bpp(_c_nls_bpp, "nmf_nls_bpp", G, B, passive_in, max_rounds, outputs, stream)


def nmf_nls_bpp_noalloc(G: torch.Tensor, B: torch.Tensor, passive_in: torch.Tensor | None = None,
                        max_rounds: int = 100, outputs: bool = True, stream=None):
    """Same as nmf_nls_bpp, through the allocation-free entry point: the
    library allocates no device memory for the call (its workspace is a fixed
    array inside the library). The output tensors are allocated here, by the
    caller's side, as for nmf_nls_bpp."""
    return _nls_bpp(_c_nls_bpp_noalloc, "nmf_nls_bpp_noalloc", G, B, passive_in, max_rounds,
                    outputs, stream)


def nmf_nls_bpp_tune(G: torch.Tensor, B: torch.Tensor, passive_in: torch.Tensor | None = None,
                     max_rounds: int = 100, stream=None):
    """Autotune the solve kernels' launch shape for k on this batch (kept for
    every later solve of that k). Returns (warps per CTA, RHS per grab,
    group-tile pass on, X)."""
    _dev(G, torch.float64, "G")
    _matrix(_dev(B, torch.float32, "B"), "B")
    nrhs, k = B.shape
    _shape(G, (k, k), "G")
    X = torch.empty_like(B)
    if passive_in is not None:
        _dev(passive_in, torch.int64, "passive_in")
        _shape(passive_in, (nrhs, (k + 63) // 64), "passive_in")
    d = nmf_nls_desc(k, nrhs, _ptr(G), _ptr(B), _ptr(X), _ptr(passive_in), None, None, None,
                     max_rounds)
    w, c, g = _I32(0), _I32(0), _I32(0)
    _check(_c_nls_bpp_tune(ctypes.byref(d), _stream(stream), ctypes.byref(w), ctypes.byref(c),
                           ctypes.byref(g)), "nmf_nls_bpp_tune")
    return w.value, c.value, g.value, X


def nmf_nls_bpp_set_shape(k: int, warps: int, chunk: int, group: int) -> None:
    """Launch shape of every later solve of this k (results do not depend on it)."""
    _check(_c_nls_bpp_set_shape(k, warps, chunk, group), "nmf_nls_bpp_set_shape")


def nmf_nls_bpp_get_shape(k: int) -> tuple[int, int, int]:
    """(warps per CTA, right-hand sides per grab, group-tile pass on) for k."""
    w, c, g = _I32(0), _I32(0), _I32(0)
    _check(_c_nls_bpp_get_shape(k, ctypes.byref(w), ctypes.byref(c), ctypes.byref(g)),
           "nmf_nls_bpp_get_shape")
    return w.value, c.value, g.value


def _nls_bpp(fn, name, G, B, passive_in, max_rounds, outputs, stream):
    _dev(G, torch.float64, "G")
    _matrix(_dev(B, torch.float32, "B"), "B")
    nrhs, k = B.shape
    nwords = (k + 63) // 64
    _shape(G, (k, k), "G")
    if passive_in is not None:
        _shape(passive_in, (nrhs, nwords), "passive_in")
    dev = B.device
    X = torch.empty_like(B)
    passive = rounds = status = None
    if outputs:
        passive = torch.empty((nrhs, nwords), dtype=torch.int64, device=dev)
        rounds = torch.empty(nrhs, dtype=torch.int32, device=dev)
        status = torch.empty(nrhs, dtype=torch.int8, device=dev)
    if passive_in is not None:
        _dev(passive_in, torch.int64, "passive_in")
    d = nmf_nls_desc(k, nrhs, _ptr(G), _ptr(B), _ptr(X), _ptr(passive_in), _ptr(passive),
                     _ptr(rounds), _ptr(status), max_rounds)
    worst = fn(ctypes.byref(d), _stream(stream))
    if worst in (NMF_ERR_INVALID_ARG, NMF_ERR_CUDA, NMF_ERR_OOM):
        raise NMFError(worst, name)
    return dict(X=X, passive=passive, rounds=rounds, status=status, worst=worst)


def nmf_objective_dense(A: torch.Tensor, W: torch.Tensor, Ht: torch.Tensor, precision="fp32",
                        stream=None) -> float:
    if A.dtype != torch.float32 or not A.is_cuda or A.dim() != 2 or A.stride(1) != 1:
        raise TypeError("A must be a row-major float32 CUDA matrix")
    _matrix(_dev(W, torch.float32, "W"), "W")
    _dev(Ht, torch.float32, "Ht")
    f = ctypes.c_double(0.0)
    m, n = A.shape
    _shape(W, (m, W.shape[1]), "W")
    _shape(Ht, (n, W.shape[1]), "Ht")
    _check(_c_objective_dense(_ptr(A), m, n, A.stride(0), _ptr(W), _ptr(Ht), W.shape[1],
                              _prec(precision), ctypes.byref(f), _stream(stream)),
           "nmf_objective_dense")
    return f.value


class nmf_init:
    """An ANLS handle (``nmf_init`` ... ``nmf_destroy``).

    A: dense float32 CUDA matrix (m x n, row stride >= n) or a CSR tuple
    (rowptr int64, colidx int32, vals float32) with ``shape=(m, n)``. The input
    tensors are borrowed and kept referenced by the handle. W0 (m x k) and
    Ht0 (n x k) float32 CUDA: starting point (copied)."""

    def __init__(self, A, W0: torch.Tensor, Ht0: torch.Tensor, precision="fp32",
                 start="cold", max_bpp_rounds: int = 100, objective_every: bool = True,
                 shape=None, stream=None, solver="bpp", split_copies: bool = True,
                 fused_products: bool = True):
        _matrix(_dev(W0, torch.float32, "W0"), "W0")
        _matrix(_dev(Ht0, torch.float32, "Ht0"), "Ht0")
        m, k = W0.shape
        n = Ht0.shape[0]
        _shape(Ht0, (n, k), "Ht0")
        mat = nmf_matrix()
        if isinstance(A, torch.Tensor):
            if A.dtype != torch.float32 or not A.is_cuda or A.stride(1) != 1:
                raise TypeError("A must be a row-major float32 CUDA matrix")
            if tuple(A.shape) != (m, n):
                raise ValueError("A shape does not match W0 / Ht0")
            mat.dense = A.data_ptr()
            mat.lda = A.stride(0)
            kind = NMF_INPUT_DENSE
        else:
            rowptr, colidx, vals = A
            _dev(rowptr, torch.int64, "rowptr")
            _dev(colidx, torch.int32, "colidx")
            _dev(vals, torch.float32, "vals")
            if shape is None or tuple(shape) != (m, n) or rowptr.numel() != m + 1:
                raise ValueError("CSR input needs shape=(m, n) matching W0 / Ht0")
            mat.rowptr, mat.colidx, mat.vals = _ptr(rowptr), _ptr(colidx), _ptr(vals)
            mat.nnz = colidx.numel()
            kind = NMF_INPUT_CSR
        self._A = A   # keep the borrowed input alive
        self.shape = (m, n, k)
        self.device = W0.device
        cfg = nmf_config(m, n, k, kind, _prec(precision),
                         NMF_START_WARM if start == "warm" else NMF_START_COLD,
                         max_bpp_rounds, int(bool(objective_every)), SOLVERS[solver],
                         int(not split_copies), int(not fused_products))
        self._stream_obj = stream if stream is not None else torch.cuda.current_stream()
        h = _P()
        _check(_c_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.byref(mat), _ptr(W0), _ptr(Ht0),
                       _stream(self._stream_obj)), "nmf_init")
        self._h = h

    def nmf_iterate(self, iters: int = 1):
        _check(_c_iterate(self._h, iters), "nmf_iterate")

    def nmf_sync(self) -> int:
        s = _c_sync(self._h)
        if s in (NMF_ERR_INVALID_ARG, NMF_ERR_CUDA, NMF_ERR_OOM):
            raise NMFError(s, "nmf_sync")
        return s

    def nmf_objective(self) -> float:
        f = ctypes.c_double(0.0)
        _check(_c_objective(self._h, ctypes.byref(f)), "nmf_objective")
        return f.value

    def nmf_set_pgrad(self, on: bool = True) -> None:
        _check(_c_set_pgrad(self._h, int(bool(on))), "nmf_set_pgrad")

    def nmf_pgrad_history(self, cap: int = 1 << 16):
        buf = (ctypes.c_double * cap)()
        cnt = _I64(0)
        _check(_c_pgrad_history(self._h, ctypes.cast(buf, _P), cap, ctypes.byref(cnt)),
               "nmf_pgrad_history")
        return list(buf[:cnt.value])

    def nmf_iterate_until(self, max_iters: int, rel_tol: float):
        """Returns (iterations run, Delta / Delta(t0) of the last complete iterate)."""
        done = _I32(0)
        ratio = ctypes.c_double(0.0)
        _check(_c_iterate_until(self._h, max_iters, rel_tol, ctypes.byref(done),
                                ctypes.byref(ratio)), "nmf_iterate_until")
        return done.value, ratio.value

    def nmf_objective_history(self, cap: int = 1 << 16):
        buf = (ctypes.c_double * cap)()
        cnt = _I64(0)
        _check(_c_history(self._h, ctypes.cast(buf, _P), cap, ctypes.byref(cnt)),
               "nmf_objective_history")
        return list(buf[:cnt.value])

    def nmf_get_factors(self):
        m, n, k = self.shape
        W = torch.empty((m, k), dtype=torch.float32, device=self.device)
        Ht = torch.empty((n, k), dtype=torch.float32, device=self.device)
        _check(_c_get_factors(self._h, _ptr(W), _ptr(Ht)), "nmf_get_factors")
        self._stream_obj.synchronize()
        return W, Ht

    def nmf_set_factors(self, W=None, Ht=None):
        m, n, k = self.shape
        if W is not None:
            _shape(_dev(W, torch.float32, "W"), (m, k), "W")
        if Ht is not None:
            _shape(_dev(Ht, torch.float32, "Ht"), (n, k), "Ht")
        _check(_c_set_factors(self._h, _ptr(W), _ptr(Ht)), "nmf_set_factors")
        self._stream_obj.synchronize()

    def nmf_get_passive(self):
        m, n, k = self.shape
        nw = (k + 63) // 64
        pW = torch.empty((m, nw), dtype=torch.int64, device=self.device)
        pH = torch.empty((n, nw), dtype=torch.int64, device=self.device)
        _check(_c_get_passive(self._h, _ptr(pW), _ptr(pH)), "nmf_get_passive")
        self._stream_obj.synchronize()
        return pW, pH

    def nmf_get_stats(self) -> dict:
        st = nmf_stats()
        _check(_c_get_stats(self._h, ctypes.byref(st)), "nmf_get_stats")
        return {name: getattr(st, name) for name, _ in nmf_stats._fields_}

    def nmf_set_timing(self, on: bool = True):
        _check(_c_set_timing(self._h, int(bool(on))), "nmf_set_timing")

    def nmf_set_graph(self, on: bool = True):
        _check(_c_set_graph(self._h, int(bool(on))), "nmf_set_graph")

    def nmf_set_proposal(self, mlp, mode: str = "use", epochs: int = 1, batch: int = 8192,
                         lr: float = 1e-3):
        """Attach an nmf_mlp_create network: mode "train", "use" or "off"."""
        modes = {"off": NMF_PROPOSAL_OFF, "train": NMF_PROPOSAL_TRAIN, "use": NMF_PROPOSAL_USE}
        _check(_c_set_proposal(self._h, None if mlp is None else mlp._h, modes[mode], epochs,
                               batch, lr), "nmf_set_proposal")
        self._mlp = mlp   # the handle borrows the network

    def nmf_destroy(self):
        if getattr(self, "_h", None):
            _lib.nmf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.nmf_destroy()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def passive_to_bool(words: torch.Tensor, k: int) -> torch.Tensor:
    """Unpack nrhs x ceil(k/64) int64 bitmasks into an nrhs x k bool tensor."""
    w = words.to(torch.int64)
    bits = torch.arange(64, device=w.device, dtype=torch.int64)
    out = ((w.unsqueeze(-1) >> bits) & 1).bool().reshape(w.shape[0], -1)
    return out[:, :k]


def bool_to_passive(P: torch.Tensor) -> torch.Tensor:
    """Pack an nrhs x k bool tensor into nrhs x ceil(k/64) int64 bitmasks."""
    nrhs, k = P.shape
    nw = (k + 63) // 64
    pad = torch.zeros((nrhs, nw * 64), dtype=torch.int64, device=P.device)
    pad[:, :k] = P.to(torch.int64)
    bits = torch.arange(64, device=P.device, dtype=torch.int64)
    return (pad.reshape(nrhs, nw, 64) << bits).sum(dim=-1)


# ------------------------------------------------------------------ proposal
def nmf_mlp_param_count(k: int, hidden: int) -> int:
    return int(_c_mlp_param_count(k, hidden))


def nmf_mlp_features(G: torch.Tensor, B: torch.Tensor, Xprev=None, out=None,
                     stream=None) -> torch.Tensor:
    """nrhs x 3k features of right-hand sides B (nrhs x k) with Gram G (k x k FP64)."""
    _dev(G, torch.float64, "G")
    _matrix(_dev(B, torch.float32, "B"), "B")
    nrhs, k = B.shape
    _shape(G, (k, k), "G")
    if Xprev is not None:
        _shape(_dev(Xprev, torch.float32, "Xprev"), (nrhs, k), "Xprev")
    out = _out(out, nrhs, 3 * k, B)
    _check(_c_mlp_features(_ptr(G), _ptr(B), _ptr(Xprev), nrhs, k, _ptr(out), _stream(stream)),
           "nmf_mlp_features")
    return out


class nmf_mlp_create:
    """The proposal network (C ABI nmf_mlp_*); `params` is the flat FP32 array."""

    def __init__(self, k: int, hidden: int, params: torch.Tensor, stream=None):
        _dev(params, torch.float32, "params")
        if params.numel() != nmf_mlp_param_count(k, hidden):
            raise ValueError("params has the wrong length")
        self.k, self.hidden = k, hidden
        self.device = params.device
        h = _P()
        _check(_c_mlp_create(ctypes.byref(h), k, hidden, _ptr(params), _stream(stream)),
               "nmf_mlp_create")
        self._h = h

    def nmf_mlp_get_params(self, stream=None) -> torch.Tensor:
        out = torch.empty(nmf_mlp_param_count(self.k, self.hidden), dtype=torch.float32,
                          device=self.device)
        _check(_c_mlp_get_params(self._h, _ptr(out), _stream(stream)), "nmf_mlp_get_params")
        return out

    def _features(self, F: torch.Tensor) -> torch.Tensor:
        _matrix(_dev(F, torch.float32, "F"), "F")
        return _shape(F, (F.shape[0], 3 * self.k), "F")

    def _labels(self, passive: torch.Tensor, nrhs: int) -> torch.Tensor:
        _dev(passive, torch.int64, "passive")
        return _shape(passive, (nrhs, (self.k + 63) // 64), "passive")

    def nmf_mlp_forward(self, F: torch.Tensor, stream=None) -> torch.Tensor:
        self._features(F)
        out = torch.empty((F.shape[0], self.k), dtype=torch.float32, device=F.device)
        _check(_c_mlp_forward(self._h, _ptr(F), F.shape[0], _ptr(out), _stream(stream)),
               "nmf_mlp_forward")
        return out

    def nmf_mlp_propose(self, F: torch.Tensor, stream=None) -> torch.Tensor:
        self._features(F)
        nw = (self.k + 63) // 64
        out = torch.empty((F.shape[0], nw), dtype=torch.int64, device=F.device)
        _check(_c_mlp_propose(self._h, _ptr(F), F.shape[0], _ptr(out), _stream(stream)),
               "nmf_mlp_propose")
        return out

    def nmf_mlp_gradient(self, F: torch.Tensor, passive: torch.Tensor, stream=None):
        self._labels(passive, self._features(F).shape[0])
        g = torch.empty(nmf_mlp_param_count(self.k, self.hidden), dtype=torch.float32,
                        device=F.device)
        loss = torch.empty(1, dtype=torch.float64, device=F.device)
        _check(_c_mlp_gradient(self._h, _ptr(F), _ptr(passive), F.shape[0], _ptr(g), _ptr(loss),
                               _stream(stream)), "nmf_mlp_gradient")
        return g, loss

    def nmf_mlp_train(self, F: torch.Tensor, passive: torch.Tensor, batch: int = 8192,
                      lr: float = 1e-3, stream=None) -> torch.Tensor:
        self._labels(passive, self._features(F).shape[0])
        loss = torch.empty(1, dtype=torch.float64, device=F.device)
        _check(_c_mlp_train(self._h, _ptr(F), _ptr(passive), F.shape[0], batch, lr, _ptr(loss),
                            _stream(stream)), "nmf_mlp_train")
        return loss

    def nmf_mlp_destroy(self):
        if getattr(self, "_h", None):
            _lib.nmf_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.nmf_mlp_destroy()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass
