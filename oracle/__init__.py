"""ctypes binding of the FP64 CPU oracle (``nmf_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg. The product path never imports it.

All functions take numpy arrays and return numpy arrays in float64. The
float32 input matrix A is passed as stored (both paths read the same bits);
factors are promoted to float64 before any arithmetic.

``Oracle(path)`` wraps one compiled copy of the C source; the module-level
functions use the default build. Tests compile deliberately broken copies of
the source into other paths to check that the pins catch the mistake.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "nmf_oracle.c")
LIB_PATH = os.path.join(_HERE, "liboracle.so")

OK = 0
NOT_CONVERGED = 4
SINGULAR = 5
SOLVERS = {"bpp": 0, "mu": 1, "hals": 2}


def compile_source(src: str, out: str) -> str:
    """gcc -O2 with IEEE semantics kept (no fast-math, no FMA contraction)."""
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        compile_source(SRC, LIB_PATH)
    return LIB_PATH


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        lib.oracle_num_threads.restype = I
        lib.oracle_gram.argtypes = [P, I64, I, P]
        lib.oracle_mm_dense.argtypes = [P, I64, I64, I64, P, I, I, P]
        lib.oracle_mm_csr.argtypes = [P, P, P, I64, I64, P, I, I, P]
        lib.oracle_objective_dense.argtypes = [P, I64, I64, I64, P, P, I]
        lib.oracle_objective_dense.restype = ctypes.c_double
        lib.oracle_objective_csr.argtypes = [P, P, P, I64, I64, P, P, I]
        lib.oracle_objective_csr.restype = ctypes.c_double
        lib.oracle_bpp.argtypes = [P, I, P, I64, P, P, I, I, P, P]
        lib.oracle_bpp.restype = I
        lib.oracle_anls.argtypes = [I, P, I64, P, P, P, I64, I64, I, P, P, I, I, I, P, P, P, P, I]
        lib.oracle_mu.argtypes = [P, I, P, I64, P]
        lib.oracle_pgrad_sq.argtypes = [P, I, P, I64, P]
        lib.oracle_pgrad_sq.restype = ctypes.c_double
        lib.oracle_hals.argtypes = [P, I, P, I64, P]
        lib.oracle_anls.restype = I
        self.lib = lib

    def num_threads(self) -> int:
        return self.lib.oracle_num_threads()

    def gram(self, X) -> np.ndarray:
        """G = X^T X for X (rows x k): H H^T when X = H^T, W^T W when X = W."""
        X = _f64(X)
        rows, k = X.shape
        G = np.empty((k, k), dtype=np.float64)
        self.lib.oracle_gram(_p(X), rows, k, _p(G))
        return G

    def mm_dense(self, A, F, trans: bool) -> np.ndarray:
        """trans=False: A F (F = H^T, n x k) -> m x k.  trans=True: A^T F (F = W) -> n x k."""
        A = np.ascontiguousarray(A, dtype=np.float32)
        F = _f64(F)
        m, n = A.shape
        k = F.shape[1]
        out = np.empty((n if trans else m, k), dtype=np.float64)
        self.lib.oracle_mm_dense(_p(A), m, n, n, _p(F), k, int(trans), _p(out))
        return out

    def mm_csr(self, rowptr, colidx, vals, m, n, F, trans: bool) -> np.ndarray:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float32)
        F = _f64(F)
        k = F.shape[1]
        out = np.empty((n if trans else m, k), dtype=np.float64)
        self.lib.oracle_mm_csr(_p(rowptr), _p(colidx), _p(vals), m, n, _p(F), k, int(trans),
                               _p(out))
        return out

    def objective_dense(self, A, W, Ht) -> float:
        A = np.ascontiguousarray(A, dtype=np.float32)
        W, Ht = _f64(W), _f64(Ht)
        m, n = A.shape
        return self.lib.oracle_objective_dense(_p(A), m, n, n, _p(W), _p(Ht), W.shape[1])

    def objective_csr(self, rowptr, colidx, vals, m, n, W, Ht) -> float:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float32)
        W, Ht = _f64(W), _f64(Ht)
        return self.lib.oracle_objective_csr(_p(rowptr), _p(colidx), _p(vals), m, n, _p(W),
                                             _p(Ht), W.shape[1])

    def bpp(self, G, B, passive_in=None, max_rounds: int = 1000):
        """Batched BPP: each row b of B gives min_{x>=0} 0.5 x^T G x - b^T x.

        Returns (X, passive uint8 nrhs x k, rounds int32, status int8, worst)."""
        G = _f64(G)
        B = _f64(B)
        if B.ndim == 1:
            B = B[None, :]
        nrhs, k = B.shape
        X = np.empty_like(B)
        if passive_in is not None:
            passive = np.ascontiguousarray(passive_in, dtype=np.uint8).reshape(nrhs, k).copy()
            warm = 1
        else:
            passive = np.zeros((nrhs, k), dtype=np.uint8)
            warm = 0
        rounds = np.zeros(nrhs, dtype=np.int32)
        status = np.zeros(nrhs, dtype=np.int8)
        worst = self.lib.oracle_bpp(_p(G), k, _p(B), nrhs, _p(X), _p(passive), warm, max_rounds,
                                    _p(rounds), _p(status))
        return X, passive, rounds, status, worst

    def mu(self, G, R, X) -> np.ndarray:
        """One MU step (Eq. 5) of the rows of X (rows x k) with Gram G and
        right-hand sides R (rows x k); returns the new X."""
        G, R = _f64(G), _f64(R)
        X = _f64(X).copy()
        self.lib.oracle_mu(_p(G), G.shape[0], _p(R), X.shape[0], _p(X))
        return X

    def pgrad_sq(self, G, R, X) -> float:
        """Squared projected-gradient norm of the rows of X: grad = X G - R,
        entries with x = 0 count only where grad < 0."""
        G, R, X = _f64(G), _f64(R), _f64(X)
        return self.lib.oracle_pgrad_sq(_p(G), G.shape[0], _p(R), X.shape[0], _p(X))

    def pgrad(self, W, Ht, A=None, csr=None, shape=None) -> float:
        """Projected-gradient norm of f at (W, H) (half the gradient of Eq. 1):
        sqrt(|P[W H H^T - A H^T]|^2 + |P[H^T W^T W - A^T W]|^2)."""
        W, Ht = _f64(W), _f64(Ht)
        if csr is None:
            V, Y = self.mm_dense(A, Ht, False), self.mm_dense(A, W, True)
        else:
            m, n = shape
            V = self.mm_csr(*csr, m, n, Ht, False)
            Y = self.mm_csr(*csr, m, n, W, True)
        return float(np.sqrt(self.pgrad_sq(self.gram(Ht), V, W) + self.pgrad_sq(self.gram(W), Y, Ht)))

    def hals(self, G, R, X) -> np.ndarray:
        """One HALS sweep (Eq. 6) of the rows of X; returns the new X."""
        G, R = _f64(G), _f64(R)
        X = _f64(X).copy()
        self.lib.oracle_hals(_p(G), G.shape[0], _p(R), X.shape[0], _p(X))
        return X

    def anls(self, A=None, W0=None, Ht0=None, iters: int = 10, warm: bool = False,
             max_rounds: int = 1000, csr=None, shape=None, solver: str = "bpp"):
        """Alg. 1 for ``iters`` iterations from (W0, H0^T). Dense A (float32 m x n)
        or csr=(rowptr, colidx, vals) with shape=(m, n). solver: "bpp" (Sec. 4.2),
        "mu" (Eq. 5) or "hals" (Eq. 6).

        Returns dict(W, Ht, f (iters+1), passive_W, passive_H, rounds (2*iters),
        status)."""
        W = _f64(W0).copy()
        Ht = _f64(Ht0).copy()
        m, k = W.shape
        n = Ht.shape[0]
        f = np.empty(iters + 1, dtype=np.float64)
        pW = np.zeros((m, k), dtype=np.uint8)
        pH = np.zeros((n, k), dtype=np.uint8)
        rh = np.zeros(2 * iters, dtype=np.int64)
        if csr is None:
            A = np.ascontiguousarray(A, dtype=np.float32)
            assert A.shape == (m, n)
            st = self.lib.oracle_anls(0, _p(A), n, None, None, None, m, n, k, _p(W), _p(Ht),
                                      iters, int(warm), max_rounds, _p(f), _p(pW), _p(pH), _p(rh),
                                      SOLVERS[solver])
        else:
            rowptr, colidx, vals = csr
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
            colidx = np.ascontiguousarray(colidx, dtype=np.int32)
            vals = np.ascontiguousarray(vals, dtype=np.float32)
            assert shape == (m, n)
            st = self.lib.oracle_anls(1, None, 0, _p(rowptr), _p(colidx), _p(vals), m, n, k,
                                      _p(W), _p(Ht), iters, int(warm), max_rounds, _p(f), _p(pW),
                                      _p(pH), _p(rh), SOLVERS[solver])
        return dict(W=W, Ht=Ht, f=f, passive_W=pW, passive_H=pH, rounds=rh, status=st)


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def num_threads():
    return default().num_threads()


def gram(X):
    return default().gram(X)


def mm_dense(A, F, trans):
    return default().mm_dense(A, F, trans)


def mm_csr(rowptr, colidx, vals, m, n, F, trans):
    return default().mm_csr(rowptr, colidx, vals, m, n, F, trans)


def objective_dense(A, W, Ht):
    return default().objective_dense(A, W, Ht)


def objective_csr(rowptr, colidx, vals, m, n, W, Ht):
    return default().objective_csr(rowptr, colidx, vals, m, n, W, Ht)


def bpp(G, B, passive_in=None, max_rounds=1000):
    return default().bpp(G, B, passive_in, max_rounds)


def mu(G, R, X):
    return default().mu(G, R, X)


def hals(G, R, X):
    return default().hals(G, R, X)


def pgrad_sq(G, R, X):
    return default().pgrad_sq(G, R, X)


def pgrad(W, Ht, A=None, csr=None, shape=None):
    return default().pgrad(W, Ht, A, csr, shape)


def anls(A=None, W0=None, Ht0=None, iters=10, warm=False, max_rounds=1000, csr=None, shape=None,
         solver="bpp"):
    return default().anls(A, W0, Ht0, iters, warm, max_rounds, csr, shape, solver)
