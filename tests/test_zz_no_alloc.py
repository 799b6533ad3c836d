"""The allocation-free NLS entry point (nmf_nls_bpp_noalloc) against the
regular one (nmf_nls_bpp) and the FP64 oracle, all called through the C ABI.

nmf_nls_bpp_noalloc exists for callers that may not allocate device memory
(a framework's allocator owns it all, or cudaMalloc would synchronise a
latency-critical loop): it keeps its workspace in a fixed array inside the
library. It runs the same kernels with the same launch shape on the same
inputs as nmf_nls_bpp, so its results must be bitwise the same, on every call
of a sequence: leftover contents of the shared array from one call must not
leak into the next. This file is collected last; it also passes when run
alone.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_09313_gb300 as lib
    return lib


def _problem(k, nrhs, seed):
    G, B = synth.nls_batch(k, nrhs, seed=seed)
    return G, B.astype(np.float32)


def _margin_ok(G, B, X, P, rel=1e-3):
    # Right-hand sides whose KKT margin is clear of rounding: every passive x_i
    # at least rel * max|x|, every active y_i at least rel * max|b|.
    Y = X @ G - B
    xm = np.where(P, X, np.inf).min(axis=1) / np.maximum(np.abs(X).max(axis=1), 1e-300)
    ym = np.where(~P, Y, np.inf).min(axis=1) / np.maximum(np.abs(B).max(axis=1), 1e-300)
    return np.minimum(xm, ym) >= rel


def test_noalloc_matches_regular_on_calls_in_a_row(nmf):
    # Three allocation-free calls back to back: different k and batch sizes,
    # the last at the largest k the fixed array holds. Then the regular entry
    # point on the same inputs; every output must be bitwise equal.
    cases = [(50, 3000, 1), (20, 2000, 2), (nmf.NMF_MAX_K, 700, 3)]
    problems = [_problem(*c) for c in cases]
    dev = [(torch.from_numpy(G).cuda(), torch.from_numpy(B).cuda()) for G, B in problems]
    free = [nmf.nmf_nls_bpp_noalloc(G, B) for G, B in dev]
    for (k, nrhs, _), (G, B), r_free in zip(cases, dev, free):
        r_reg = nmf.nmf_nls_bpp(G, B)
        assert r_free["worst"] == r_reg["worst"] == nmf.NMF_OK, k
        for key in ("X", "passive", "rounds", "status"):
            assert torch.equal(r_free[key], r_reg[key]), (k, key)


def test_noalloc_matches_oracle(nmf):
    # One batch against the FP64 oracle, with the BPP tolerances of the kernel
    # tests: ||x - x_or|| / ||x_or|| <= 20 cond(G) 6e-8; identical passive sets
    # and round counts on right-hand sides with a clear KKT margin.
    for k, nrhs, seed in ((50, 2000, 11), (nmf.NMF_MAX_K, 500, 12)):
        G, B = _problem(k, nrhs, seed)
        r = nmf.nmf_nls_bpp_noalloc(torch.from_numpy(G).cuda(), torch.from_numpy(B).cuda())
        assert r["worst"] == nmf.NMF_OK
        X = r["X"].double().cpu().numpy()
        P = nmf.passive_to_bool(r["passive"], k).cpu().numpy()
        R = r["rounds"].cpu().numpy()
        Bd = B.astype(np.float64)
        Xo, Po, Ro, So, wo = oracle.bpp(G, Bd)
        assert wo == 0
        cond = np.linalg.cond(G)
        err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
        assert err <= 20 * cond * 6e-8, (k, err, cond)
        ok = _margin_ok(G, Bd, Xo, Po.astype(bool))
        assert ok.mean() > 0.3, ok.mean()
        assert np.array_equal(P[ok], Po.astype(bool)[ok])
        assert (R[ok] == Ro[ok]).mean() >= 0.98


def test_noalloc_rejects_k_beyond_its_maximum(nmf):
    G = torch.eye(nmf.NMF_MAX_K + 1, dtype=torch.float64, device="cuda")
    B = torch.ones((4, nmf.NMF_MAX_K + 1), dtype=torch.float32, device="cuda")
    before = nmf.nmf_kernel_launches()
    with pytest.raises(nmf.NMFError):
        nmf.nmf_nls_bpp_noalloc(G, B)
    assert nmf.nmf_kernel_launches() == before
