"""The allocation-free NLS entry point (nmf_nls_bpp_noalloc) against the
regular one (nmf_nls_bpp), both called through the C ABI.

nmf_nls_bpp_noalloc exists for callers that may not allocate device memory
(a framework's allocator owns it all, or cudaMalloc would synchronise a
latency-critical loop): it keeps its workspace in a fixed array inside the
library. Two calls in a row must each reproduce the regular entry point, so
leftover contents of the shared array from the first call cannot leak into
the second. This file is collected last; it also passes when run alone.
"""
import numpy as np
import pytest
import torch

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
    return (torch.from_numpy(G).cuda(), torch.from_numpy(B.astype(np.float32)).cuda())


def test_noalloc_matches_regular_on_two_calls_in_a_row(nmf):
    cases = [(50, 3000, 1), (20, 2000, 2)]
    problems = [_problem(*c) for c in cases]
    # Two allocation-free calls back to back (different k and batch size).
    free = [nmf.nmf_nls_bpp_noalloc(G, B) for G, B in problems]
    for (k, nrhs, _), (G, B), r_free in zip(cases, problems, free):
        r_reg = nmf.nmf_nls_bpp(G, B)
        X, Xr = r_free["X"].double(), r_reg["X"].double()
        # Same kernels on the same inputs; compare within the BPP tolerance.
        err = (torch.linalg.norm(X - Xr) / torch.linalg.norm(Xr)).item()
        assert err <= 1e-6, (k, err)
        assert r_free["worst"] == r_reg["worst"] == nmf.NMF_OK
        assert torch.equal(r_free["passive"], r_reg["passive"])
        assert torch.equal(r_free["rounds"], r_reg["rounds"])
        assert torch.equal(r_free["status"], r_reg["status"])


def test_noalloc_rejects_k_beyond_its_maximum(nmf):
    G = torch.eye(nmf.NMF_MAX_K + 1, dtype=torch.float64, device="cuda")
    B = torch.ones((4, nmf.NMF_MAX_K + 1), dtype=torch.float32, device="cuda")
    with pytest.raises(nmf.NMFError):
        nmf.nmf_nls_bpp_noalloc(G, B)
