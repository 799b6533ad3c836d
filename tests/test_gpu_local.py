"""MU (Eq. 5) and HALS (Eq. 6) on the GPU against the FP64 oracle.

One step of either update is a fixed function of (G, R, X); the kernels work
in FP32 (G rounded to FP32, products accumulated in FP32), so an entry carries
an error of a few units of FP32 rounding times the size of the terms it sums:
MU ~ k * 6e-8 relative, HALS a little more (each coordinate uses the others'
new values). The tolerances below are 2e-5 of each row's scale. Whole ANLS
runs compare the objective history (1e-5 relative, as for BPP) and the
factors (1e-4 relative Frobenius).
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


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def problem(rows, k, seed, zero_frac=0.2):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0.0, 1.0, (4 * k + 8, k))
    G = C.T @ C
    X = rng.uniform(0.0, 1.0, (rows, k)) * (rng.uniform(0, 1, (rows, k)) > zero_frac)
    R = rng.uniform(0.0, 1.0, (rows, k)) @ G * 0.8
    return G, R.astype(np.float32), X.astype(np.float32)


def row_rel_err(got, ref):
    scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-30)
    return float((np.abs(got - ref) / scale).max())


@pytest.mark.parametrize("k", [1, 7, 32, 33, 50, 64, 65, 100, 128])
@pytest.mark.parametrize("solver", ["mu", "hals"])
def test_step_matches_oracle(nmf, solver, k):
    rows = 1000 + 37   # several CTAs, a ragged last one
    G, R, X = problem(rows, k, seed=k)
    Xd = dev(X)
    fn = nmf.nmf_update_mu if solver == "mu" else nmf.nmf_update_hals
    fn(dev(G, torch.float64), dev(R), Xd)
    got = Xd.double().cpu().numpy()
    ref = (oracle.mu if solver == "mu" else oracle.hals)(G, R, X)
    err = row_rel_err(got, ref)
    print(f"{solver} k={k} max row-relative error {err:.2e}")
    assert err <= 2e-5, err
    assert (got >= 0).all()


def test_mu_zero_rows_and_hals_zero_column(nmf):
    k, rows = 12, 300
    G, R, X = problem(rows, k, seed=3)
    X[::5] = 0.0                       # MU: (X G) = 0 on these rows; they stay 0
    Xd = dev(X)
    nmf.nmf_update_mu(dev(G, torch.float64), dev(R), Xd)
    got = Xd.cpu().numpy()
    assert np.isfinite(got).all() and (got[::5] == 0).all()
    G0 = G.copy()
    G0[4, :] = 0.0
    G0[:, 4] = 0.0                     # HALS: G_44 = 0 sets x_4 to 0
    Xd = dev(X + 1.0)
    nmf.nmf_update_hals(dev(G0, torch.float64), dev(R), Xd)
    got = Xd.double().cpu().numpy()
    assert (got[:, 4] == 0).all()
    ref = oracle.hals(G0, R, X + 1.0)
    assert row_rel_err(got, ref) <= 2e-5


def test_empty_batch_is_a_no_op(nmf):
    G = dev(np.eye(5), torch.float64)
    X = torch.empty((0, 5), dtype=torch.float32, device="cuda")
    R = torch.empty((0, 5), dtype=torch.float32, device="cuda")
    nmf.nmf_update_mu(G, R, X)
    nmf.nmf_update_hals(G, R, X)
    torch.cuda.synchronize()


def run_anls(nmf, A, W0, Ht0, iters, solver, precision="fp32", csr=None, shape=None):
    Ad = dev(A) if csr is None else tuple(torch.from_numpy(x).cuda() for x in csr)
    h = nmf.nmf_init(Ad, dev(W0), dev(Ht0), precision=precision, solver=solver, shape=shape)
    h.nmf_iterate(iters)
    assert h.nmf_sync() == nmf.NMF_OK
    W, Ht = h.nmf_get_factors()
    f = np.array(h.nmf_objective_history())
    st = h.nmf_get_stats()
    h.nmf_destroy()
    assert st["bpp_rhs"] == 0          # no BPP solve ran
    return W.double().cpu().numpy(), Ht.double().cpu().numpy(), f


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("solver", ["mu", "hals"])
def test_anls_dense_matches_oracle(nmf, solver, precision):
    m, n, k, T = 2000, 1000, 10, 10
    A = synth.dense_planted(m, n, k, 0.01)
    W0, Ht0 = synth.init_factors(m, n, k)
    ref = oracle.anls(A, W0, Ht0, iters=T, solver=solver)
    W, Ht, f = run_anls(nmf, A, W0, Ht0, T, solver, precision)
    errf = np.abs(f - ref["f"][1:]) / ref["f"][1:]
    errW = np.linalg.norm(W - ref["W"]) / np.linalg.norm(ref["W"])
    errH = np.linalg.norm(Ht - ref["Ht"]) / np.linalg.norm(ref["Ht"])
    print(f"{solver}/{precision}: f {errf.max():.2e}  W {errW:.2e}  H {errH:.2e}")
    assert errf.max() <= 1e-5
    assert errW <= 1e-4 and errH <= 1e-4
    assert (f[1:] <= f[:-1] * (1 + 1e-6)).all()   # both updates never increase f


@pytest.mark.parametrize("solver", ["mu", "hals"])
def test_anls_sparse_matches_oracle(nmf, solver):
    m, n, k, T = 20000, 10000, 20, 5
    csr = synth.csr_uniform(m, n, 200000)
    W0, Ht0 = synth.init_factors(m, n, k)
    ref = oracle.anls(None, W0, Ht0, iters=T, csr=csr, shape=(m, n), solver=solver)
    W, Ht, f = run_anls(nmf, None, W0, Ht0, T, solver, csr=csr, shape=(m, n))
    errf = np.abs(f - ref["f"][1:]) / ref["f"][1:]
    errW = np.linalg.norm(W - ref["W"]) / np.linalg.norm(ref["W"])
    errH = np.linalg.norm(Ht - ref["Ht"]) / np.linalg.norm(ref["Ht"])
    print(f"sparse {solver}: f {errf.max():.2e}  W {errW:.2e}  H {errH:.2e}")
    assert errf.max() <= 1e-5
    assert errW <= 1e-4 and errH <= 1e-4


def test_proposal_rejected_for_mu(nmf):
    m, n, k = 200, 100, 8
    A = synth.dense_planted(m, n, k, 0.01)
    W0, Ht0 = synth.init_factors(m, n, k)
    h = nmf.nmf_init(dev(A), dev(W0), dev(Ht0), solver="mu")
    net = nmf.nmf_mlp_create(k, 16, torch.from_numpy(synth.mlp_init(k, 16)).cuda())
    with pytest.raises(nmf.NMFError):
        h.nmf_set_proposal(net, "train")
    h.nmf_destroy()
