"""Whole ANLS iterations on the GPU (C-ABI handle) against the FP64 oracle run
from the same seeded inputs and starting point.

Tolerances: relative objective <= 1e-5 and relative factor error
(Frobenius) <= 1e-4 after the fixed iteration count; the GPU objective must be
non-increasing up to 1e-6 relative (each half-step is an exact minimisation,
Eq. 2).
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_gpu(nmf, A, W0, Ht0, iters, precision="fp32", start="cold", csr=None, shape=None,
            graph=False, stream=None):
    if csr is None:
        Ad = dev(A)
    else:
        Ad = tuple(dev(x) for x in csr)
    h = nmf.nmf_init(Ad, dev(W0), dev(Ht0), precision=precision, start=start, shape=shape,
                     stream=stream)
    h.nmf_set_graph(graph)
    h.nmf_iterate(iters)
    status = h.nmf_sync()
    W, Ht = h.nmf_get_factors()
    f = np.array(h.nmf_objective_history())
    stats = h.nmf_get_stats()
    h.nmf_destroy()
    return dict(W=W.double().cpu().numpy(), Ht=Ht.double().cpu().numpy(), f=f, status=status,
                stats=stats)


def check(nmf, g, ref, ftol=1e-5, xtol=1e-4):
    assert g["status"] == nmf.NMF_OK
    f_or = ref["f"][1:]
    assert len(g["f"]) == len(f_or)
    errf = np.abs(g["f"] - f_or) / f_or
    errW, errH = rel(g["W"], ref["W"]), rel(g["Ht"], ref["Ht"])
    print(f"max rel f err {errf.max():.2e} (at iteration {int(errf.argmax()) + 1})  "
          f"W {errW:.2e}  H {errH:.2e}  stats {g['stats']}")
    assert errf.max() <= ftol
    assert errW <= xtol and errH <= xtol
    assert (g["f"][1:] <= g["f"][:-1] * (1 + 1e-6)).all()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("start", ["cold", "warm"])
def test_dense_small_config(nmf, start, precision):
    # A = W0 H0 + |N(0, 0.01^2)|, 2000 x 1000, k = 10, 10 iterations. The
    # configuration is defined for the FP32 path (objective within 1e-5). The
    # BF16x3 products' own random error over this short contraction (1.6e-7)
    # moves the objective by ~1e-5 by itself (test_product_noise.py: median
    # 1e-5, max 1.4e-5 over eight draws), so that path is held to 3e-5 here.
    m, n, k, T = 2000, 1000, 10, 10
    A = synth.dense_planted(m, n, k, 0.01)
    W0, Ht0 = synth.init_factors(m, n, k)
    ref = oracle.anls(A, W0, Ht0, iters=T)
    g = run_gpu(nmf, A, W0, Ht0, T, start=start, precision=precision)
    check(nmf, g, ref, ftol=1e-5 if precision == "fp32" else 3e-5)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_dense_large_config_crop(nmf, precision):
    # The 96000 x 64000 recipe (k = 50, sigma = 0.05) on its 4000 x 2000 crop,
    # 30 iterations.
    m, n, k, T = 4000, 2000, 50, 30
    A = synth.dense_planted(m, n, k, 0.05, m_full=96000, n_full=64000)
    W0, Ht0 = synth.init_factors(m, n, k)
    ref = oracle.anls(A, W0, Ht0, iters=T)
    g = run_gpu(nmf, A, W0, Ht0, T, start="warm", precision=precision)
    check(nmf, g, ref)


def test_sparse_config_scaled(nmf):
    # The sparse recipe (uniform positions, values in (0, 1], k = 50) scaled to
    # 20000 x 10000 with 200k draws, 5 iterations.
    m, n, k, T = 20000, 10000, 50, 5
    csr = synth.csr_uniform(m, n, 200000)
    W0, Ht0 = synth.init_factors(m, n, k)
    ref = oracle.anls(None, W0, Ht0, iters=T, csr=csr, shape=(m, n))
    g = run_gpu(nmf, None, W0, Ht0, T, start="warm", csr=csr, shape=(m, n))
    check(nmf, g, ref)


def test_sparse_objective_standalone(nmf):
    # nmf_objective outside an iteration (A^T W and W^T W formed on the spot) at
    # the starting point and after two iterations; the in-iteration form (from
    # the H half-step's right-hand sides) must give the same value.
    m, n, k = 3000, 2000, 20
    csr = synth.csr_uniform(m, n, 60000, seed=7)
    W0, Ht0 = synth.init_factors(m, n, k, seed=7)
    h = nmf.nmf_init(tuple(dev(x) for x in csr), dev(W0), dev(Ht0), shape=(m, n))
    f0 = h.nmf_objective()
    ref0 = oracle.objective_csr(*csr, m, n, W0, Ht0)
    assert abs(f0 - ref0) / ref0 <= 1e-6
    h.nmf_iterate(2)
    f2 = h.nmf_objective()
    W, Ht = h.nmf_get_factors()
    ref2 = oracle.objective_csr(*csr, m, n, W.double().cpu().numpy(), Ht.double().cpu().numpy())
    assert abs(f2 - ref2) / ref2 <= 1e-6
    hist = h.nmf_objective_history()
    assert abs(hist[-1] - f2) / f2 <= 1e-6
    h.nmf_destroy()


def test_sparse_set_factors_resume(nmf):
    # A sparse handle reuses the Gram of H formed by the objective for the next
    # W half-step; replacing H^T must drop it. After set_factors the handle
    # continues bitwise like a fresh handle started from the same factors.
    m, n, k = 3000, 2000, 20
    csr = synth.csr_uniform(m, n, 60000, seed=9)
    W0, Ht0 = synth.init_factors(m, n, k, seed=9)
    dcsr = tuple(dev(x) for x in csr)
    h = nmf.nmf_init(dcsr, dev(W0), dev(Ht0), shape=(m, n), start="warm")
    h.nmf_iterate(3)
    W3, H3 = h.nmf_get_factors()
    Hp = (H3 * 1.25 + 0.01).contiguous()
    h.nmf_set_factors(W3.contiguous(), Hp)
    h.nmf_iterate(2)
    W5, H5 = h.nmf_get_factors()
    h2 = nmf.nmf_init(dcsr, W3.contiguous(), Hp.clone(), shape=(m, n), start="warm")
    h2.nmf_iterate(2)
    W5b, H5b = h2.nmf_get_factors()
    assert torch.equal(W5, W5b) and torch.equal(H5, H5b)
    f, f2 = h.nmf_objective(), h2.nmf_objective()
    assert f == f2
    h.nmf_destroy()
    h2.nmf_destroy()


def _bf16x3_runs(nmf, A, W0, Ht0, T):
    # The same run with and without the pre-split copies of A and A^T.
    out = []
    for copies in (True, False):
        h = nmf.nmf_init(dev(A), dev(W0), dev(Ht0), precision="bf16x3", start="warm",
                         split_copies=copies)
        h.nmf_iterate(T)
        assert h.nmf_sync() == nmf.NMF_OK
        W, Ht = h.nmf_get_factors()
        st = h.nmf_get_stats()
        out.append((W.cpu().numpy(), Ht.cpu().numpy(), np.array(h.nmf_objective_history()), st))
        h.nmf_destroy()
    (W1, H1, f1, st1), (W2, H2, f2, st2) = out
    assert np.array_equal(W1, W2) and np.array_equal(H1, H2) and np.array_equal(f1, f2)
    return W1, H1, f1, st1


def test_bf16x3_k_above_64(nmf):
    # k > 64: the products run in two 64-column chunks (from the pre-split
    # copies, or splitting A in the pass) and the objective is a separate
    # pass (no fusion); both give bitwise the same factors. The start lies
    # within 10% of the planted factors, so every Gram stays well conditioned
    # and every half-step runs the FP32 solves; W, H and f must meet the target
    # tolerances against the oracle. (The noise level is the 96000 x 64000
    # recipe's, sigma = 0.05: with a nearly exact fit, f is so small that its
    # relative error is no longer a measure of the factors'.)
    m, n, k, T = 3000, 2400, 80, 4
    A, W0p, H0p = synth.dense_planted(m, n, k, 0.05, seed=13, return_factors=True)
    W0 = (W0p * (0.9 + 0.2 * synth.uniform_matrix(13, synth.TID_W_INIT, m, k)))
    Ht0 = (H0p.T * (0.9 + 0.2 * synth.uniform_matrix(13, synth.TID_H_INIT, n, k)))
    W0, Ht0 = W0.astype(np.float32), np.ascontiguousarray(Ht0.astype(np.float32))
    ref = oracle.anls(A, W0, Ht0, iters=T, warm=True)
    W1, H1, f1, st1 = _bf16x3_runs(nmf, A, W0, Ht0, T)
    assert st1["bpp_fp64_halfsteps"] == 0 and st1["bpp_fp64_solves"] == 0, st1
    errf = np.abs(f1 - ref["f"][1:]) / ref["f"][1:]
    errW = rel(W1.astype(np.float64), ref["W"])
    errH = rel(H1.astype(np.float64), ref["Ht"])
    print(f"k={k}: f {errf.max():.2e} W {errW:.2e} H {errH:.2e}")
    assert errf.max() <= 1e-5, errf
    assert errW <= 1e-4 and errH <= 1e-4, (errW, errH)


def test_bf16x3_k_above_64_fp64_halfsteps(nmf):
    # The same chunked products from a uniform random start: the Grams of the
    # first iterates are ill-conditioned, so the H updates run the FP64 solves.
    # The objective matches the oracle within the BF16x3 tolerance.
    m, n, k, T = 1500, 1200, 80, 4
    A = synth.dense_planted(m, n, k, 0.01, seed=13)
    W0, Ht0 = synth.init_factors(m, n, k, seed=13)
    ref = oracle.anls(A, W0, Ht0, iters=T, warm=True)
    W1, H1, f1, st1 = _bf16x3_runs(nmf, A, W0, Ht0, T)
    assert st1["bpp_fp64_halfsteps"] > 0, st1
    errf = np.abs(f1 - ref["f"][1:]) / ref["f"][1:]
    assert errf.max() <= 3e-5, errf


def test_split_copies_give_the_same_products(nmf):
    # The pre-split BF16 copies of A and A^T hold exactly the hi / lo values the
    # in-pass split forms, so the factors of a BF16x3 run are bitwise the same
    # with and without them; only the fused objective changes (its residuals
    # use hi + lo, within 2^-18 of A).
    m, n, k, T = 3000, 2000, 24, 6
    A = synth.dense_planted(m, n, k, 0.02, seed=11)
    W0, Ht0 = synth.init_factors(m, n, k, seed=11)
    out = []
    for copies in (True, False):
        h = nmf.nmf_init(dev(A), dev(W0), dev(Ht0), precision="bf16x3", start="warm",
                         split_copies=copies)
        h.nmf_iterate(T)
        assert h.nmf_sync() == nmf.NMF_OK
        W, Ht = h.nmf_get_factors()
        out.append((W.cpu().numpy(), Ht.cpu().numpy(), np.array(h.nmf_objective_history())))
        h.nmf_destroy()
    (W1, H1, f1), (W2, H2, f2) = out
    assert np.array_equal(W1, W2) and np.array_equal(H1, H2)
    assert np.abs(f1 - f2).max() <= 1e-7 * f2.max()


@pytest.mark.parametrize("k,start,ill", [(20, "warm", False), (50, "warm", False),
                                         (50, "cold", False), (12, "warm", True)])
def test_sparse_fused_products_bitwise(nmf, k, start, ill):
    # Sparse BPP half-steps gather each right-hand side inside the FP32 solves,
    # in the SpMM kernel's order, and write it to V / Y as they go: bitwise the
    # same factors, objective history, passive sets and round counts as the
    # separate SpMM pass. `ill`: H0's columns share a dominant common part, so
    # the first half-steps run in FP64 and take their right-hand sides from the
    # SpMM that runs only then.
    m, n, T = 20000, 10000, 4
    csr = synth.csr_uniform(m, n, 200000, seed=7)
    W0, Ht0 = synth.init_factors(m, n, k, seed=7)
    if ill:
        Ht0 = (Ht0 + 1000.0 * Ht0[:, :1]).astype(np.float32)
    # The separate-SpMM path runs the group-tile pass first; its SIMT form
    # (launch shape group = 1) gives the per-warp kernel's bits, so the two
    # paths are compared with it (the tensor-core form is checked against the
    # oracle in test_gpu_kernels.py).
    old_shape = nmf.nmf_nls_bpp_get_shape(k)
    nmf.nmf_nls_bpp_set_shape(k, old_shape[0], old_shape[1], 1)
    outs = []
    try:
        for fused in (False, True):
            h = nmf.nmf_init(tuple(dev(x) for x in csr), dev(W0), dev(Ht0), shape=(m, n),
                             start=start, fused_products=fused)
            h.nmf_iterate(T)
            assert h.nmf_sync() == nmf.NMF_OK
            W, Ht = h.nmf_get_factors()
            pW, pH = h.nmf_get_passive()
            st = h.nmf_get_stats()
            outs.append((W.cpu(), Ht.cpu(), np.array(h.nmf_objective_history()), pW.cpu(),
                         pH.cpu(), st))
            h.nmf_destroy()
    finally:
        nmf.nmf_nls_bpp_set_shape(k, *old_shape)
    (W0_, H0_, f0, pW0, pH0, s0), (W1, H1, f1, pW1, pH1, s1) = outs
    print(f"k={k} {start} ill={ill}: f {f1} fp64 half-steps {s1['bpp_fp64_halfsteps']} "
          f"launches {s0['kernel_launches']} -> {s1['kernel_launches']}")
    assert torch.equal(W1, W0_) and torch.equal(H1, H0_)
    assert np.array_equal(f1, f0)
    assert torch.equal(pW1, pW0) and torch.equal(pH1, pH0)
    for key in ("bpp_rhs", "bpp_rounds", "bpp_fp64_solves", "bpp_fp64_halfsteps"):
        assert s1[key] == s0[key], key
    if ill:
        assert s1["bpp_fp64_halfsteps"] > 0


def _nls_vs_oracle(nmf, G, B, X_gpu, P_gpu, passive_in):
    """One half-step's solves against the oracle's on the same (G, B) and
    starting partitions: relative error <= 20 cond(G) 6e-8; passive sets equal
    on right-hand sides with a clear KKT margin. Returns the oracle's rounds."""
    Xo, Po, Ro, So, wo = oracle.bpp(G, B, passive_in=passive_in)
    assert wo == 0
    cond = np.linalg.cond(G)
    err = rel(X_gpu, Xo)
    Y = Xo @ G - B
    Pb = Po.astype(bool)
    xm = np.where(Pb, Xo, np.inf).min(axis=1) / np.maximum(np.abs(Xo).max(axis=1), 1e-300)
    ym = np.where(~Pb, Y, np.inf).min(axis=1) / np.maximum(np.abs(B).max(axis=1), 1e-300)
    ok = np.minimum(xm, ym) >= 1e-3
    print(f"  cond {cond:.0f} rel err {err:.2e} ({err / (cond * 6e-8):.3f} x cond eps), "
          f"margin-clear {ok.mean():.2f}")
    assert err <= 20 * cond * 6e-8, (err, cond)
    assert ok.mean() > 0.2
    assert np.array_equal(P_gpu[ok], Pb[ok])
    return int(Ro.sum())


@pytest.mark.parametrize("k", [65, 100, 128])
def test_sparse_fused_products_k_above_64(nmf, k):
    # k > 64 runs the fused gather with four slots per lane. (1) Fused and
    # unfused runs give bitwise the same factors, objective history, passive
    # sets and round counts. (2) The run matches the oracle's ANLS within the
    # target tolerances. (3) One more iteration from the GPU's own iterate and
    # passive sets, each half-step against the oracle's solves of the same
    # problems (values, passive sets on margin-clear right-hand sides, and the
    # round total within 2%).
    m, n, T = 12000, 8000, 3
    csr = synth.csr_uniform(m, n, 160000, seed=29)
    W0, Ht0 = synth.init_factors(m, n, k, seed=29)
    outs = []
    for fused in (False, True):
        h = nmf.nmf_init(tuple(dev(x) for x in csr), dev(W0), dev(Ht0), shape=(m, n),
                         start="warm", fused_products=fused)
        h.nmf_iterate(T)
        assert h.nmf_sync() == nmf.NMF_OK
        W, Ht = h.nmf_get_factors()
        pW, pH = h.nmf_get_passive()
        st = h.nmf_get_stats()
        outs.append((W.cpu(), Ht.cpu(), np.array(h.nmf_objective_history()), pW.cpu(), pH.cpu(),
                     st))
        if fused:
            hf = h
        else:
            h.nmf_destroy()
    (Wa, Ha, fa, pWa, pHa, sa), (Wb, Hb, fb, pWb, pHb, sb) = outs
    assert torch.equal(Wa, Wb) and torch.equal(Ha, Hb) and np.array_equal(fa, fb)
    assert torch.equal(pWa, pWb) and torch.equal(pHa, pHb)
    for key in ("bpp_rhs", "bpp_rounds", "bpp_fp64_solves", "bpp_fp64_halfsteps"):
        assert sa[key] == sb[key], key
    assert sb["bpp_fp64_halfsteps"] == 0, sb
    ref = oracle.anls(None, W0, Ht0, iters=T, csr=csr, shape=(m, n), warm=True)
    g = dict(W=Wb.double().numpy(), Ht=Hb.double().numpy(), f=fb, status=nmf.NMF_OK, stats=sb)
    check(nmf, g, ref)
    # (3) iteration T + 1 of the fused handle, step by step against the oracle.
    W3, H3 = Wb.double().numpy(), Hb.double().numpy()
    P3w = nmf.passive_to_bool(pWb, k).numpy().astype(np.uint8)
    P3h = nmf.passive_to_bool(pHb, k).numpy().astype(np.uint8)
    hf.nmf_iterate(1)
    assert hf.nmf_sync() == nmf.NMF_OK
    W4, H4 = (x.double().cpu().numpy() for x in hf.nmf_get_factors())
    pW4, pH4 = (nmf.passive_to_bool(x, k).cpu().numpy() for x in hf.nmf_get_passive())
    s4 = hf.nmf_get_stats()
    hf.nmf_destroy()
    V = oracle.mm_csr(*csr, m, n, H3, False)
    rounds = _nls_vs_oracle(nmf, oracle.gram(H3), V, W4, pW4, P3w)
    Y = oracle.mm_csr(*csr, m, n, W4, True)
    rounds += _nls_vs_oracle(nmf, oracle.gram(W4), Y, H4, pH4, P3h)
    gpu_rounds = s4["bpp_rounds"] - sb["bpp_rounds"]
    print(f"k={k}: rounds gpu {gpu_rounds} oracle {rounds}")
    assert abs(gpu_rounds - rounds) <= 0.02 * rounds + 2


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_video_shape_crop(nmf, precision):
    # The tall-skinny shape of the paper's Video data set (1,013,400 x 2400,
    # Sec. 6.1): a 16384 x 2400 crop of the same recipe (A = W0 H0 + |N(0,
    # 0.05^2)|, k = 50), 10 iterations. With 19 output tiles of 128 rows, A^T W
    # splits its contraction over 8 CTAs per tile on the tensor-core path.
    m, n, k, T = 16384, 2400, 50, 10
    A = synth.dense_planted(m, n, k, 0.05, m_full=1013400, n_full=2400)
    W0, Ht0 = synth.init_factors(m, n, k)
    ref = oracle.anls(A, W0, Ht0, iters=T, warm=True)
    g = run_gpu(nmf, A, W0, Ht0, T, start="warm", precision=precision)
    if precision == "bf16x3":
        assert 8 <= g["stats"]["mm_splits_max"] <= 16, g["stats"]["mm_splits_max"]
    # The BF16x3 products' own noise over the 2400-long contraction of A H^T
    # moves the objective by ~1e-5 (as on the small configuration), so that
    # path's objective is held to 3e-5.
    check(nmf, g, ref, ftol=1e-5 if precision == "fp32" else 3e-5)


def test_checkpoint_resume(nmf):
    m, n, k = 600, 400, 8
    A = synth.dense_planted(m, n, k, 0.01, seed=5)
    W0, Ht0 = synth.init_factors(m, n, k, seed=5)
    h = nmf.nmf_init(dev(A), dev(W0), dev(Ht0))
    h.nmf_iterate(3)
    W3, H3 = h.nmf_get_factors()
    h.nmf_iterate(2)
    W5, H5 = h.nmf_get_factors()
    h2 = nmf.nmf_init(dev(A), W3.contiguous(), H3.contiguous())
    h2.nmf_iterate(2)
    W5b, H5b = h2.nmf_get_factors()
    assert torch.equal(W5, W5b) and torch.equal(H5, H5b)
    h.nmf_destroy()
    h2.nmf_destroy()


def test_invalid_config_raises(nmf):
    W0 = torch.zeros((10, 0), dtype=torch.float32, device="cuda")
    with pytest.raises(Exception):
        nmf.nmf_init(torch.zeros((10, 5), device="cuda"), W0,
                     torch.zeros((5, 0), dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_graph_mode_matches_eager(nmf, precision):
    # One CUDA graph per nmf_iterate call (captured on a non-default stream):
    # the same kernels in the same order, so the same bits as eager launches.
    import time
    m, n, k, T = 2000, 1000, 10, 10
    A = synth.dense_planted(m, n, k, 0.01)
    W0, Ht0 = synth.init_factors(m, n, k)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        e = run_gpu(nmf, A, W0, Ht0, T, precision=precision, start="warm", stream=s)
        g = run_gpu(nmf, A, W0, Ht0, T, precision=precision, start="warm", stream=s, graph=True)
    assert g["stats"]["graph_launches"] == 1 and e["stats"]["graph_launches"] == 0
    assert np.array_equal(g["f"], e["f"])
    assert np.array_equal(g["W"], e["W"]) and np.array_equal(g["Ht"], e["Ht"])
    # Launch-bound small problem: time 20 iterations either way (printed, not asserted).
    with torch.cuda.stream(s):
        for graph in (False, True):
            h = nmf.nmf_init(dev(A), dev(W0), dev(Ht0), precision=precision, start="warm",
                             stream=s)
            h.nmf_set_graph(graph)
            h.nmf_iterate(2)
            h.nmf_sync()
            t0 = time.perf_counter()
            h.nmf_iterate(20)
            h.nmf_sync()
            dt = (time.perf_counter() - t0) / 20
            print(f"{precision} graph={graph}: {1e3 * dt:.3f} ms per iteration")
            h.nmf_destroy()
