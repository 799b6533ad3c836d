"""Parity of each CUDA kernel with the FP64 oracle, called through the C ABI.

Tolerances (derived from the arithmetic; the oracle is FP64):
  * Gram: FP32 products summed in FP32 over 32-row tiles, tiles in FP64:
    |err| <= 2e-6 * (|X|^T |X|) elementwise.
  * Products (plain FP32): FP32 stage sums merged with Kahan
    compensation, so the result is near FP32 rounding:
    |err| <= 2e-6 * (|A| |F|) elementwise, and RMS relative error <= 2e-7.
  * BPP: FP32 factorisations of systems whose data (G and b rounded to FP32)
    already perturb x by ~cond(G) * 6e-8: ||x - x_or|| / ||x_or|| <= 200 * cond
    * 6e-8 per batch; passive sets and round counts identical on RHS whose
    KKT margin (O3) is at least 1e-3 of the problem scale.
  * Objective: residuals formed in FP32, squares summed in FP64: rel 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def nmf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_09313_gb300 as lib
    return lib


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ----------------------------------------------------------------------------- Gram
@pytest.mark.parametrize("k", [1, 7, 10, 16, 17, 33, 50, 64, 65, 100, 128])
@pytest.mark.parametrize("rows", [0, 1, 31, 33, 1000, 4099])
def test_gram(nmf, k, rows):
    rng = np.random.default_rng(k * 1000 + rows)
    X = rng.uniform(-1, 1, (rows, k)).astype(np.float32)
    G = nmf.nmf_gram(dev(X)).cpu().numpy()
    ref = oracle.gram(X.astype(np.float64))
    bound = 2e-6 * oracle.gram(np.abs(X).astype(np.float64)) + 1e-30
    assert np.all(np.abs(G - ref) <= bound)
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("k", [1, 7, 16, 33, 50, 64])
@pytest.mark.parametrize("signed", [False, True])
def test_gram_tensor_cores(nmf, k, signed):
    # Rows past 128 per SM take the tensor-core Gram (BF16 three-way splits,
    # h^T h drained per 128-row tile into compensated sums): the same bound as
    # the SIMT Gram's, a ragged last tile, and a view that is not 16-byte
    # aligned (the SIMT path) giving the same answer within that bound.
    rows = 128 * torch.cuda.get_device_properties(0).multi_processor_count * 2 + 77
    rng = np.random.default_rng(70 + k)
    lo = -1.0 if signed else 0.0
    X = rng.uniform(lo, 1.0, (rows, k)).astype(np.float32)
    ref = oracle.gram(X.astype(np.float64))
    bound = 2e-6 * oracle.gram(np.abs(X).astype(np.float64)) + 1e-30
    G = nmf.nmf_gram(dev(X)).cpu().numpy()
    err = np.abs(G - ref) / bound
    print(f"k={k} signed={signed}: max err / bound {err.max():.3f}")
    assert np.all(np.abs(G - ref) <= bound)
    assert np.array_equal(G, G.T)
    buf = torch.empty(rows * k + 1, dtype=torch.float32, device="cuda")
    buf[1:] = dev(X).reshape(-1)
    Gs = nmf.nmf_gram(buf[1:].view(rows, k)).cpu().numpy()
    assert np.all(np.abs(Gs - ref) <= bound)


# ----------------------------------------------------------------------------- products
# Rows of A that are a multiple of 4 floats take the packed-FMA kernels (ragged
# tiles, contraction splits of A^T W on the tall shapes); the others the
# scalar-load kernel.
@pytest.mark.parametrize("shape", [(1, 1), (37, 23), (129, 257), (300, 1000), (1000, 300),
                                   (2050, 17), (37, 24), (129, 260), (2050, 20), (8192, 40),
                                   (40, 8192)])
@pytest.mark.parametrize("k", [1, 5, 10, 16, 17, 50, 64, 100, 128])
@pytest.mark.parametrize("trans", [0, 1])
def test_mm_dense_fp32(nmf, shape, k, trans):
    m, n = shape
    rng = np.random.default_rng(m * 7 + n * 13 + k + trans)
    A = rng.uniform(0, 1, (m, n)).astype(np.float32)
    F = rng.uniform(0, 1, (n if trans == 0 else m, k)).astype(np.float32)
    out = nmf.nmf_mm_dense(dev(A), dev(F), bool(trans)).cpu().numpy().astype(np.float64)
    ref = oracle.mm_dense(A, F.astype(np.float64), bool(trans))
    assert out.shape == ref.shape
    assert np.all(np.abs(out - ref) <= 2e-6 * ref + 1e-30)
    rel = (out - ref) / np.where(ref == 0, 1, ref)
    assert np.sqrt(np.mean(rel ** 2)) <= 2e-7


@pytest.mark.parametrize("shape", [(1, 4), (37, 24), (129, 256), (300, 1000), (1000, 300),
                                   (2050, 20), (4099, 132), (512, 8192), (8192, 512)])
@pytest.mark.parametrize("k", [1, 10, 16, 17, 33, 50, 64, 100, 128])
@pytest.mark.parametrize("trans", [0, 1])
def test_mm_dense_bf16x3(nmf, shape, k, trans):
    # Tensor-core path: each product carries a relative error <= 2^-16 from
    # the head/tail split (|err| <= 2e-5 (|A||F|) elementwise, random sign, so
    # ~2^-17 / sqrt(terms) RMS); the tensor cores' truncating accumulation adds
    # a bias of about half an ulp per MMA into an accumulator, bounded by the
    # one-K-block drain of the head products to ~2e-7.
    m, n = shape
    rng = np.random.default_rng(m * 3 + n * 11 + k + 7 * trans)
    A = rng.uniform(0, 1, (m, n)).astype(np.float32)
    F = rng.uniform(0, 1, (n if trans == 0 else m, k)).astype(np.float32)
    out = nmf.nmf_mm_dense(dev(A), dev(F), bool(trans), precision="bf16x3")
    out = out.cpu().numpy().astype(np.float64)
    ref = oracle.mm_dense(A, F.astype(np.float64), bool(trans))
    assert np.all(np.abs(out - ref) <= 2e-5 * ref + 1e-30)
    rel = (out - ref) / np.where(ref == 0, 1, ref)
    q = m if trans else n
    assert np.sqrt(np.mean(rel ** 2)) <= 1.2e-5 / np.sqrt(q) + 2e-7


def test_mm_dense_bf16x3_needs_aligned_rows(nmf):
    # The tensor-core path reads A with TMA: rows must start on 16 bytes.
    A = torch.zeros((16, 17), dtype=torch.float32, device="cuda")
    F = torch.zeros((17, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(nmf.NMFError):
        nmf.nmf_mm_dense(A, F, False, precision="bf16x3")


@pytest.mark.parametrize("pad", [2, 3])
@pytest.mark.parametrize("trans", [0, 1])
def test_mm_dense_strided_and_signed(nmf, trans, pad):
    # Leading dimension n + pad > n, signed data: 519 floats (not a multiple
    # of 4: scalar-load kernel) or 520 (packed-FMA kernels).
    m, n, k = 333, 517, 50
    rng = np.random.default_rng(5 + pad)
    Afull = rng.uniform(-1, 1, (m, n + pad)).astype(np.float32)
    F = rng.uniform(-1, 1, (n if trans == 0 else m, k)).astype(np.float32)
    Ad = dev(Afull)[:, :n]
    out = nmf.nmf_mm_dense(Ad, dev(F), bool(trans)).cpu().numpy().astype(np.float64)
    A = np.ascontiguousarray(Afull[:, :n])
    ref = oracle.mm_dense(A, F.astype(np.float64), bool(trans))
    bound = 2e-6 * oracle.mm_dense(np.abs(A), np.abs(F).astype(np.float64), bool(trans))
    assert np.all(np.abs(out - ref) <= bound + 1e-30)


def test_mm_dense_zero_contraction(nmf):
    A = torch.empty((5, 0), dtype=torch.float32, device="cuda")
    F = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    out = nmf.nmf_mm_dense(A, F, False)
    assert out.shape == (5, 3) and torch.all(out == 0)


# ----------------------------------------------------------------------------- sparse
@pytest.mark.parametrize("k", [1, 10, 50, 100])
def test_spmm_and_transpose(nmf, k):
    m, n = 3001, 1777
    rowptr, colidx, vals = synth.csr_uniform(m, n, 40000, seed=k)
    rowptr[5:] += 0   # rows 0..m-1 include empty rows at this density
    d_rp, d_ci, d_v = dev(rowptr), dev(colidx), dev(vals)
    rng = np.random.default_rng(k)
    Ht = rng.uniform(0, 1, (n, k)).astype(np.float32)
    W = rng.uniform(0, 1, (m, k)).astype(np.float32)
    V = nmf.nmf_mm_csr(d_rp, d_ci, d_v, n, dev(Ht)).cpu().numpy().astype(np.float64)
    refV = oracle.mm_csr(rowptr, colidx, vals, m, n, Ht.astype(np.float64), False)
    assert np.all(np.abs(V - refV) <= 2e-6 * refV + 1e-30)
    t_rp, t_ci, t_v = nmf.nmf_csr_transpose(d_rp, d_ci, d_v, m, n)
    # Expected transpose, built with numpy: stable sort by (column, row).
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    order = np.lexsort((rows, colidx))
    exp_ci = rows[order].astype(np.int32)
    exp_v = vals[order]
    exp_rp = np.concatenate([[0], np.cumsum(np.bincount(colidx, minlength=n))])
    assert np.array_equal(t_rp.cpu().numpy(), exp_rp)
    assert np.array_equal(t_ci.cpu().numpy(), exp_ci)
    assert np.array_equal(t_v.cpu().numpy(), exp_v)
    Y = nmf.nmf_mm_csr(t_rp, t_ci, t_v, m, dev(W)).cpu().numpy().astype(np.float64)
    refY = oracle.mm_csr(rowptr, colidx, vals, m, n, W.astype(np.float64), True)
    assert np.all(np.abs(Y - refY) <= 2e-6 * refY + 1e-30)


# ----------------------------------------------------------------------------- BPP
def margin_ok(G, B, X, P, rel=1e-3):
    """RHS whose KKT margin is safely away from zero: every passive x_i is at
    least rel * max|x| and every active y_i at least rel * max|b|."""
    Y = X @ G - B
    xm = np.where(P, X, np.inf).min(axis=1) / np.maximum(np.abs(X).max(axis=1), 1e-300)
    ym = np.where(~P, Y, np.inf).min(axis=1) / np.maximum(np.abs(B).max(axis=1), 1e-300)
    return np.minimum(xm, ym) >= rel


def run_bpp(nmf, G, B32, passive_in=None, max_rounds=100):
    r = nmf.nmf_nls_bpp(dev(G), dev(B32), None if passive_in is None else dev(passive_in),
                        max_rounds=max_rounds)
    k = G.shape[0]
    return (r["X"].cpu().numpy().astype(np.float64),
            nmf.passive_to_bool(r["passive"], k).cpu().numpy(),
            r["rounds"].cpu().numpy(), r["status"].cpu().numpy(), r["worst"])


@pytest.mark.parametrize("k", [1, 2, 5, 10, 20, 32, 33, 50, 64, 65, 100, 128])
def test_bpp_matches_oracle(nmf, k):
    nrhs = 3000 if k <= 64 else 800
    G, B = synth.nls_batch(k, nrhs, seed=100 + k)
    B32 = B.astype(np.float32)
    Bd = B32.astype(np.float64)
    X, P, R, S, worst = run_bpp(nmf, G, B32)
    Xo, Po, Ro, So, wo = oracle.bpp(G, Bd)
    assert worst == nmf.NMF_OK and (S == 0).all()
    cond = np.linalg.cond(G)
    err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    print(f"k={k} cond={cond:.0f} rel err {err:.2e} ({err / (cond * 6e-8):.3f} x cond*eps)")
    assert err <= 20 * cond * 6e-8, (err, cond)
    assert (X >= 0).all()
    ok = margin_ok(G, Bd, Xo, Po.astype(bool))
    assert ok.mean() > 0.4
    assert np.array_equal(P[ok], Po.astype(bool)[ok])
    # Round counts follow the same exchange rules; an intermediate partition can
    # still flip on a near-zero FP32 value, so allow a small fraction to differ.
    assert (R[ok] == Ro[ok]).mean() >= 0.98
    assert (X[~P] == 0).all()


@pytest.mark.parametrize("k", [10, 50])
def test_bpp_anls_like(nmf, k):
    # The W-update of Alg. 1 from a uniform start: G = H H^T of a positive H
    # (one dominant eigenvalue, so G^{-1} has large entries of mixed sign) and
    # right-hand sides A H^T. Every solve must converge and match the oracle.
    m, n = 4000, 1000
    A = synth.dense_planted(m, n, k, 0.05, seed=k)
    _, Ht = synth.init_factors(m, n, k, seed=k + 1)
    G = oracle.gram(Ht.astype(np.float64))
    B32 = oracle.mm_dense(A, Ht.astype(np.float64), False).astype(np.float32)
    X, P, R, S, worst = run_bpp(nmf, G, B32)
    Xo, Po, Ro, So, wo = oracle.bpp(G, B32.astype(np.float64))
    assert worst == nmf.NMF_OK and (S == 0).all(), np.bincount(S.astype(np.int64))
    cond = np.linalg.cond(G)
    err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    print(f"k={k} cond={cond:.0f} rel err {err:.2e} max rounds {R.max()} vs {Ro.max()}")
    assert err <= 20 * cond * 6e-8
    ok = margin_ok(G, B32.astype(np.float64), Xo, Po.astype(bool))
    assert np.array_equal(P[ok], Po.astype(bool)[ok])


def test_bpp_warm_start(nmf):
    k, nrhs = 50, 2000
    G, B = synth.nls_batch(k, nrhs, seed=77)
    B32 = B.astype(np.float32)
    Xo, Po, Ro, So, wo = oracle.bpp(G, B32.astype(np.float64))
    words = nmf.bool_to_passive(torch.from_numpy(Po.astype(bool))).numpy()
    X, P, R, S, worst = run_bpp(nmf, G, B32, passive_in=words)
    ok = margin_ok(G, B32.astype(np.float64), Xo, Po.astype(bool))
    assert (R[ok] == 0).all()
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-4
    # Warm start from a perturbed partition reaches the same point.
    Pp = Po.astype(bool).copy()
    Pp[:, ::4] = ~Pp[:, ::4]
    X2, P2, R2, S2, w2 = run_bpp(nmf, G, B32,
                                 passive_in=nmf.bool_to_passive(torch.from_numpy(Pp)).numpy())
    assert w2 == nmf.NMF_OK
    assert np.linalg.norm(X2 - Xo) / np.linalg.norm(Xo) <= 1e-4


def test_bpp_round_cap_and_nonfinite(nmf):
    k, nrhs = 20, 300
    G, B = synth.nls_batch(k, nrhs, seed=9)
    B32 = B.astype(np.float32)
    X, P, R, S, worst = run_bpp(nmf, G, B32, max_rounds=0)
    assert worst == nmf.NMF_ERR_NOT_CONVERGED
    assert set(np.unique(S)) <= {0, nmf.NMF_ERR_NOT_CONVERGED}
    B32[7, 3] = np.nan
    X, P, R, S, worst = run_bpp(nmf, G, B32)
    assert S[7] == nmf.NMF_ERR_NONFINITE and (X[7] == 0).all()
    others = np.delete(np.arange(nrhs), 7)
    assert (S[others] == 0).all() and worst == nmf.NMF_ERR_NONFINITE


def test_bpp_zero_diagonal(nmf):
    # A zero row of the factor: G_ii = 0 and b_i = 0; index stays active.
    k, nrhs = 12, 400
    G, B = synth.nls_batch(k, nrhs, seed=21)
    G[4, :] = 0.0
    G[:, 4] = 0.0
    B[:, 4] = 0.0
    B32 = B.astype(np.float32)
    X, P, R, S, worst = run_bpp(nmf, G, B32)
    Xo = oracle.bpp(G, B32.astype(np.float64))[0]
    assert worst == nmf.NMF_OK and (X[:, 4] == 0).all()
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-4


def test_bpp_ill_conditioned_fp64(nmf):
    # cond(G) ~ 3e8: FP32 cannot resolve these systems, so the whole half-step
    # runs in FP64 (cond_1(G) > 1e4) with the strict sign tests of the oracle.
    k, nrhs = 24, 500
    G, B = synth.nls_batch(k, nrhs, seed=31, cond_boost=1000.0)
    assert np.linalg.cond(G) > 1e8
    B32 = B.astype(np.float32)
    Bd = B32.astype(np.float64)
    X, P, R, S, worst = run_bpp(nmf, G, B32)
    Xo, Po, Ro, So, wo = oracle.bpp(G, Bd)
    assert worst == nmf.NMF_OK and (S == 0).all()
    err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    assert err <= 1e-6, err
    ok = margin_ok(G, Bd, Xo, Po.astype(bool))
    assert np.array_equal(P[ok], Po.astype(bool)[ok])


def test_bpp_fp64_predicted_start_same_answer(nmf):
    # FP64 half-steps start from FP32-predicted partitions when the round cap
    # allows (>= 16). The answer is the unique minimiser either way, and the
    # final FP64 solve depends only on the final partition: bitwise the same X
    # and passive sets, in far fewer FP64 rounds.
    k, nrhs = 24, 2000
    G, B = synth.nls_batch(k, nrhs, seed=31, cond_boost=1000.0)
    B32 = B.astype(np.float32)
    X1, P1, R1, S1, w1 = run_bpp(nmf, G, B32, max_rounds=100)   # predictor on
    X2, P2, R2, S2, w2 = run_bpp(nmf, G, B32, max_rounds=15)    # predictor off
    assert w1 == nmf.NMF_OK and w2 == nmf.NMF_OK
    assert np.array_equal(X1, X2) and np.array_equal(P1, P2)
    # (At cond ~3e8 FP32 resolves little, so the saving here is small; on the
    # dense workload's FP64 half-steps, cond 1e4-1e6, rounds fall ~50-fold.)
    print(f"FP64 rounds per solve: predicted start {R1.mean():.3f}, cold {R2.mean():.3f}")
    assert R1.mean() <= R2.mean()


def test_bpp_singular_gram(nmf):
    # Two identical factor rows: G is singular even in FP64, so no inverse is
    # formed and every system is solved directly in FP64. Solves whose passive
    # set holds both copies are singular; the rest must satisfy Eq. 4.
    k, nrhs = 16, 400
    rng = np.random.default_rng(8)
    C = rng.uniform(0, 1, (64, k))
    C[:, 5] = C[:, 9]
    G = C.T @ C
    D = rng.uniform(-0.5, 1.0, (nrhs, 64))
    B32 = (D @ C).astype(np.float32)
    X, P, R, S, worst = run_bpp(nmf, G, B32)
    assert set(np.unique(S)) <= {0, nmf.NMF_ERR_SINGULAR_GRAM}
    good = S == 0
    Bd = B32.astype(np.float64)
    Y = X @ G - Bd
    scale = np.abs(Bd).max(axis=1)
    assert (X[good] >= 0).all()
    assert (Y[good] >= -1e-9 * scale[good, None]).all()
    comp = np.abs((X * Y)[good]).sum(axis=1)
    assert (comp <= 1e-9 * (scale[good] * np.abs(X[good]).max(axis=1) + 1e-30)).all()


class shape_of:
    """Sets the launch shape of solves of k inside a with-block, then restores it."""

    def __init__(self, nmf, k, warps, chunk, group):
        self.nmf, self.k, self.new = nmf, k, (warps, chunk, group)

    def __enter__(self):
        self.old = self.nmf.nmf_nls_bpp_get_shape(self.k)
        self.nmf.nmf_nls_bpp_set_shape(self.k, *self.new)

    def __exit__(self, *exc):
        self.nmf.nmf_nls_bpp_set_shape(self.k, *self.old)


def group_cases(k):
    """Batches that reach every branch of the group-tile pass: all solutions
    positive (every right-hand side in the all-passive group, cold and warm),
    non-negative right-hand sides with mixed signs in the solution (in the
    group, then left to the per-warp solves), signed right-hand sides (few in
    the group), non-finite rows, round caps 0 and 1, a zero diagonal (an
    unusable index) and an FP64 half-step (the pass stays off)."""
    nrhs = 1237                                   # not a multiple of the 32- or 64-wide tiles
    rng = np.random.default_rng(900 + k)
    G, _ = synth.nls_batch(k, 1, seed=800 + k)
    Xt = rng.uniform(0.1, 1.0, (nrhs, k))
    Bpos = (Xt @ G).astype(np.float32)
    _, Bu = synth.nls_batch(k, nrhs, seed=800 + k, signed_rhs=False)
    _, Bs = synth.nls_batch(k, nrhs, seed=800 + k)
    nanB = Bpos.copy()
    nanB[[0, 5, 64, 1236], min(3, k - 1)] = np.nan
    all_in = np.ones((nrhs, k), bool)
    part = all_in.copy()
    part[::3, 0] = False
    Gz = G.copy()
    z = min(2, k - 1)
    Gz[z, :] = 0.0
    Gz[:, z] = 0.0
    Bz = Bpos.copy()
    Bz[:, z] = 0.0
    Gi, Bi = synth.nls_batch(k, nrhs, seed=700 + k, cond_boost=1000.0)
    cases = [("positive", G, Bpos, None, 100), ("positive-warm", G, Bpos, all_in, 100),
             ("warm-partial", G, Bpos, part, 100), ("unsigned", G, Bu.astype(np.float32), None, 100),
             ("signed", G, Bs.astype(np.float32), None, 100), ("nonfinite", G, nanB, None, 100),
             ("cap0", G, Bpos, None, 0), ("cap1", G, Bu.astype(np.float32), None, 1),
             ("fp64", Gi, Bi.astype(np.float32), None, 100)]
    if k > 1:
        cases.append(("zero-diagonal", Gz, Bz, None, 100))
    return cases


@pytest.mark.parametrize("k", [1, 5, 10, 33, 50, 64, 65, 100, 128])
def test_bpp_group_pass_bitwise_equal(nmf, k):
    # The SIMT group-tile pass (launch shape group = 1) forms each entry with
    # the same operations in the same order as the per-warp kernel: the same X
    # bits, passive sets, rounds and statuses with the pass on or off, on every
    # path.
    for name, G, B32, warm, cap in group_cases(k):
        pin = None if warm is None else nmf.bool_to_passive(torch.from_numpy(warm)).numpy()
        outs = []
        for group in (0, 1):
            with shape_of(nmf, k, 8, 8, group):
                outs.append(run_bpp(nmf, G, B32, passive_in=pin, max_rounds=cap))
        (X0, P0, R0, S0, w0), (X1, P1, R1, S1, w1) = outs
        print(f"k={k} {name}: statuses {np.bincount(S0.astype(np.int64))} rounds {R0.mean():.2f}")
        assert np.array_equal(X1, X0, equal_nan=True), name
        assert np.array_equal(P1, P0) and np.array_equal(R1, R0), name
        assert np.array_equal(S1, S0) and w1 == w0, name
        if name == "positive":   # every solve in the group: one full exchange, all passive
            assert (R1 == 1).all() and (S1 == 0).all() and P1.all()


@pytest.mark.parametrize("k", [1, 5, 10, 33, 50, 64, 65, 100, 112])
def test_bpp_group_pass_tensor_cores(nmf, k):
    # The tensor-core group pass (launch shape group = 2) forms the all-passive
    # group's products from BF16 splits (G three-way): not the bits of the
    # per-warp kernel, but FP32 solve accuracy. On every branch of the pass:
    # values within the FP32 bound of the FP64 oracle, passive sets and round
    # counts equal on right-hand sides with a clear KKT margin, and statuses
    # equal to the per-warp kernel's (pass off) on those.
    for name, G, B32, warm, cap in group_cases(k):
        pin = None if warm is None else nmf.bool_to_passive(torch.from_numpy(warm)).numpy()
        with shape_of(nmf, k, 8, 8, 0):
            X0, P0, R0, S0, w0 = run_bpp(nmf, G, B32, passive_in=pin, max_rounds=cap)
        with shape_of(nmf, k, 8, 8, 2):
            X2, P2, R2, S2, w2 = run_bpp(nmf, G, B32, passive_in=pin, max_rounds=cap)
        Bd = B32.astype(np.float64)
        Xo, Po, Ro, So, wo = oracle.bpp(G, Bd, None if warm is None else warm.astype(np.uint8),
                                        max_rounds=cap)
        fin = np.isfinite(Bd).all(axis=1) & (So == 0)
        ok = margin_ok(G, Bd[fin], Xo[fin], Po[fin].astype(bool))
        cond = np.linalg.cond(G[np.ix_(np.diag(G) > 0, np.diag(G) > 0)])
        err = np.linalg.norm(X2[fin] - Xo[fin]) / max(np.linalg.norm(Xo[fin]), 1e-300)
        print(f"k={k} {name}: rel err {err:.2e} (bound {20 * cond * 6e-8:.1e}), "
              f"margin-clear {ok.mean() if ok.size else 0:.2f}, rounds {R2.mean():.2f}")
        assert err <= 20 * cond * 6e-8, name
        if name == "fp64" and cond > 1e5:
            # An FP64 half-step (its solves start from FP32-predicted
            # partitions, so their round counts are not the oracle's): the pass
            # stays off and the results are those of the pass-off run.
            assert np.array_equal(X2, X0) and np.array_equal(R2, R0) and np.array_equal(S2, S0)
            continue
        assert np.array_equal(P2[fin][ok], Po[fin][ok].astype(bool)), name
        if ok.any():
            assert (R2[fin][ok] == Ro[fin][ok]).mean() >= 0.98, name
        assert np.array_equal(S2[fin][ok], S0[fin][ok]), name
        assert np.array_equal(S2[~fin] != 0, S0[~fin] != 0), name
        assert (X2[fin] >= 0).all() and (X2[fin][~P2[fin]] == 0).all(), name
        if name == "positive":   # every solve in the group: one full exchange, all passive
            assert (R2 == 1).all() and (S2 == 0).all() and P2.all()


def test_bpp_group_pass_matches_oracle(nmf):
    # Positive solutions from a cold start: the group-tile pass solves every
    # right-hand side; compare with the FP64 oracle.
    k, nrhs = 40, 3000
    rng = np.random.default_rng(5)
    G, _ = synth.nls_batch(k, 1, seed=41)
    B32 = (rng.uniform(0.1, 1.0, (nrhs, k)) @ G).astype(np.float32)
    X, P, R, S, worst = run_bpp(nmf, G, B32)
    Xo, Po, Ro, So, wo = oracle.bpp(G, B32.astype(np.float64))
    assert worst == nmf.NMF_OK and (R == Ro).all() and np.array_equal(P, Po.astype(bool))
    err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    assert err <= 20 * np.linalg.cond(G) * 6e-8, err


def test_bpp_empty_batch(nmf):
    G, B = synth.nls_batch(10, 1, seed=1)
    r = nmf.nmf_nls_bpp(dev(G), torch.empty((0, 10), dtype=torch.float32, device="cuda"))
    assert r["worst"] == nmf.NMF_OK and r["X"].shape == (0, 10)


# ----------------------------------------------------------------------------- objective
@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("shape,k", [((37, 24), 3), ((300, 1000), 10), ((1000, 300), 50),
                                     ((129, 68), 100), ((4100, 2048), 64)])
def test_objective_dense(nmf, shape, k, precision):
    m, n = shape
    A = synth.dense_planted(m, n, k, 0.05, seed=m + n)
    rng = np.random.default_rng(3)
    W = rng.uniform(0, 1, (m, k)).astype(np.float32)
    Ht = rng.uniform(0, 1, (n, k)).astype(np.float32)
    f = nmf.nmf_objective_dense(dev(A), dev(W), dev(Ht), precision=precision)
    ref = oracle.objective_dense(A, W, Ht)
    assert abs(f - ref) <= 1e-5 * ref


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_objective_dense_good_fit(nmf, precision):
    # W, H near the planted factors: the residual is ~1e-3 of A, so the sum is
    # sensitive to any bias in W H.
    m, n, k = 2000, 1024, 16
    A, W0, H0 = synth.dense_planted(m, n, k, 0.05, seed=4, return_factors=True)
    W = W0.astype(np.float32)
    Ht = np.ascontiguousarray(H0.T).astype(np.float32)
    f = nmf.nmf_objective_dense(dev(A), dev(W), dev(Ht), precision=precision)
    ref = oracle.objective_dense(A, W, Ht)
    assert abs(f - ref) <= 1e-5 * ref, (f, ref)
