"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError on
a mismatch. They are called by the oracle tests, and again on deliberately
broken builds of the oracle (tests/test_oracle_mutations.py) to show that a
plausible mistake anywhere in it fails at least one pin.

None of these checks reuses the oracle's own arithmetic: the expected values
come from hand-worked examples, brute force over all partitions, scipy's
Lawson-Hanson NNLS, numpy products, closed forms, or invariants.
"""
from __future__ import annotations

import itertools
import os
from fractions import Fraction

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "nls_hand.txt")


def _numbers(text):
    """Whitespace-separated numbers; exact fractions such as 107/173 allowed."""
    return np.array([float(Fraction(t)) for t in text.split()], dtype=np.float64)


def load_golden():
    cases = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, k, G, g, x, y, rounds = [t.strip() for t in line.split("|")]
            k = int(k)
            cases.append(dict(name=name, k=k, G=_numbers(G).reshape(k, k), g=_numbers(g),
                              x=_numbers(x), y=_numbers(y), rounds=int(rounds)))
    return cases


def kkt_residuals(G, B, X):
    """Eq. 4 residuals per RHS, scaled: (min x, min y, |x.y|) relative to the
    problem's size scale max(|g|_inf, max diag G * |x|_inf)."""
    Y = X @ G.T - B
    scale = np.maximum(np.abs(B).max(axis=1), np.abs(np.diag(G)).max() * np.abs(X).max(axis=1))
    scale = np.maximum(scale, 1e-300)
    neg_x = np.minimum(X.min(axis=1), 0.0) / np.maximum(np.abs(X).max(axis=1), 1e-300)
    neg_y = np.minimum(Y.min(axis=1), 0.0) / scale
    comp = np.abs((X * Y).sum(axis=1)) / (scale * np.maximum(np.abs(X).max(axis=1), 1e-300))
    return neg_x, neg_y, comp


def brute_force_nls(G, g, tol=1e-10):
    """All 2^k partitions; keep those whose restricted normal-equations
    solution satisfies Eq. 4. Returns the list of KKT points."""
    k = len(g)
    scale = max(np.abs(g).max(), 1e-300)
    sols = []
    for mask in itertools.product([0, 1], repeat=k):
        F = np.array(mask, dtype=bool)
        x = np.zeros(k)
        if F.any():
            x[F] = np.linalg.solve(G[np.ix_(F, F)], g[F])
        y = G @ x - g
        if (x >= -tol * max(np.abs(x).max(), 1.0)).all() and (y[~F] >= -tol * scale).all():
            sols.append(x)
    return sols


def pin_golden(orc):
    for c in load_golden():
        X, P, R, S, worst = orc.bpp(c["G"], c["g"][None, :])
        assert worst == 0, c["name"]
        np.testing.assert_allclose(X[0], c["x"], rtol=0, atol=1e-14, err_msg=c["name"])
        y = c["G"] @ X[0] - c["g"]
        np.testing.assert_allclose(y, c["y"], rtol=0, atol=1e-14, err_msg=c["name"])
        assert int(R[0]) == c["rounds"], (c["name"], int(R[0]), c["rounds"])
        np.testing.assert_array_equal(P[0].astype(bool), c["x"] > 0, err_msg=c["name"])


def pin_bruteforce(orc, ks=(1, 2, 3, 5, 8), nrhs=40, seed=7):
    for k in ks:
        G, B = synth.nls_batch(k, nrhs, seed=seed + k)
        X, P, R, S, worst = orc.bpp(G, B)
        assert worst == 0
        for j in range(nrhs):
            sols = brute_force_nls(G, B[j])
            assert len(sols) >= 1
            for s in sols:
                np.testing.assert_allclose(X[j], s, rtol=1e-12, atol=1e-12 * np.abs(s).max())


def pin_nnls(orc, ks=(10, 20, 50), nrhs=30, seed=11):
    from scipy.linalg import cholesky, solve_triangular
    from scipy.optimize import nnls
    for k in ks:
        G, B = synth.nls_batch(k, nrhs, seed=seed + k)
        X, P, R, S, worst = orc.bpp(G, B)
        assert worst == 0
        L = cholesky(G, lower=True)
        for j in range(nrhs):
            # 0.5 x^T G x - g^T x = 0.5 ||L^T x - L^{-1} g||^2 - const
            b = solve_triangular(L, B[j], lower=True)
            xs, _ = nnls(L.T, b, maxiter=50 * k)
            np.testing.assert_allclose(X[j], xs, rtol=1e-9, atol=1e-9 * np.abs(xs).max())


def pin_closed_forms(orc, seed=5):
    rng = np.random.default_rng(seed)
    # k = 1: x = max(0, g / G).
    g = rng.uniform(-2, 2, 50)
    X, P, R, S, w = orc.bpp(np.array([[2.5]]), g[:, None])
    np.testing.assert_allclose(X[:, 0], np.maximum(0.0, g / 2.5), rtol=1e-15, atol=0)
    # Diagonal G: x_i = max(0, g_i / G_ii).
    d = rng.uniform(0.5, 3.0, 12)
    Bd = rng.uniform(-1, 1, (20, 12))
    X, P, R, S, w = orc.bpp(np.diag(d), Bd)
    np.testing.assert_allclose(X, np.maximum(0.0, Bd / d), rtol=1e-15, atol=0)
    # g <= 0 everywhere: x = 0, zero exchange rounds.
    G, B = synth.nls_batch(9, 10, seed=seed)
    Bn = -np.abs(B)
    X, P, R, S, w = orc.bpp(G, Bn)
    assert (X == 0).all() and (R == 0).all() and not P.any()
    # G^{-1} g > 0 with g > 0: one full exchange to the full passive set.
    xs = rng.uniform(0.5, 1.5, (10, 9))
    Bp = xs @ G  # G symmetric: g = G x*
    X, P, R, S, w = orc.bpp(G, Bp)
    np.testing.assert_allclose(X, xs, rtol=1e-10)
    assert (R == 1).all() and P.all()


def pin_kkt_and_warm(orc, seed=3):
    for k, nrhs in ((7, 300), (30, 200), (64, 100)):
        G, B = synth.nls_batch(k, nrhs, seed=seed + k)
        X, P, R, S, w = orc.bpp(G, B)
        assert w == 0
        nx, ny, comp = kkt_residuals(G, B, X)
        assert (nx >= -1e-14).all() and (ny >= -1e-12).all() and (comp <= 1e-12).all()
        np.testing.assert_array_equal(P.astype(bool), X > 0)
        # Warm start from the answer: zero rounds, same point.
        X2, P2, R2, S2, w2 = orc.bpp(G, B, passive_in=P)
        assert (R2 == 0).all()
        np.testing.assert_allclose(X2, X, rtol=1e-12, atol=1e-14)
        # Warm start from a perturbed set: same unique point.
        Pp = P.copy()
        Pp[:, ::3] ^= 1
        X3, P3, R3, S3, w3 = orc.bpp(G, B, passive_in=Pp)
        assert w3 == 0
        np.testing.assert_allclose(X3, X, rtol=1e-10, atol=1e-12 * np.abs(X).max())


def pin_products(orc, seed=2):
    rng = np.random.default_rng(seed)
    m, n, k = 37, 23, 5
    A = rng.uniform(0, 1, (m, n)).astype(np.float32)
    Ad = A.astype(np.float64)
    Ht = rng.uniform(0, 1, (n, k))
    W = rng.uniform(0, 1, (m, k))
    np.testing.assert_allclose(orc.mm_dense(A, Ht, False), Ad @ Ht, rtol=1e-13)
    np.testing.assert_allclose(orc.mm_dense(A, W, True), Ad.T @ W, rtol=1e-13)
    np.testing.assert_allclose(orc.gram(Ht), Ht.T @ Ht, rtol=1e-13)
    np.testing.assert_allclose(orc.gram(W), W.T @ W, rtol=1e-13)
    f = np.sum((Ad - W @ Ht.T) ** 2)
    np.testing.assert_allclose(orc.objective_dense(A, W, Ht), f, rtol=1e-12)
    # Sparse: compare with the dense routines on the same matrix.
    rowptr, colidx, vals = synth.csr_uniform(m, n, 150, seed=seed)
    D = synth.csr_to_dense(rowptr, colidx, vals, m, n).astype(np.float64)
    np.testing.assert_allclose(orc.mm_csr(rowptr, colidx, vals, m, n, Ht, False), D @ Ht,
                               rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(orc.mm_csr(rowptr, colidx, vals, m, n, W, True), D.T @ W,
                               rtol=1e-13, atol=1e-15)
    fs = np.sum((D - W @ Ht.T) ** 2)
    np.testing.assert_allclose(orc.objective_csr(rowptr, colidx, vals, m, n, W, Ht), fs,
                               rtol=1e-11)


def halfstep_kkt(A, H_t, W_new, tol):
    """W_new must minimise ||A - W H|| over W >= 0 for fixed H (Eq. 2, first
    line): gradient R = W (H H^T) - A H^T satisfies Eq. 4 row by row."""
    R = W_new @ (H_t.T @ H_t) - A @ H_t
    scale = np.abs(A @ H_t).max()
    assert W_new.min() >= 0.0
    assert R.min() >= -tol * scale, R.min() / scale
    assert np.abs(W_new * R).max() <= tol * scale * max(np.abs(W_new).max(), 1.0)


def pin_anls(orc, seed=9):
    m, n, k = 80, 50, 6
    A = synth.dense_planted(m, n, k, 0.05, seed=seed)
    W0, Ht0 = synth.init_factors(m, n, k, seed=seed)
    r1 = orc.anls(A, W0, Ht0, iters=1)
    Ad = A.astype(np.float64)
    halfstep_kkt(Ad, Ht0.astype(np.float64), r1["W"], 1e-10)
    halfstep_kkt(Ad.T, r1["W"], r1["Ht"], 1e-10)
    r = orc.anls(A, W0, Ht0, iters=15)
    f = r["f"]
    assert (f[1:] <= f[:-1] * (1 + 1e-12)).all(), f
    np.testing.assert_allclose(f[-1], np.sum((Ad - r["W"] @ r["Ht"].T) ** 2), rtol=1e-12)
    assert r["status"] == 0
    # Warm-started passive sets do not change the iterates (unique solves).
    rw = orc.anls(A, W0, Ht0, iters=15, warm=True)
    np.testing.assert_allclose(rw["W"], r["W"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(rw["f"], f, rtol=1e-10)


def pin_planted(orc):
    """Exact planted factorisation A = W0 H0 with separable W0 and H0 (each
    contains a scaled identity block, so the NMF is unique up to scaling and
    permutation): ANLS drives the residual to rounding level and recovers the
    factors' columns."""
    m, n, k = 60, 40, 4
    rng = np.random.default_rng(0)
    W0 = np.vstack([np.eye(k) * 2.0, rng.uniform(0, 1, (m - k, k))])
    H0 = rng.uniform(0, 1, (k, n)) * (rng.uniform(0, 1, (k, n)) < 0.5)
    H0[:, :k] = np.eye(k)
    A = (W0 @ H0).astype(np.float32)
    Wi, Hti = synth.init_factors(m, n, k, seed=100)
    r = orc.anls(A, Wi, Hti, iters=150)
    rel = r["f"][-1] / np.sum(A.astype(np.float64) ** 2)
    assert rel <= 1e-10, rel
    Wn = r["W"] / np.linalg.norm(r["W"], axis=0)
    W0n = W0 / np.linalg.norm(W0, axis=0)
    C = W0n.T @ Wn
    assert np.all(np.sort(C.max(axis=1)) > 1 - 1e-6), C


def _spd_nonneg(k, rng):
    """A Gram of a nonnegative factor (entrywise >= 0, positive definite)."""
    C = rng.uniform(0.0, 1.0, (3 * k, k))
    return C.T @ C


def _nls_value(G, g, x):
    return 0.5 * x @ G @ x - g @ x


def pin_mu(orc, seed=13):
    """Eq. 5 (MU). Hand-worked step: G = [[2, 1], [1, 2]], R = (3, 3),
    x = (1, 2): X G = (4, 5), so x becomes (1*3/4, 2*3/5) = (0.75, 1.2); every
    denominator uses the x from before the step (taking the new x_1 would give
    x_2 = 6/4.75). Then: the NLS minimiser (brute force) is a fixed point;
    k = 1 reaches R/G in one step; a zero row stays zero (no 0/0); and the
    NLS objective never increases (Lee and Seung 2001)."""
    G = np.array([[2.0, 1.0], [1.0, 2.0]])
    X = orc.mu(G, np.array([[3.0, 3.0]]), np.array([[1.0, 2.0]]))
    np.testing.assert_allclose(X, [[0.75, 1.2]], rtol=0, atol=1e-15)
    rng = np.random.default_rng(seed)
    for k in (2, 4, 6):
        G = _spd_nonneg(k, rng)
        g = rng.uniform(0.0, 1.0, k) * np.diag(G)
        sols = brute_force_nls(G, g)
        assert len(sols) == 1
        xs = sols[0]
        np.testing.assert_allclose(orc.mu(G, g[None, :], xs[None, :])[0], xs, rtol=1e-10,
                                   atol=1e-14)
    X = orc.mu(np.array([[4.0]]), np.array([[6.0], [2.0]]), np.array([[0.3], [7.0]]))
    np.testing.assert_allclose(X[:, 0], [1.5, 0.5], rtol=1e-15)
    X = orc.mu(G, g[None, :], np.zeros((1, len(g))))
    assert np.isfinite(X).all() and (X == 0).all()
    k = 8
    G = _spd_nonneg(k, rng)
    g = rng.uniform(0.0, 1.0, k) * np.diag(G)
    x = rng.uniform(0.1, 1.0, k)
    f = [_nls_value(G, g, x)]
    for _ in range(30):
        x = orc.mu(G, g[None, :], x[None, :])[0]
        f.append(_nls_value(G, g, x))
    f = np.array(f)
    assert (f[1:] <= f[:-1] + 1e-12 * np.abs(f[:-1])).all(), f


def pin_hals(orc, seed=17):
    """Eq. 6 (HALS). Hand-worked sweep: G = [[2, 1], [1, 2]], R = (3, 3),
    x = (0, 0): x_1 = (3 - 1*0)/2 = 1.5, then x_2 = (3 - 1*1.5)/2 = 0.75 with the
    new x_1 (the old one would give 1.5). With R = (3, -3) the second numerator
    is -4.5 and the projection gives x_2 = 0. A diagonal G gives the exact NLS
    solution max(R, 0)/G_ii in one sweep; repeated sweeps converge to the
    brute-force minimiser (coordinate descent on a strictly convex quadratic)
    with a non-increasing objective; a zero Gram column gives 0."""
    G = np.array([[2.0, 1.0], [1.0, 2.0]])
    X = orc.hals(G, np.array([[3.0, 3.0], [3.0, -3.0]]), np.zeros((2, 2)))
    np.testing.assert_allclose(X, [[1.5, 0.75], [1.5, 0.0]], rtol=0, atol=1e-15)
    D = np.diag([2.0, 4.0, 0.5])
    R = np.array([[1.0, -2.0, 3.0]])
    np.testing.assert_allclose(orc.hals(D, R, np.ones((1, 3))), [[0.5, 0.0, 6.0]], rtol=1e-15)
    rng = np.random.default_rng(seed)
    for k in (3, 5, 7):
        G = _spd_nonneg(k, rng)
        g = rng.normal(0.0, 1.0, k) * np.diag(G)
        sols = brute_force_nls(G, g)
        assert len(sols) == 1
        x = np.zeros(k)
        f = [_nls_value(G, g, x)]
        for _ in range(3000):
            x = orc.hals(G, g[None, :], x[None, :])[0]
            f.append(_nls_value(G, g, x))
        f = np.array(f)
        assert (f[1:] <= f[:-1] + 1e-12 * np.abs(f[:-1]) + 1e-300).all()
        np.testing.assert_allclose(x, sols[0], rtol=1e-7, atol=1e-9 * np.abs(sols[0]).max())
        np.testing.assert_allclose(orc.hals(G, g[None, :], sols[0][None, :])[0], sols[0],
                                   rtol=1e-10, atol=1e-12 * np.abs(sols[0]).max())
    Gz = np.array([[2.0, 0.0], [0.0, 0.0]])
    np.testing.assert_allclose(orc.hals(Gz, np.array([[4.0, 1.0]]), np.ones((1, 2))), [[2.0, 0.0]])


def pin_anls_local(orc, seed=19):
    """Alg. 1 with the MU and HALS updates: the objective never increases
    (each update does not increase f with the other factor fixed) and it ends
    at the recomputed ||A - W H||^2; MU keeps the starting zero pattern."""
    m, n, k = 70, 40, 5
    A = synth.dense_planted(m, n, k, 0.05, seed=seed)
    W0, Ht0 = synth.init_factors(m, n, k, seed=seed)
    Ad = A.astype(np.float64)
    for solver in ("mu", "hals"):
        r = orc.anls(A, W0, Ht0, iters=25, solver=solver)
        f = r["f"]
        assert (f[1:] <= f[:-1] * (1 + 1e-12)).all(), (solver, f)
        assert f[-1] < 0.5 * f[0], (solver, f[0], f[-1])
        np.testing.assert_allclose(f[-1], np.sum((Ad - r["W"] @ r["Ht"].T) ** 2), rtol=1e-12)
        assert (r["W"] >= 0).all() and (r["Ht"] >= 0).all()
    Wz = W0.astype(np.float64).copy()
    Wz[::7, 2] = 0.0
    r = orc.anls(A, Wz, Ht0, iters=3, solver="mu")
    assert (r["W"][::7, 2] == 0).all()


def pin_pgrad(orc, seed=23):
    """Projected-gradient norm (Lin 2007). Hand-worked: G = [[2, 1], [1, 2]],
    R = (3, 3), x = (1, 0): x G - R = (-1, -2), both count (x_1 > 0; the second
    is negative): 1 + 4 = 5; with R = (3, 0) the gradient is (-1, 1) and the
    positive entry at x_2 = 0 is dropped: 1. The full measure equals half the
    finite-difference gradient of f = ||A - W H||^2 where it is unconstrained
    (all entries positive), vanishes in H after an exact H half-step (Eq. 4)
    and at an exact planted factorisation."""
    G = np.array([[2.0, 1.0], [1.0, 2.0]])
    assert abs(orc.pgrad_sq(G, np.array([[3.0, 3.0]]), np.array([[1.0, 0.0]])) - 5.0) < 1e-15
    assert abs(orc.pgrad_sq(G, np.array([[3.0, 0.0]]), np.array([[1.0, 0.0]])) - 1.0) < 1e-15
    rng = np.random.default_rng(seed)
    m, n, k = 9, 7, 3
    A = rng.uniform(0, 1, (m, n)).astype(np.float32)
    W = rng.uniform(0.5, 1.5, (m, k))
    Ht = rng.uniform(0.5, 1.5, (n, k))
    Ad = A.astype(np.float64)
    f = lambda W_, Ht_: np.sum((Ad - W_ @ Ht_.T) ** 2)
    gW = np.zeros_like(W)
    gH = np.zeros_like(Ht)
    h = 1e-6
    for idx in np.ndindex(W.shape):
        E = np.zeros_like(W)
        E[idx] = h
        gW[idx] = (f(W + E, Ht) - f(W - E, Ht)) / (2 * h)
    for idx in np.ndindex(Ht.shape):
        E = np.zeros_like(Ht)
        E[idx] = h
        gH[idx] = (f(W, Ht + E) - f(W, Ht - E)) / (2 * h)
    expect = 0.5 * np.sqrt(np.sum(gW ** 2) + np.sum(gH ** 2))
    np.testing.assert_allclose(orc.pgrad(W, Ht, A), expect, rtol=1e-6)
    m, n, k = 60, 40, 4
    A = synth.dense_planted(m, n, k, 0.05, seed=seed)
    W0, Ht0 = synth.init_factors(m, n, k, seed=seed)
    r = orc.anls(A, W0, Ht0, iters=2)
    pH = orc.pgrad_sq(orc.gram(r["W"]), orc.mm_dense(A, r["W"], True), r["Ht"])
    total = orc.pgrad(r["W"], r["Ht"], A)
    assert pH <= 1e-18 * max(total ** 2, 1e-300) + 1e-20, (pH, total)
    Wp = rng.uniform(0, 1, (m, k))
    Hp = rng.uniform(0, 1, (n, k)) * (rng.uniform(0, 1, (n, k)) > 0.3)
    Ap = Wp @ Hp.T
    assert orc.pgrad(Wp, Hp, Ap.astype(np.float32)) <= 1e-5 * np.linalg.norm(Ap)


ALL_PINS = [pin_golden, pin_bruteforce, pin_nnls, pin_closed_forms, pin_kkt_and_warm,
            pin_products, pin_anls, pin_planted, pin_mu, pin_hals, pin_anls_local, pin_pgrad]
