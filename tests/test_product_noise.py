"""How far a BF16x3-sized product error moves the ANLS objective (CPU only).

The BF16 head/tail split keeps 16 of FP32's 24 mantissa bits per operand, so
every term of the tensor-core products carries a random relative error of
about 2^-17.6; summed over a contraction of length q the products' relative
error has a spread of ~5e-6 / sqrt(q) (measured against FP64 on the GPU:
1.6e-7 at q = 1000, 2.9e-8 at q = 64000) and a bias of -6e-8. This test
runs Alg. 1 in FP64 through the oracle's NLS solver with exactly that much
random error injected into A H^T and A^T W, on the small dense configuration
(A = W0 H0 + |N(0, 0.01^2)|, 2000 x 1000, k = 10, 10 iterations), and
records the spread of the maximum relative objective error against the
unperturbed oracle over eight draws. The result (median ~1e-5, max ~1.4e-5)
is why the GPU test of this configuration holds the BF16x3 path to 3e-5 while
the FP32 path, which the configuration is defined for, keeps 1e-5; the bias
alone moves the objective by ~1e-11.
"""
import numpy as np

import oracle
import synth


def _anls_with_product_noise(A, W0, Ht0, iters, eps, bias, seed):
    rng = np.random.default_rng(seed)
    Ht = Ht0.astype(np.float64)
    f = []
    for _ in range(iters):
        V = A @ Ht
        W = oracle.bpp(Ht.T @ Ht, V * (1.0 + bias + eps * rng.standard_normal(V.shape)))[0]
        U = A.T @ W
        Ht = oracle.bpp(W.T @ W, U * (1.0 + bias + eps * rng.standard_normal(U.shape)))[0]
        R = A - W @ Ht.T
        f.append(float((R * R).sum()))
    return np.array(f)


def test_bf16x3_product_noise_moves_small_config_objective_about_1e5():
    m, n, k, T = 2000, 1000, 10, 10
    A32 = synth.dense_planted(m, n, k, 0.01)
    A = A32.astype(np.float64)
    W0, Ht0 = synth.init_factors(m, n, k)
    f_or = oracle.anls(A32, W0, Ht0, iters=T)["f"][1:]
    clean = _anls_with_product_noise(A, W0, Ht0, T, 0.0, 0.0, 0)
    assert np.abs(clean - f_or).max() / f_or.min() < 1e-11      # same algorithm
    errs = [np.max(np.abs(_anls_with_product_noise(A, W0, Ht0, T, 1.6e-7, -6e-8, s) - f_or) / f_or)
            for s in range(8)]
    print("max rel f err per draw:", ["%.2e" % e for e in errs])
    assert 3e-6 < np.median(errs) < 2e-5
    assert max(errs) < 3e-5
    bias_only = np.max(np.abs(_anls_with_product_noise(A, W0, Ht0, T, 0.0, -6e-8, 0) - f_or) / f_or)
    assert bias_only < 1e-8
