"""Pins of the FP64 reference of the learned passive-set proposal (oracle/mlp.py):
BF16 rounding against an independent implementation, features on hand-worked
cases, a hand-worked forward pass with nonzero weights and biases (with planted
mistakes that it must catch), gradients against central finite differences and
closed forms, the first Adam step in closed form, and training that learns a
simple rule."""
import numpy as np
import pytest
import torch

import synth
from oracle import mlp


def test_bf16_rounding_matches_torch():
    x = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -2.5e-3, 3.0e5, 1e-30, 0.1], np.float32)
    x = np.concatenate([x, np.random.default_rng(0).standard_normal(1000).astype(np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)
    assert mlp.bf16(np.float32(1.0 + 2**-8)) == 1.0                 # tie to even
    assert mlp.bf16(np.float32(1.0 + 3 * 2**-8)) == 1.0 + 2**-6     # tie to even (up)


def test_features_hand_worked():
    G = np.diag([4.0, 9.0, 0.0])
    g = np.array([[2.0, -3.0, 0.0]])
    xp = np.array([[1.0, 0.5, 0.0]])
    f = mlp.features(G, g, xp)[0]
    # d = (2, 3, 1); s = max(2/2, 3/3, 0) = 1; G x - g = (2, 7.5, 0)
    assert np.allclose(f[:3], [1.0, 2.5, 0.0])
    assert np.allclose(f[3:6], [np.log(4 / 6.5), np.log(9 / 6.5), 0.0])
    assert np.allclose(f[6:], [2.0, 1.5, 0.0])
    # Scale invariance: scaling g and x_p by c, or G by c, leaves the features unchanged.
    G2 = np.array([[2.0, 0.5], [0.5, 1.0]])
    g2 = np.array([[1.0, -0.3]])
    x2 = np.array([[0.2, 0.7]])
    f0 = mlp.features(G2, g2, x2)
    assert np.allclose(mlp.features(G2, 5 * g2, 5 * x2), f0)
    assert np.allclose(mlp.features(3 * G2, 3 * g2, x2), f0)


def _tiny(seed=3, k=3, h=5, n=7):
    rng = np.random.default_rng(seed)
    p = synth.mlp_init(k, h, seed=seed).astype(np.float64)
    p += 0.05 * rng.standard_normal(p.size)            # nonzero biases too
    F = rng.standard_normal((n, 3 * k))
    y = rng.random((n, k)) < 0.5
    return p, F, y, k, h


def test_gradient_matches_central_differences():
    p, F, y, k, h = _tiny()
    loss, g = mlp.loss_and_grad(p, F, y, k, h, round_bf16=False)
    eps = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        q = p.copy(); q[i] += eps
        lp = mlp.bce(mlp.forward(q, F, k, h, round_bf16=False)[4], y)
        q[i] -= 2 * eps
        lm = mlp.bce(mlp.forward(q, F, k, h, round_bf16=False)[4], y)
        fd[i] = (lp - lm) / (2 * eps)
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-9), np.abs(g - fd).max()
    assert loss == pytest.approx(mlp.bce(mlp.forward(p, F, k, h, round_bf16=False)[4], y))


def test_gradient_closed_form_with_zero_weights():
    # W1 = W2 = W3 = 0: a1 = relu(b1), a2 = relu(b2), logits = b3 for every sample.
    k, h, n = 4, 6, 9
    rng = np.random.default_rng(1)
    W1, b1, W2, b2, W3, b3 = (np.zeros((h, 3 * k)), rng.random(h) + 0.1, np.zeros((h, h)),
                              rng.random(h) - 0.5, np.zeros((k, h)), rng.standard_normal(k))
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    F = rng.standard_normal((n, 3 * k))
    y = rng.random((n, k)) < 0.3
    _, g = mlp.loss_and_grad(p, F, y, k, h, round_bf16=False)
    gW1, gb1, gW2, gb2, gW3, gb3 = mlp.unpack(g, k, h)
    sig = 1 / (1 + np.exp(-b3))
    dz3 = (sig[None, :] - y) / (n * k)
    assert np.allclose(gb3, dz3.sum(0))
    assert np.allclose(gW3, np.outer(dz3.sum(0), np.maximum(b2, 0)))
    assert np.allclose(gW2, 0) and np.allclose(gb2, 0) and np.allclose(gW1, 0) and np.allclose(gb1, 0)


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + mlp.ADAM_EPS))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_learns_a_simple_rule():
    # Label i passive iff the previous iterate's scaled entry is positive.
    k, h, n = 5, 32, 512
    rng = np.random.default_rng(4)
    F = rng.standard_normal((n, 3 * k))
    y = F[:, 2 * k:] > 0
    p = synth.mlp_init(k, h, seed=9).astype(np.float64)
    m = np.zeros_like(p); v = np.zeros_like(p)
    loss0 = mlp.loss_and_grad(p, F, y, k, h)[0]
    for t in range(1, 301):
        loss, g = mlp.loss_and_grad(p.astype(np.float32), F, y, k, h)
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-2)
    assert loss < 0.25 * loss0
    assert (mlp.propose(p.astype(np.float32), F, k, h) == y).mean() > 0.95


# A hand-worked forward pass, k = 1, hidden 2 (3 features). Every weight but
# W1[0][0] is a BF16 value; W1[0][0] = 1 + 3*2^-9 lies between the BF16 neighbours
# 1 and 1 + 2^-7, nearer the upper, so it is used as 1.0078125. Biases stay FP32.
#   z1 = W1 f + b1 = (1.0078125 + 1 - 0.25 + 0.125, -1 + 1 - 1 - 0.5) = (1.8828125, -1.5)
#   a1 = relu(z1) = (1.8828125, 0)
#   z2 = W2 a1 + b2 = (1.8828125 + 0.25, 0.94140625 - 1.5) = (2.1328125, -0.55859375)
#   a2 = (2.1328125, 0)
#   logit = 2 * 2.1328125 + 4 * 0 - 1 = 3.265625
HAND_F = np.array([[1.0, 2.0, -1.0]])
HAND_PARAMS = np.array([1.0 + 3 * 2**-9, 0.5, 0.25, -1.0, 0.5, 1.0,   # W1 (2 x 3)
                        0.125, -0.5,                                   # b1
                        1.0, -2.0, 0.5, 1.0,                           # W2 (2 x 2)
                        0.25, -1.5,                                    # b2
                        2.0, 4.0,                                      # W3 (1 x 2)
                        -1.0], dtype=np.float32)                       # b3
HAND_Z1 = [1.8828125, -1.5]
HAND_Z2 = [2.1328125, -0.55859375]
HAND_LOGIT = 3.265625


def pin_mlp_forward_hand(mod):
    z1, a1, z2, a2, logits = mod.forward(HAND_PARAMS, HAND_F, 1, 2)
    np.testing.assert_array_equal(z1[0], HAND_Z1)
    np.testing.assert_array_equal(a1[0], [HAND_Z1[0], 0.0])
    np.testing.assert_array_equal(z2[0], HAND_Z2)
    np.testing.assert_array_equal(a2[0], [HAND_Z2[0], 0.0])
    assert logits[0, 0] == HAND_LOGIT
    assert bool(mod.propose(HAND_PARAMS, HAND_F, 1, 2)[0, 0])


def test_forward_hand_worked():
    pin_mlp_forward_hand(mlp)


MLP_MUTANTS = {
    "relu1_dropped": ("a1 = np.maximum(z1, 0.0)", "a1 = z1"),
    "relu2_dropped": ("a2 = np.maximum(z2, 0.0)", "a2 = z2"),
    "w1_not_rounded": ("z1 = F @ q(W1).T", "z1 = F @ np.asarray(W1, dtype=np.float64).T"),
    "b3_dropped": ("logits = a2 @ q(W3).T + np.asarray(b3, dtype=np.float64)",
                   "logits = a2 @ q(W3).T"),
}


@pytest.mark.parametrize("name", sorted(MLP_MUTANTS))
def test_forward_mutant_is_caught(name):
    # The mistake is planted in a copy of oracle/mlp.py's source, loaded as a
    # separate module; the real module is untouched.
    import types
    old, new = MLP_MUTANTS[name]
    src = open(mlp.__file__).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType(f"mlp_mutant_{name}")
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), mod.__dict__)
    with pytest.raises(AssertionError):
        pin_mlp_forward_hand(mod)
