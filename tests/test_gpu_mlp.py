"""The learned passive-set proposal on the GPU (C ABI nmf_mlp_*) against the FP64
reference in oracle/mlp.py: features, logits, the gradient of the mean BCE,
Adam steps, proposals, and ANLS with the network attached (training, then
proposing), which must reach the same factors as the plain run."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_09313_gb300 as lib
    return lib


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _problem(k, nrhs, seed):
    G, B = synth.nls_batch(k, nrhs, seed=seed)
    Xp = synth.uniform_matrix(seed, synth.TID_W_INIT, nrhs, k) * 0.2
    return G, B.astype(np.float32), Xp.astype(np.float32)


@pytest.mark.parametrize("k", [5, 50, 100])
def test_features_match_oracle(nmf, k):
    G, B, Xp = _problem(k, 777, 11 + k)
    F = nmf.nmf_mlp_features(dev(G), dev(B), dev(Xp)).cpu().numpy().astype(np.float64)
    Fo = omlp.features(G, B.astype(np.float64), Xp.astype(np.float64))
    # FP32 on the GPU: entries within 1e-5 of each row's largest entry.
    scale = np.abs(Fo).max(axis=1, keepdims=True)
    assert np.abs(F - Fo).max() <= 1e-5 * scale.max()
    assert (np.abs(F - Fo) <= 2e-5 * scale).all()
    # Cold start: Xprev = NULL means zeros.
    F0 = nmf.nmf_mlp_features(dev(G), dev(B)).cpu().numpy().astype(np.float64)
    assert np.allclose(F0, omlp.features(G, B.astype(np.float64), np.zeros_like(Xp)),
                       rtol=2e-5, atol=1e-6)


def _net(nmf, k, h, seed=1509):
    p = synth.mlp_init(k, h, seed=seed)
    return nmf.nmf_mlp_create(k, h, dev(p)), p


@pytest.mark.parametrize("k,h,n", [(5, 32, 100), (50, 256, 3000), (100, 64, 129)])
def test_forward_matches_oracle(nmf, k, h, n):
    net, p = _net(nmf, k, h)
    F = np.random.default_rng(k).standard_normal((n, 3 * k)).astype(np.float32)
    z = net.nmf_mlp_forward(dev(F)).cpu().numpy().astype(np.float64)
    zo = omlp.forward(p, F, k, h)[4]
    assert np.abs(z - zo).max() <= 1e-4 * max(1.0, np.abs(zo).max())
    P = nmf.passive_to_bool(net.nmf_mlp_propose(dev(F)), k).cpu().numpy()
    sure = np.abs(zo) > 1e-3
    assert np.array_equal(P[sure], (zo > 0)[sure])


@pytest.mark.parametrize("k,h,n", [(5, 32, 100), (50, 256, 4000), (33, 64, 65)])
def test_gradient_matches_oracle(nmf, k, h, n):
    net, p = _net(nmf, k, h, seed=7)
    rng = np.random.default_rng(h)
    F = rng.standard_normal((n, 3 * k)).astype(np.float32)
    y = rng.random((n, k)) < 0.4
    g, loss = net.nmf_mlp_gradient(dev(F), nmf.bool_to_passive(torch.from_numpy(y).cuda()))
    lo, go = omlp.loss_and_grad(p, F, y, k, h)
    assert loss.item() == pytest.approx(lo, rel=1e-5)
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    for a, b in zip(omlp.unpack(g, k, h), omlp.unpack(go, k, h)):
        assert np.linalg.norm(a - b) <= 2e-4 * np.linalg.norm(b) + 1e-9


def test_adam_steps_match_oracle(nmf):
    k, h, n, lr = 20, 64, 512, 1e-3
    net, p = _net(nmf, k, h, seed=3)
    rng = np.random.default_rng(5)
    F = rng.standard_normal((n, 3 * k)).astype(np.float32)
    y = rng.random((n, k)) < 0.5
    lab = nmf.bool_to_passive(torch.from_numpy(y).cuda())
    master = p.astype(np.float64)
    m = np.zeros_like(master); v = np.zeros_like(master)
    for t in range(1, 4):                           # three full-batch steps
        net.nmf_mlp_train(dev(F), lab, batch=n, lr=lr)
        _, go = omlp.loss_and_grad(master.astype(np.float32), F, y, k, h)
        master, m, v = omlp.adam_step(master, go, m, v, t, lr)
    pg = net.nmf_mlp_get_params().cpu().numpy().astype(np.float64)
    # Each step moves a weight by at most ~lr; FP32 gradients differ by ~1e-4 relative.
    assert np.abs(pg - master).max() <= 0.05 * lr


def test_training_lowers_loss_and_learns_rule(nmf):
    k, h, n = 10, 64, 8192
    net, _ = _net(nmf, k, h, seed=4)
    F = np.random.default_rng(6).standard_normal((n, 3 * k)).astype(np.float32)
    y = F[:, 2 * k:] > 0
    Fd, lab = dev(F), nmf.bool_to_passive(torch.from_numpy(y).cuda())
    l0 = net.nmf_mlp_gradient(Fd, lab)[1].item()
    for _ in range(30):
        net.nmf_mlp_train(Fd, lab, batch=1024, lr=3e-3)
    l1 = net.nmf_mlp_gradient(Fd, lab)[1].item()
    assert l1 < 0.3 * l0
    P = nmf.passive_to_bool(net.nmf_mlp_propose(Fd), k).cpu().numpy()
    assert (P == y).mean() > 0.97


def test_bad_arguments(nmf):
    with pytest.raises(ValueError):
        nmf.nmf_mlp_create(10, 16, torch.zeros(5, device="cuda"))
    assert nmf.nmf_mlp_param_count(0, 16) == 0
    assert nmf.nmf_mlp_param_count(10, 2000) == 0


def _run(nmf, A, W0, Ht0, T, start, net=None, mode=None, epochs=2):
    h = nmf.nmf_init(dev(A), dev(W0), dev(Ht0), precision="fp32", start=start)
    if net is not None:
        h.nmf_set_proposal(net, mode, epochs=epochs, batch=2048, lr=2e-3)
    h.nmf_iterate(T)
    assert h.nmf_sync() == nmf.NMF_OK
    st = h.nmf_get_stats()
    W, Ht = h.nmf_get_factors()
    f = np.array(h.nmf_objective_history())
    h.nmf_destroy()
    return W.double().cpu().numpy(), Ht.double().cpu().numpy(), f, st


def test_anls_with_learned_proposal_reaches_the_same_factors(nmf):
    # Train during the first iterations, then propose; every solve still ends
    # at the unique minimiser, so the run matches the plain one.
    m, n, k = 1500, 1000, 12
    A = synth.dense_planted(m, n, k, 0.01, seed=21)
    W0, Ht0 = synth.init_factors(m, n, k, seed=21)
    Wr, Hr, fr, st_cold = _run(nmf, A, W0, Ht0, 8, "cold")
    net, _ = _net(nmf, k, 64, seed=2)
    h = nmf.nmf_init(dev(A), dev(W0), dev(Ht0), precision="fp32", start="cold")
    h.nmf_set_proposal(net, "train", epochs=3, batch=1024, lr=2e-3)
    h.nmf_iterate(4)
    st_train = h.nmf_get_stats()
    h.nmf_set_proposal(net, "use")
    h.nmf_iterate(4)
    assert h.nmf_sync() == nmf.NMF_OK
    st = h.nmf_get_stats()
    W, Ht = h.nmf_get_factors()
    f = np.array(h.nmf_objective_history())
    h.nmf_destroy()
    assert np.abs(f - fr).max() / fr.min() <= 1e-5
    assert np.linalg.norm(W.double().cpu().numpy() - Wr) <= 1e-4 * np.linalg.norm(Wr)
    # Rounds of the last four iterations: learned start against a cold start.
    learned = st["bpp_rounds"] - st_train["bpp_rounds"]
    _, _, _, st_cold4 = _run(nmf, A, W0, Ht0, 4, "cold")
    cold_last4 = st_cold["bpp_rounds"] - st_cold4["bpp_rounds"]
    print(f"rounds in iterations 5-8: learned {learned}, cold {cold_last4}")
    assert learned < 0.5 * cold_last4
    assert st["ms_proposal"] >= 0.0


def test_forward_hand_worked(nmf):
    # The hand-worked pass of tests/test_oracle_mlp.py (every intermediate
    # value exact in FP32, so the GPU must reproduce the logit exactly): one
    # weight is not a BF16 value and must be used rounded, and each ReLU
    # zeroes one unit.
    from tests.test_oracle_mlp import HAND_F, HAND_LOGIT, HAND_PARAMS
    net = nmf.nmf_mlp_create(1, 2, dev(HAND_PARAMS))
    z = net.nmf_mlp_forward(dev(HAND_F.astype(np.float32))).cpu().numpy()
    assert z[0, 0] == np.float32(HAND_LOGIT)
    P = nmf.passive_to_bool(net.nmf_mlp_propose(dev(HAND_F.astype(np.float32))), 1).cpu()
    assert bool(P[0, 0])
    net.nmf_mlp_destroy()
