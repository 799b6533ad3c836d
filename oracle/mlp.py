"""FP64 CPU reference of the learned passive-set proposal.

TEST INFRASTRUCTURE ONLY: imported by tests/ and nothing on the product path.
The paper has no counterpart: the proposal only chooses the starting partition
of block principal pivoting (Sec. 4.2), which then runs to the KKT point of
Eq. 4 as always, so the answer of every solve is unchanged and BPP's own
tests decide whether each proposal is optimal. Plain numpy in FP64, one line per step of the
definition below; the weights are used after rounding to BF16, as the GPU
uses them.

Definition
----------
For one right-hand side of Eq. 3 in normal-equations form,
min_{x >= 0} 1/2 x^T G x - g^T x, with the previous iterate x_p of the same
row of the factor (zero on a cold start):

  d_i = sqrt(G_ii) where G_ii > 0, else 1
  s   = max_i |g_i| / d_i, or 1 where that is 0
  features (3k) = [ (G x_p - g)_i / (d_i s),
                    log(G_ii / mean_j G_jj) (0 where G_ii <= 0),
                    x_p,i d_i / s ]

i.e. the gradient, the Gram diagonal and the previous iterate, in the
diagonally scaled variables and normalised by the right-hand side's scale.
The network is 3k -> h -> h -> k with ReLU after the first two layers
(y = W x + b per layer, W stored rows = outputs); the proposed passive set is
{i : logit_i > 0}. Training minimises the mean binary cross-entropy of
sigmoid(logits) against the final passive set the solve reached, with Adam
(Kingma and Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
FP32 master weights; the gradient is taken with respect to the BF16-rounded
weights the forward pass used.

Parameter layout (flat, FP32): W1 (h x 3k), b1 (h), W2 (h x h), b2 (h),
W3 (k x h), b3 (k).
"""
from __future__ import annotations

import numpy as np

BETA1 = 0.9
BETA2 = 0.999
ADAM_EPS = 1e-8


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def sizes(k: int, h: int):
    return [(h, 3 * k), (h,), (h, h), (h,), (k, h), (k,)]


def unpack(params, k: int, h: int):
    """The six tensors of a flat parameter array (views, same dtype)."""
    out, off = [], 0
    for shp in sizes(k, h):
        n = int(np.prod(shp))
        out.append(params[off:off + n].reshape(shp))
        off += n
    assert off == params.size
    return out


def features(G, B, Xp) -> np.ndarray:
    """nrhs x 3k features of right-hand sides B (nrhs x k) with Gram G (k x k)
    and previous iterates Xp (nrhs x k)."""
    G = np.asarray(G, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    Xp = np.asarray(Xp, dtype=np.float64)
    diag = np.diag(G)
    pos = diag > 0
    d = np.where(pos, np.sqrt(np.where(pos, diag, 1.0)), 1.0)
    s = np.max(np.abs(B) / d, axis=1)
    s = np.where(s > 0, s, 1.0)[:, None]
    grad = Xp @ G - B                        # G symmetric: row j is (G x_p - g)^T
    mean_diag = diag[pos].mean() if pos.any() else 1.0
    logd = np.where(pos, np.log(np.where(pos, diag, 1.0) / mean_diag), 0.0)
    return np.concatenate([grad / d / s, np.broadcast_to(logd, B.shape), Xp * d / s], axis=1)


def forward(params, F, k: int, h: int, round_bf16: bool = True):
    """Returns (z1, a1, z2, a2, logits) for features F (nrhs x 3k)."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(params), k, h)
    q = bf16 if round_bf16 else (lambda w: np.asarray(w, dtype=np.float64))
    F = np.asarray(F, dtype=np.float64)
    z1 = F @ q(W1).T + np.asarray(b1, dtype=np.float64)
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ q(W2).T + np.asarray(b2, dtype=np.float64)
    a2 = np.maximum(z2, 0.0)
    logits = a2 @ q(W3).T + np.asarray(b3, dtype=np.float64)
    return z1, a1, z2, a2, logits


def bce(logits, labels) -> float:
    """Mean binary cross-entropy of sigmoid(logits) against labels in {0, 1}."""
    z = np.asarray(logits, dtype=np.float64)
    y = np.asarray(labels, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def loss_and_grad(params, F, labels, k: int, h: int, round_bf16: bool = True):
    """Mean BCE and its gradient (flat, FP64) with respect to the parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(params), k, h)
    q = bf16 if round_bf16 else (lambda w: np.asarray(w, dtype=np.float64))
    F = np.asarray(F, dtype=np.float64)
    z1, a1, z2, a2, logits = forward(params, F, k, h, round_bf16)
    y = np.asarray(labels, dtype=np.float64)
    n = logits.size
    dz3 = (1.0 / (1.0 + np.exp(-logits)) - y) / n       # d loss / d logits
    gW3 = dz3.T @ a2
    gb3 = dz3.sum(axis=0)
    da2 = dz3 @ q(W3)
    dz2 = da2 * (z2 > 0)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(axis=0)
    da1 = dz2 @ q(W2)
    dz1 = da1 * (z1 > 0)
    gW1 = dz1.T @ F
    gb1 = dz1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return bce(logits, y), grad


def adam_step(master, grad, m, v, t: int, lr: float):
    """One Adam step (step number t >= 1); returns new (master, m, v), FP64."""
    m = BETA1 * np.asarray(m, dtype=np.float64) + (1 - BETA1) * grad
    v = BETA2 * np.asarray(v, dtype=np.float64) + (1 - BETA2) * grad * grad
    mhat = m / (1 - BETA1 ** t)
    vhat = v / (1 - BETA2 ** t)
    master = np.asarray(master, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + ADAM_EPS)
    return master, m, v


def propose(params, F, k: int, h: int) -> np.ndarray:
    """Proposed passive sets (nrhs x k bool): logit > 0."""
    return forward(params, F, k, h)[4] > 0
