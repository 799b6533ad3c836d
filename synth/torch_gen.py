"""Device-side copy of the seeded generator in ``synth`` for inputs too large to
build on the host (the 96000 x 64000 dense workload is 24.6 GB).

Same definition as ``synth``: SplitMix64 outputs indexed by element, uniforms
from the top 53 bits, Box-Muller normals, A = W0 H0 + |sigma N| formed in FP64
and stored FP32. The integer steps use int64 arithmetic, whose wrap-around
multiplication equals the uint64 one; right shifts are made logical by
masking. W0 and H0 themselves are generated on the host (they are small) so
they are bit-identical; the FP64 product may round differently from numpy's,
so A can differ from the host recipe by one FP32 ulp in rare elements.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (DEFAULT_SEED, GOLDEN, TID_H0, TID_NOISE_U1, TID_NOISE_U2, TID_STRESS_A, TID_W0,
               stream_state, stress_factor, uniform_matrix)


def _i64(u) -> int:
    u = int(u) & 0xFFFFFFFFFFFFFFFF
    return u - (1 << 64) if u >= (1 << 63) else u


_M1 = _i64(0xBF58476D1CE4E5B9)
_M2 = _i64(0x94D049BB133111EB)
_G = _i64(GOLDEN)


def _lsr(z: torch.Tensor, s: int) -> torch.Tensor:
    return (z >> s) & ((1 << (64 - s)) - 1)


def _mix64(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _lsr(z, 30)) * _M1
    z = (z ^ _lsr(z, 27)) * _M2
    return z ^ _lsr(z, 31)


def _uniform(seed, tid, idx: torch.Tensor, open0: bool) -> torch.Tensor:
    s = _i64(stream_state(seed, tid))
    z = _mix64(s + (idx + 1) * _G)
    top = _lsr(z, 11).to(torch.float64)
    return (top + (1.0 if open0 else 0.0)) * (2.0 ** -53)


def dense_planted_device(m: int, n: int, k: int, sigma: float, seed: int,
                         device: torch.device, rows_per_chunk: int = 2048) -> torch.Tensor:
    """The ``synth.dense_planted`` recipe built on the device, float32 m x n."""
    W0 = torch.from_numpy(uniform_matrix(seed, TID_W0, m, k, 0, 0, k)).to(device)
    H0 = torch.from_numpy(uniform_matrix(seed, TID_H0, k, n, 0, 0, n)).to(device)
    A = torch.empty((m, n), dtype=torch.float32, device=device)
    cols = torch.arange(n, dtype=torch.int64, device=device)
    for r0 in range(0, m, rows_per_chunk):
        r1 = min(m, r0 + rows_per_chunk)
        blk = W0[r0:r1] @ H0
        if sigma:
            rows = torch.arange(r0, r1, dtype=torch.int64, device=device)
            idx = rows[:, None] * n + cols[None, :]
            u1 = _uniform(seed, TID_NOISE_U1, idx, True)
            u2 = _uniform(seed, TID_NOISE_U2, idx, False)
            del idx
            blk += (sigma * (torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * np.pi * u2))).abs()
            del u1, u2
        A[r0:r1] = blk.to(torch.float32)
        del blk
    return A


def normal_device(seed: int, tensor_pair, rows: int, cols: int, device: torch.device,
                  row0: int = 0) -> torch.Tensor:
    """``synth.normal_matrix`` on the device (float64)."""
    r = torch.arange(row0, row0 + rows, dtype=torch.int64, device=device)[:, None]
    c = torch.arange(cols, dtype=torch.int64, device=device)[None, :]
    idx = r * cols + c
    u1 = _uniform(seed, tensor_pair[0], idx, True)
    u2 = _uniform(seed, tensor_pair[1], idx, False)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * np.pi * u2)


def stress_batch_device(device: torch.device, rows: int = 200000, k: int = 100,
                        nrhs: int = 1000000, seed: int = DEFAULT_SEED, mean_a: float = 0.5):
    """The batched-NLS stress inputs: G = W^T W of W = ``synth.stress_factor``
    (rows x k) and nrhs right-hand sides drawn from the distribution of W^T a
    for a uniform in [0, 1)^rows (central limit theorem: mean W^T 1 / 2,
    covariance G / 12), b = W^T 1 / 2 + L z / sqrt(12) with G = L L^T and z
    standard normal. Forming W^T a itself would cost 2 rows k nrhs flops.
    mean_a shifts a (a = u + mean_a - 1/2, u uniform in [0, 1)): b = mean_a
    W^T 1 + L z / sqrt(12). mean_a = 1/2 (the default) makes every solution
    positive; a small mean_a gives solutions of mixed signs, so the passive
    sets vary from one right-hand side to the next.
    Returns (G float64 k x k, B float32 nrhs x k), both on `device`. The
    factor L is taken on the host (input generation only)."""
    W = torch.from_numpy(stress_factor(rows, k, seed=seed)).to(device).double()
    G = W.T @ W
    mean = mean_a * W.sum(dim=0)
    L = torch.linalg.cholesky(G.cpu()).to(device)
    B = torch.empty((nrhs, k), dtype=torch.float32, device=device)
    pair = (TID_STRESS_A, TID_NOISE_U2)
    step = 100000
    for r0 in range(0, nrhs, step):
        r1 = min(nrhs, r0 + step)
        z = normal_device(seed, pair, r1 - r0, k, device, row0=r0)
        B[r0:r1] = (mean + z @ L.T / np.sqrt(12.0)).float()
        del z
    return G.contiguous(), B
