"""The product path has no CPU fallback: without a GPU, the binding rejects
host tensors and bench.py fails instead of printing a number. (These run on
hosts without CUDA; on a GPU host they are skipped.)"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU behaviour")


def test_binding_rejects_host_tensors():
    import paper_1509_09313_gb300 as nmf
    G = torch.eye(4, dtype=torch.float64)
    B = torch.from_numpy(np.ones((3, 4), dtype=np.float32))
    with pytest.raises((TypeError, ValueError, RuntimeError)):
        nmf.nmf_nls_bpp(G, B)


def test_bench_fails_without_a_gpu():
    out = subprocess.run([sys.executable, "bench.py", "--steps", "1", "--warmup", "3",
                          "--workload", "dense-small", "--no-e2e", "--no-cpu-baseline"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode != 0
    assert not any(l.startswith("{") for l in out.stdout.splitlines())
