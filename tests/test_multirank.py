"""N > 1 on the host. The path shards into independent replicas (no exchange
step, so no collective in the data path); bench.py under torchrun runs one
replica per rank and reports the units of all ranks over the slowest rank's
time. Two gloo ranks on the CPU check that reduction, and the reference arm
under torchrun prints one line, from rank 0, while the other rank exits 0."""
import json
import os
import socket
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, port, outdir):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=2)
    try:
        v = bench.max_over_ranks(1.5 + rank, 2, torch.device("cpu"))   # rank times 1.5 and 2.5
        with open(os.path.join(outdir, f"rank{rank}"), "w") as fh:
            fh.write(repr(v))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks(tmp_path):
    mp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    got = [float(open(tmp_path / f"rank{r}").read()) for r in range(2)]
    assert got == [2.5, 2.5]


def test_max_over_ranks_one_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, torch.device("cpu")) == 3.25


def test_reference_arm_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--workload", "dense-small", "--gpus", "2", "--steps", "1",
           "--warmup", "3"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
