"""The N > 1 path of bench.py (replicas: one process per GPU, each on its own
operands, no data-path collective) on CPU with world_size-2 gloo groups:
max-over-ranks timing, the whole-job value, distinct per-rank inputs, and the
reference arm under torchrun (rank 0 alone runs and prints)."""
import json
import os
import socket
import subprocess
import sys

import multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, ws, _, d = bench._dist()
    elapsed_ms = 10.0 + 2.5 * rank          # the slower rank decides
    mx = bench.replica_max(elapsed_ms, d)
    value = bench.replica_value(1024, 10, mx, ws)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, r, ws, mx, value, bench.replica_seed(rank)))


def test_replica_aggregation_gloo_world2():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = set()
    for rank, r, ws, mx, value, seed in res:
        assert r == rank and ws == 2
        assert mx == 12.5                     # max over ranks
        assert abs(value - 2 * 1024 * 10 / 12.5e-3) < 1e-6 * value
        seeds.add(seed)
    assert len(seeds) == 2                    # every replica has its own operands


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max(3.0, None) == 3.0
    assert bench.replica_value(8, 2, 4.0, 1) == 8 * 2 / 4e-3


def test_reference_arm_under_torchrun():
    """`bench.py --impl reference` launched like the N = 2 driver run: rank 0
    prints one JSON line, rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--log2n", "10"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
