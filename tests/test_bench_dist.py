"""The multi-rank host logic of bench.py on CPU with the gloo backend
(world size 2): every rank gets its own seed, the job time is the slowest
rank's, and the work is summed over ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms, units = bench.aggregate(dist, local_ms=10.0 + rank, local_units=100.0 * (rank + 1), device="cpu")
        q.put((rank, bench.rank_seed(rank), ms, units))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert [o[1] for o in out] == [0, 1]                 # distinct seeds
    assert all(o[2] == 11.0 for o in out)                 # max time over ranks
    assert all(o[3] == 300.0 for o in out)                # summed work


def test_single_rank_passthrough():
    import bench

    assert bench.aggregate(None, 5.0, 7.0, "cpu") == (5.0, 7.0)


def test_oracle_parity_reads_the_stored_oracle_solution():
    """bench.py states each default-workload result's error against the FP64
    oracle's stored solution of the same problem, and nothing for another."""
    import numpy as np

    import bench
    import workloads as W

    p = bench.problem(0)
    g = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sincos2d_n2049_s0.npz"))
    u = np.full(p.n_nodes, np.inf)
    u[g["idx"]] = g["u"]
    r = bench.oracle_parity(p, u, g["labels"])
    assert r["max_abs_err"] == 0.0 and r["label_agreement"] == 1.0 and r["nodes_sampled"] == g["idx"].size
    u[g["idx"][7]] += 1e-3
    assert bench.oracle_parity(p, u, g["labels"])["max_abs_err"] == pytest.approx(1e-3)
    assert bench.oracle_parity(W.sincos2d(0, n=1025, n_coarse=33), u, g["labels"]) is None
    assert bench.oracle_parity(W.sincos2d(1), u, g["labels"]) is None


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the FP64 oracle on the host cores and
    prints one JSON line with the keys the measurement contract asks for."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "node-control updates/s" and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "patchy2d_sincos_n2049_c65_nc64_R4"


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the multi-GPU bench is (torchrun, two ranks), the reference
    arm runs on rank 0 alone, prints one line, and every rank exits 0."""
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert len([l for l in r.stdout.splitlines() if l.startswith("{")]) == 1
