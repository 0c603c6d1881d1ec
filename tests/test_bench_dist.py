"""The N > 1 path of bench.py on CPU: world size 2 over gloo.

N GPUs run N independent replicas of the workload (the grid is not split,
no data-path collective); the host logic that remains is the rendezvous,
the max over ranks of the timed region, the whole-job value, and rank 0
alone printing.  These run here as two processes with the gloo backend."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    w, r, loc = bench._dist()
    bench._init_dist(w, loc)
    bench._barrier(w)
    ms = 10.0 + 5.0 * r                      # rank 1 is the slow replica
    ms_max = bench._barrier_max(ms, w)
    q.put((r, w, ms_max, bench.replica_value(w, 1000, 4, ms_max)))
    bench._close_dist(w)


def test_gloo_two_ranks_max_and_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms_max, val in out:
        assert w == 2
        assert ms_max == 15.0                 # the slowest rank's time on every rank
        # all ranks' cell-stages (2 x 1000 cells x 3 stages x 4 steps) / 15 ms
        assert val == pytest.approx(2 * 1000 * 3 * 4 / 15e-3)


def test_replica_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_value(1, 4096 * 4096, 40, 1000.0) == pytest.approx(4096 ** 2 * 120)


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` under torchrun: rank 0 times the oracle
    and prints one line; the other rank exits 0 without work."""
    import oracle
    oracle.build()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}",
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS=str(max(1, (os.cpu_count() or 2) // 2)))
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
