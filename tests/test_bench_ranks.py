"""Host logic of the benchmark's multi-rank runs (independent replicas, one field per rank), on CPU ranks.

Under torchrun every rank estimates its own gauge field and the job's time is the slowest rank's: the only
collective is that max, outside the data path.  Here two gloo ranks on 127.0.0.1 run the same reduction; the
reference arm's non-zero ranks exit at once without output."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, world, local = bench.dist_env()
dist.init_process_group("gloo")
t = bench.max_over_ranks(1.5 + 2.0 * rank, world, device="cpu")
dist.barrier()
dist.destroy_process_group()
print("rank=%d world=%d max=%r seed=%d" % (rank, world, t, bench.replica_seed(0, rank)))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port))
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return env


def test_two_gloo_ranks_take_the_slowest_replica():
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_SCRIPT, ROOT], env=_env(r, 2, port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-2000:]
        outs.append(out.strip().splitlines()[-1])
    assert outs[0] == "rank=0 world=2 max=3.5 seed=0", outs
    assert outs[1] == "rank=1 world=2 max=3.5 seed=1", outs


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.25, 1) == 0.25
    assert bench.replica_seed(3, 0) == 3


def test_reference_arm_runs_on_rank_zero_only():
    # rank 1 of a two-rank reference run: no work, no output, exit status 0
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=_env(1, 2, _free_port()), capture_output=True,
                       text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
