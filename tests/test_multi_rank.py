"""The N > 1 path of bench.py on the CPU: two gloo ranks, the way torchrun
launches the replicas (one process per GPU).  Each rank advances its own
lattice, so the only cross-rank steps are the barrier and the maximum of the
ranks' times; the job's throughput counts every rank's nodes in the slowest
rank's time.  The reference arm prints on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo")
ms = [3.0, 5.0][rank]
dist.barrier()
m = bench.max_over_ranks(ms, world)
print("RESULT", rank, m, bench.job_mlups(1000, 10, world, m * 1e-3), flush=True)
dist.destroy_process_group()
"""


def run_ranks(code, world=2, extra_args=()):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT, *extra_args], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_two_gloo_ranks_take_the_slowest_time():
    outs = run_ranks(WORKER)
    res = {}
    for o in outs:
        for line in o.splitlines():
            if line.startswith("RESULT"):
                _, r, m, mlups = line.split()
                res[int(r)] = (float(m), float(mlups))
    assert res[0] == res[1]
    assert res[0][0] == 5.0
    # 2 ranks x 1000 nodes x 10 steps in 5 ms
    assert res[0][1] == pytest.approx(2 * 1000 * 10 / 5e-3 / 1e6)


REF = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
import bench
sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3", "--cpu-n", "8", "--gpus", "2"]
bench.main()
"""


@pytest.mark.slow
def test_reference_arm_prints_on_rank_zero_only(orc):
    outs = run_ranks(REF)
    assert '"impl": "reference"' in outs[0]
    assert outs[1].strip() == ""


def test_nested_measurement_failure_keeps_the_main_line():
    """A batched or surrogate measurement that raises is reported in its
    place in the bench line; the training log is dropped from one that runs."""
    import bench

    def fails(args):
        raise RuntimeError("no batched cases")

    assert bench.nested_run(fails, None) == {"error": "RuntimeError: no batched cases"}
    ok = bench.nested_run(lambda a: {"metric": "m", "value": 1.0, "loss": [0.5], "n_gpus": 1}, None)
    assert ok == {"metric": "m", "value": 1.0}
