"""Multi-process host logic of the benchmark on CPU (gloo, world size 2):
process-group set-up, the barrier and the max-over-ranks reduction that the
N-GPU replica runs use.  Each rank is a separate process, as under torchrun."""
import os
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]

SCRIPT = r'''
import os, sys
sys.path.insert(0, sys.argv[1])
import bench
world, rank, local = bench.dist_init("gloo")
assert world == 2 and rank == int(os.environ["RANK"])
bench.barrier(world)
v = bench.max_over_ranks(float(10 + rank), world)
assert v == 11.0, v
print("rank", rank, "ok", v)
'''


def test_two_gloo_ranks_barrier_and_max():
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT="29561")
        procs.append(subprocess.Popen([sys.executable, "-c", SCRIPT, str(ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    outs = [p.communicate(timeout=120)[0].decode() for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    assert all("ok 11.0" in o for o in outs)


def test_clock_sampler_without_gpu_tools():
    import bench
    with bench.ClockSampler(0) as c:
        pass
    s = c.summary()
    assert set(s) >= {"sm_mhz", "sm_max_mhz", "reasons"}
