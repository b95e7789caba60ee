"""Multi-process host logic of the benchmark, on CPU (gloo, world size 2): the replicas'
rendezvous, barrier and max-over-ranks timing, one seeded scene per replica, and the reference
arm under torchrun (rank 0 alone runs and prints).  The library path does not shard within a
scene (replicas only), so these are the parts of `bench.py --gpus N` that run on every rank."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# one replica: rendezvous, a barrier, the max of a per-rank value, and the first depth frame of
# its scene (a checksum), printed as one JSON line
_REPLICA = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import bench
rank, world, local = bench.dist_init()
bench.barrier(world)
m = bench.reduce_max(10.0 + rank, world)
d = bench.scene_for(rank, 2).depth(0)
print(json.dumps({"rank": rank, "world": world, "local": local, "max": m,
                  "depth_sum": float(np.nansum(d.astype(np.float64)))}), flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_replicas_rendezvous_and_take_the_max_over_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _REPLICA, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err
        outs.append(json.loads([l for l in out.splitlines() if l.startswith("{")][-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    assert all(o["world"] == 2 and o["max"] == 11.0 for o in outs)
    # each replica integrates its own seeded scene
    assert outs[0]["depth_sum"] != outs[1]["depth_sum"]


def test_replica_scenes_are_seeded_per_rank():
    sys.path.insert(0, ROOT)
    import bench

    a0 = bench.scene_for(0, 2).depth(0)
    assert np.array_equal(a0, bench.scene_for(0, 2).depth(0), equal_nan=True)  # deterministic
    assert not np.array_equal(a0, bench.scene_for(1, 2).depth(0), equal_nan=True)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2",
           "--warmup", "3"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2 and d["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
