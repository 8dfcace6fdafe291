"""bench.py's multi-process host logic on the CPU: two `gloo` ranks.

One process per GPU is the benchmark's N > 1 form (independent replicas, no
collective on the data path); what the ranks share is host logic: the rank
environment, a distinct seeded workload per rank, the slowest rank's time
(an all-reduce MAX) and the whole-job rate over all ranks' units.  The GPU
form runs the same functions over NCCL.
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent.parent

RANK_SCRIPT = r"""
import importlib.util, json, sys
import numpy as np
import torch.distributed as dist
spec = importlib.util.spec_from_file_location("bench", sys.argv[1])
b = importlib.util.module_from_spec(spec); spec.loader.exec_module(b)
world, rank, local = b.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
ms = 10.0 + 5.0 * rank  # this rank's time
slowest = b.max_over_ranks(ms, dist, "cpu")
rp = b.make_workload(rank, P=8)
print(json.dumps({"rank": rank, "world": world, "local": local, "slowest": slowest,
                  "rate": b.job_rate(world, 4096, 3, slowest),
                  "digest": float(np.abs(rp.pts).sum()), "n_curves": int(rp.offsets.size - 1)}))
dist.barrier()
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank: int, world: int, port: int) -> dict:
    env = dict(os.environ)
    env.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
               LOCAL_RANK=str(rank), WORLD_SIZE=str(world), CUDA_VISIBLE_DEVICES="")
    env["PYTHONPATH"] = str(ROOT) + os.pathsep + env.get("PYTHONPATH", "")
    return env


def test_two_gloo_ranks_share_the_slowest_time():
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_SCRIPT, str(ROOT / "bench.py")],
                              env=_env(r, 2, port), cwd=ROOT, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=240)
            assert p.returncode == 0, err[-2000:]
            outs.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    outs.sort(key=lambda d: d["rank"])
    assert [d["rank"] for d in outs] == [0, 1]
    assert all(d["world"] == 2 and d["local"] == d["rank"] for d in outs)
    # every rank reports the slowest rank's time, and the rate counts both ranks' units
    assert all(d["slowest"] == 15.0 for d in outs)
    assert all(abs(d["rate"] - 2 * 4096 * 3 / 15e-3) < 1e-6 for d in outs)
    # each rank aligns its own pairs (weak scaling): the workloads differ
    assert outs[0]["n_curves"] == outs[1]["n_curves"] == 16
    assert outs[0]["digest"] != outs[1]["digest"]


def test_single_process_defaults_and_seeded_workloads():
    spec_env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    code = ("import importlib.util, json, sys; import numpy as np\n"
            "spec = importlib.util.spec_from_file_location('bench', sys.argv[1])\n"
            "b = importlib.util.module_from_spec(spec); spec.loader.exec_module(b)\n"
            "a, c = b.make_workload(1, P=8), b.make_workload(1, P=8)\n"
            "print(json.dumps({'env': b.dist_env(), 'same': bool(np.array_equal(a.pts, c.pts)),\n"
            "                  'slowest': b.max_over_ranks(7.5)}))")
    spec_env["PYTHONPATH"] = str(ROOT) + os.pathsep + spec_env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", code, str(ROOT / "bench.py")], env=spec_env,
                       cwd=ROOT, capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["env"] == [1, 0, 0]
    assert d["same"] and d["slowest"] == 7.5


def test_reference_arm_runs_on_rank_zero_only():
    # ranks other than 0 exit 0 without work and print nothing
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=_env(1, 2, _free_port()),
                       cwd=ROOT, capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
    # rank 0 times the oracle on a bounded sample and prints one reference line
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--ref-pairs", "8"],
                       env=_env(0, 2, _free_port()), cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.strip().splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["unit"] == "pairs/s"
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and np.isfinite(d["ms_per_step"])
