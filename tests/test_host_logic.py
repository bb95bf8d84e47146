"""Host-side logic that needs no GPU: the C ABI exports, the multi-rank
replica/shard bookkeeping of bench.py (gloo, world size 2), and the serving
request generator."""
import os
import re
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in ("chol.h", "chol_testing.h"):
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(chol_[a-z0-9_]+)\s*\(", txt, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    import ctypes

    from paper_2606_11937_gb300 import build as libbuild
    path = libbuild.build()
    lib = ctypes.CDLL(path)
    names = _declared_functions()
    assert len(names) >= 25
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    import paper_2606_11937_gb300 as chol
    names = _declared_functions()
    missing = [n for n in sorted(names) if n not in chol.SIGNATURES]
    assert not missing, missing


def test_binding_constants_match_the_header():
    """Every enumerator the header assigns (statuses, precisions, schedules,
    flags) has the same value in the Python binding."""
    import paper_2606_11937_gb300 as chol
    txt = open(os.path.join(ROOT, "include", "chol.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    found = dict((m.group(1), int(m.group(2))) for m in re.finditer(r"\b(CHOL_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt))
    assert len(found) >= 25
    for name, value in found.items():
        assert hasattr(chol, name), name
        assert getattr(chol, name) == value, (name, getattr(chol, name), value)


def test_reference_arm_json_line():
    """bench.py --impl reference runs the oracle on the host cores (no GPU) and
    prints one JSON line with the keys of the bench contract."""
    import json
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_shard_partitions_exactly():
    import bench_batched
    for count in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            seen = []
            for rank in range(world):
                r = bench_batched.shard(count, world, rank)
                seen.extend(r)
                assert abs(len(r) - count / world) < 1
            assert seen == list(range(count))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo")
import bench, bench_batched
world, rank = dist.get_world_size(), dist.get_rank()
# replica timing: the job time is the slowest rank's time
mx = bench.allreduce_max(1.0 + rank, world)
assert mx == float(world), mx
bench.barrier(world)
# batched shards cover the batch once across ranks
import torch
mine = list(bench_batched.shard(4096, world, rank))
t = torch.tensor([len(mine), sum(mine)], dtype=torch.int64)
dist.all_reduce(t)
assert int(t[0]) == 4096 and int(t[1]) == 4095 * 4096 // 2
dist.destroy_process_group()
print("rank", rank, "ok")
"""


def test_multi_rank_bookkeeping_gloo_world2():
    port = _free_port()
    code = WORKER.format(root=ROOT)
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2")
    procs = []
    for rank in range(2):
        e = dict(env, RANK=str(rank), LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=e, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    assert all("ok" in o for o in outs)
