"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the
maximum over ranks that the timed region reports, and the reference arm,
which runs on rank 0 only while the other ranks exit at once. The transform
itself runs replicas only (no collective on the data path)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
rank = dist.get_rank()
m = bench._max_over_ranks(1.5 + rank, "cpu")
print(json.dumps({"rank": rank, "max": m}), flush=True)
dist.barrier()
sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
            "--workload", "tubes32_no42"]
rc = bench.main()
dist.barrier()
dist.destroy_process_group()
sys.exit(rc)
"""


def test_two_ranks_max_and_reference_arm():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2",
                   RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            p.kill()
            pytest.fail("rank timed out")
        assert p.returncode == 0, e[-2000:]
        outs.append([json.loads(l) for l in o.splitlines() if l.startswith("{")])
    for r, lines in enumerate(outs):
        assert lines[0] == {"rank": r, "max": 2.5}
    # rank 0 alone prints the reference line; rank 1 did no work
    assert len(outs[1]) == 1
    ref = outs[0][1]
    assert ref["impl"] == "reference" and ref["n_gpus"] == 2 and ref["value"] > 0
    assert ref["e2e"]["h2d_bytes_per_step"] == 0 and ref["cpu_baseline"]["kind"] == "oracle"
    assert ref["config"]["workload"] == "tubes32_no42" and ref["config"]["n_o"] == 42
    assert ref["cpu_baseline"]["cores"] == min(os.cpu_count(), 42)
