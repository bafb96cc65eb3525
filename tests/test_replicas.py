"""Replicas on several GPUs (one process per GPU, launched by torchrun): the
host-side reductions, run here as two gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_replica_rate_two_gloo_ranks():
    """Two ranks: the whole-job rate is the units of all ranks over the
    slowest rank's time (3000 units / 2 s), the same on every rank; each rank
    gets its own seed."""
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE="2",
                   LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "replica_worker.py")], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    out = []
    for p in procs:
        o, e = p.communicate(timeout=180)
        assert p.returncode == 0, e
        out.append(json.loads(o.strip().splitlines()[-1]))
    out.sort(key=lambda d: d["rank"])
    assert [d["world"] for d in out] == [2, 2]
    for d in out:
        assert d["rate"] == 1500.0 and d["tmax"] == 2.0
    assert out[0]["seed"] != out[1]["seed"]
