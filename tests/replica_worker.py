"""One rank of the two-process replica test (run by test_replicas.py): the
bench's process-group setup, barrier and reductions over gloo on the CPU."""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import bench  # noqa: E402


def main():
    w, r, _, pg = bench.dist_setup(argparse.Namespace(impl="gb300"), backend="gloo")
    cpu = torch.device("cpu")
    # rank r processed (r + 1) * 1000 units in (r + 1) seconds
    rate, tmax = bench.replica_rate(pg, (r + 1) * 1000.0, float(r + 1), cpu)
    bench.barrier(pg)
    print(json.dumps({"rank": r, "world": w, "rate": rate, "tmax": tmax, "seed": bench.replica_seed(2, r)}))
    pg.destroy_process_group()


if __name__ == "__main__":
    main()
