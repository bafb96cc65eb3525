"""Benchmark of the DSMC particle loop (particle-steps/s) on one GB300.

Workload: the argon lid-driven cavity refined to 30x30x30 hexahedra (162,000
Kuhn tets) at Kn = 0.01 with 8,000,000 particles, Maxwellian initial state,
seed 2.  One bench step is one outer DIG cycle (paper Alg. 1): N_s = 200 DSMC
time steps (move with diffuse walls, sort by cell, NTC collisions, sampling,
moving average, wall-flux sampling) followed by one coupling (HoT extraction
and filter, synthetic-equation solve, particle recalibration).  The particle
state (2 x 352 MB) is far larger than L2, so no L2 flush is needed between
steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (the reference of this build) on a
bounded sample of the same workload.  Under torchrun every rank runs an
independent replica (different seed) on its own GPU; value is the sum.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_S = 200  # DSMC steps per bench step (one coupling window of the benchmarked cavity)


def read_traffic():
    """DRAM bytes per particle pass (k_order + k_collide + k_move + k_track of
    one DSMC step) from the committed ncu summary, if the kernel source is
    still the one that was profiled (else None)."""
    import hashlib

    src = os.path.join(ROOT, "paper_2607_08195_gb300", "csrc", "dig_kernels.cu")
    prof = os.path.join(ROOT, "profiles", "particle_pass-cavity30-Kn0.01-8M.md")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        fields = dict(l.split(":", 1) for l in open(prof) if l.startswith(("kernel_source_sha256_16:", "dram_bytes")))
        if fields["kernel_source_sha256_16"].strip() == h:
            return float(fields["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg, device=None):
    if pg is not None:
        if device is not None:
            pg.barrier(device_ids=[device.index])
        else:
            pg.barrier()


def allreduce_max(pg, x, device):
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(scen, seconds_target=12.0, steps=3):
    """Time the CPU oracle (single thread) on `steps` DSMC steps of the
    workload from its initial state; init is not timed."""
    from oracle import orc

    o = orc.Oracle(scen)
    o.init()
    t0 = time.perf_counter()
    o.step(steps, orc.EWMA)
    dt = time.perf_counter() - t0
    o.close()
    return scen.n_particles * steps / dt, dt, steps


def run_reference(args):
    from paper_2607_08195_gb300 import workload as W

    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return 0
    scen = W.config_c2()
    times, vals = [], []
    for i in range(args.warmup + args.steps):
        v, dt, st = oracle_sample(scen, steps=1)
        if i >= args.warmup:
            vals.append(v)
            times.append(dt)
    value = scen.n_particles * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32",
        "data": "synthetic",
        "config": {"workload": scen.name, "particles": scen.n_particles, "tets": len(scen.mesh.tets),
                   "dsmc_steps_per_step": 1},
        "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                         "sample": "1 DSMC step of the 8M-particle cavity per bench step (oracle, single thread)"},
        "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-couple", action="store_true", help="DSMC steps only (no DIG coupling)")
    ap.add_argument("--workload", default="cavity30", choices=["cavity30", "cavity20"],
                    help="cavity30: 30^3 hexes, Kn 0.01, 8M particles (the benchmark); cavity20: 20^3 hexes, "
                         "Kn 0.001, 3M particles (smaller case for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_2607_08195_gb300 import dig
    from paper_2607_08195_gb300 import workload as W

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    scen = W.config_c2(seed=2 + rank) if args.workload == "cavity30" else W.config_c3(seed=3 + rank)
    g = dig.Solver(scen, str(device))
    g.init()
    g.synchronize()
    flags = dig.EWMA | dig.WALLFLUX
    reports = []

    def cycle(timing=0):
        g.step(N_S, flags | timing)
        if not args.no_couple:
            reports.append(g.couple())

    # warm-up steps (untimed)
    for _ in range(args.warmup):
        cycle()
    g.synchronize()
    stream = g.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = g.launches()
    g.kernel_time()  # reset the per-kernel record
    with ClockSampler(local) as clk:
        barrier(pg, device)
        torch.cuda.synchronize(device)
        e0.record(stream)
        for _ in range(args.steps):
            cycle(dig.TIMING)
        e1.record(stream)
        torch.cuda.synchronize(device)
        barrier(pg, device)
    g.synchronize()
    ms = e0.elapsed_time(e1)
    ms = allreduce_max(pg, ms, device)
    launches = g.launches() - l0
    k_ms, k_n = g.kernel_time()
    N = g.count()
    psteps = N * N_S * args.steps
    value = psteps * world / (ms * 1e-3)

    # dominant kernel: the particle pass of one DSMC step (k_order, k_collide,
    # k_move, k_track launched back to back, timed together with CUDA events
    # on the library's stream); algorithmic bytes = read + write of the
    # particle state once per particle-step (x,y,z f64 + vx,vy,vz f32 = 36 B,
    # plus the 4-byte cell id) = 80 B
    alg_bytes_per_pstep = 80.0
    peak, peak_kind = read_peaks()
    cp_launch_ms = k_ms / max(k_n, 1)
    # passes: n_steps + 1 per dsmc_step call; particle-steps per pass
    psteps_per_launch = psteps / max(k_n, 1)
    achieved = alg_bytes_per_pstep * psteps_per_launch / (cp_launch_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": read_traffic(), "kernel": "particle pass (k_order+k_collide+k_move+k_track)",
                "peak_kind": peak_kind, "kernel_ms_per_launch": cp_launch_ms, "kernel_share_of_step": k_ms / ms}

    # end to end through the C ABI with host buffers: pinned host particle
    # state in, N_S DSMC steps, moving-average sums out, every bench step
    e2e = None
    if not args.no_e2e:
        x, v, Ir, cell = g.read()
        hx = torch.from_numpy(x).pin_memory()
        hv = torch.from_numpy(v).pin_memory()
        hc = torch.from_numpy(cell).pin_memory()
        out = torch.empty((g.n_tets, dig.NPHI), dtype=torch.float64).pin_memory()
        xn, vn, cn, on = hx.numpy(), hv.numpy(), hc.numpy(), out.numpy()
        h2d = xn.nbytes + vn.nbytes + cn.nbytes
        d2h = on.nbytes
        g.write(xn, vn, None, cn)
        cycle()
        g.moments(dig.PHI_EWMA, on)
        barrier(pg, device)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g.write(xn, vn, None, cn)
            cycle()
            g.moments(dig.PHI_EWMA, on)
        t1 = time.perf_counter()
        barrier(pg, device)
        el = allreduce_max(pg, t1 - t0, device)
        e2e = {"value": len(cn) * N_S * args.steps * world / el, "unit": "particle-steps/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v_cpu, dt_cpu, st = oracle_sample(scen, steps=3)
        cpu = {"value": v_cpu, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{st} DSMC steps of the 8M-particle cavity from its initial state "
                         f"({dt_cpu:.1f} s, single thread)"}
    if rank == 0:
        line = {
            "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32",
            "data": "synthetic",
            "config": {"workload": scen.name, "particles": scen.n_particles, "tets": len(scen.mesh.tets),
                       "dsmc_steps_per_step": N_S, "parallelism": f"replicas{world}",
                       "coupling": "none" if args.no_couple else f"DIG every {N_S} steps, N_m={g.cfg.N_m}",
                       "l2": "inputs larger than L2 (2 x 320 MB particle buffers)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
            "couple_last": reports[-1] if reports else None,
        }
        print(json.dumps(line), flush=True)
    g.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
