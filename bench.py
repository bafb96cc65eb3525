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
                  [--workload cavity30|cavity20|sphere|capsule] [--no-couple]
  python bench.py --convergence | --rconv

--impl reference times the CPU oracle on a bounded sample of the same
workload.  Under torchrun every rank runs an independent replica (its own
seed) on its own GPU; value is the units of all ranks over the slowest rank's
time.  The default line (one GPU, with the coupling) also carries the
metric's second part under "convergence": the time-to-converged-field
experiment (plain DSMC, DIG, DIG with the learned closure) on the Kn = 0.001
cavity, run after the timed region; --convergence prints only that experiment
in full, --no-convergence leaves it out.
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


def read_solve_flops():
    """Executed FP64 FLOPs (DADD + DMUL + 2 DFMA thread instructions, ncu) per
    cell and synthetic-solver iteration, from the committed summary, if the
    coupling kernels' source is still the one that was counted (else None)."""
    import hashlib

    src = os.path.join(ROOT, "paper_2607_08195_gb300", "csrc", "dig_couple.cu")
    prof = os.path.join(ROOT, "profiles", "synthetic_solver-cavity30-Kn0.01.md")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        fields = dict(l.split(":", 1) for l in open(prof)
                      if l.startswith(("kernel_source_sha256_16:", "fp64_flops_per_cell_iteration:")))
        if fields["kernel_source_sha256_16"].strip() == h:
            return float(fields["fp64_flops_per_cell_iteration"])
    except Exception:
        pass
    return None


# FP64 peak of the part: ncu's sm__sass_thread_inst_executed_op_dfma_pred_on
# peak_sustained is 2 per SM and cycle; 152 SMs x 2 FMA x 2 FLOP x 2.07 GHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07


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


def dist_setup(args, backend=None):
    """Replicas: one process per GPU (torchrun's RANK / LOCAL_RANK /
    WORLD_SIZE); the process group only carries the barrier around the timed
    region and the reductions of the timings and unit counts."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        if backend is None:
            backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def replica_seed(base: int, rank: int) -> int:
    """Each replica runs the same workload with its own seed."""
    return base + rank


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


def allreduce_sum(pg, x, device):
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def replica_rate(pg, units: float, seconds: float, device):
    """Whole-job rate of independent replicas: the units all ranks processed
    over the slowest rank's time (weak scaling); returns (rate, max seconds)."""
    tmax = allreduce_max(pg, seconds, device)
    return allreduce_sum(pg, units, device) / tmax, tmax


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


def centreline_map(scen):
    """Profile point of every tet for the two centreline profiles of the
    cavity: u_x against y (hexahedra of the central half in x and z) and u_y
    against x (central half in y and z).  The Kuhn tets of a hexahedron are
    consecutive (6 per hex, hex-major in i, j, k = x, y, z order).  Returns
    (index into the u_x profile or -1, index into the u_y profile or -1, nh)."""
    import numpy as np

    nt = len(scen.mesh.tets)
    nh = round((nt // 6) ** (1.0 / 3.0))
    h = np.arange(nt) // 6
    i, j, k = h // (nh * nh), (h // nh) % nh, h % nh
    mid = lambda a: (a >= nh // 4) & (a < nh - nh // 4)
    pu = np.where(mid(i) & mid(k), j, -1)
    pv = np.where(mid(j) & mid(k), i, -1)
    return pu, pv, nh


def _cavity_tools(scen):
    """Mass weights, centreline map and field readers of a cavity scenario."""
    import numpy as np

    from paper_2607_08195_gb300 import dig

    P = scen.mesh.nodes[scen.mesh.tets]
    vol = np.abs(np.einsum("ni,ni->n", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6.0
    pu, pv, nh = centreline_map(scen)

    def profiles(g, which=dig.PHI_EWMA):
        """Mass-weighted centreline profiles (u_x(y), u_y(x)) of a moving
        average or cumulative field: 2 nh points."""
        m = g.moments(which | dig.MACRO)
        w = m[:, 1] * vol
        out = []
        for idx, q in ((pu, 2), (pv, 3)):
            sel = idx >= 0
            den = np.bincount(idx[sel], w[sel], nh)
            out.append(np.bincount(idx[sel], w[sel] * m[sel, q], nh) / np.maximum(den, 1e-300))
        return np.concatenate(out)

    def velocity(g, which):
        return g.moments(which | dig.MACRO)[:, 2:5]

    return vol, profiles, velocity


def _timed(f):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(torch.cuda.current_stream())
    r = f()
    e1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1) * 1e-3


def convergence_experiment(args):
    """GPU time to the converged cavity field: plain DSMC vs DIG vs DIG with
    the learned closure, on the near-continuum cavity (20^3 hexahedra, Kn =
    0.001, 3M particles, lid 50 m/s; or, with --conv-workload cavity30, the
    30^3-hexahedra Kn = 0.01 cavity with 8M particles).

    The closure is trained on other flows of the same cavity (lid speeds 30
    and 70 m/s, their own seeds): their windows are its inputs and their
    long-time averages its targets; the GPU seconds spent generating those
    data and training are reported beside the result.  The reference field
    is the cumulative average of a separate long DIG run of the 50 m/s flow;
    every timed run starts from the initial equilibrium.  Returns the result
    object."""
    import numpy as np
    import torch

    from paper_2607_08195_gb300 import dig
    from paper_2607_08195_gb300 import workload as W

    dev = "cuda:0"
    c30 = getattr(args, "conv_workload", "cavity20") == "cavity30"
    base = W.config_c2() if c30 else W.config_c3()
    nhx = 30 if c30 else 20
    kn = base.Kn

    def flow(U_lid, seed):
        return W.cavity_scenario(nhx, base.n_particles, kn, seed, U_lid=U_lid, name=f"{base.name}-lid{U_lid:g}")

    scen = base
    Uw = 50.0
    vol, profiles, _ = _cavity_tools(scen)
    NSC = 200            # DSMC steps per coupling cycle
    WIN = 50             # closure input window (the last WIN steps of a cycle)
    fl = dig.EWMA | dig.WALLFLUX

    def err(prof, ref):
        return float(np.sqrt(np.mean((prof - ref) ** 2)) / Uw)

    def cycle(g, closure):
        if closure:
            g.step(NSC - WIN, fl)
            g.sample(dig.RESET_WINDOW)
            g.step(WIN, fl | dig.WINDOW)
        else:
            g.step(NSC, fl)
        return g.couple()

    def windows(g, X, nwin):
        """nwin closure input rows blocks (50-step windows, four per cycle)
        into X, while the cumulative average runs; returns nothing."""
        n = g.n_tets
        g.sample(dig.RESET_CUMUL)
        w = 0
        while w < nwin:
            g.step(NSC - 4 * WIN, fl | dig.CUMUL)
            for _ in range(4):
                g.sample(dig.RESET_WINDOW)
                g.step(WIN, fl | dig.CUMUL | dig.WINDOW)
                if w < nwin:
                    g.closure_features(dig.PHI_WINDOW, X[w * n:(w + 1) * n])
                    w += 1
            g.couple()

    # 1. training data: other flows of the same cavity
    n = len(scen.mesh.tets)
    train_flows = [(30.0, scen.seed + 100), (70.0, scen.seed + 200)]
    nwin_f = args.conv_windows // len(train_flows)
    X = torch.empty((nwin_f * len(train_flows) * n, 13), dtype=torch.float32, device=dev)
    Y = torch.empty((nwin_f * len(train_flows) * n, 8), dtype=torch.float32, device=dev)
    t_data = 0.0
    for f_i, (U_lid, seed) in enumerate(train_flows):
        g = dig.Solver(flow(U_lid, seed), dev, closure=0)
        g.init()

        def gen():
            for _ in range(args.conv_train_warm):
                cycle(g, False)
            sl = slice(f_i * nwin_f * n, (f_i + 1) * nwin_f * n)
            windows(g, X[sl], nwin_f)
            Y[sl] = g.closure_targets(dig.PHI_CUM, X[sl])

        _, dt = _timed(gen)
        t_data += dt
        g.close()
    # 2. the reference field of the measured flow, and windows of it for the
    #    closure's transfer check (never used for training)
    g = dig.Solver(scen, dev, closure=0)
    g.init()
    warm_fields = []
    for _ in range(args.conv_warm):
        cycle(g, False)
        warm_fields.append(profiles(g))
    nval = 8
    Xt = torch.empty((nval * n, 13), dtype=torch.float32, device=dev)
    windows(g, Xt, nval)
    for _ in range(max(0, args.conv_ref - nval // 4)):
        g.step(NSC, fl | dig.CUMUL)
        g.couple()
    Yt = g.closure_targets(dig.PHI_CUM, Xt)
    ref = profiles(g, dig.PHI_CUM)
    warm_err = [round(err(u, ref), 4) for u in warm_fields][4::5]
    post = []
    for _ in range(args.conv_noise):
        cycle(g, False)
        post.append(err(profiles(g), ref))
    noise = float(np.median(post))
    # 3. training on the other flows (the library's BF16 tensor-core kernels), 90/10 split
    nrow = X.shape[0]
    rng = np.random.default_rng(scen.seed)
    order = torch.from_numpy(rng.permutation(nrow).astype(np.int64)).to(dev)
    X, Y = X[order].contiguous(), Y[order].contiguous()
    ntr = int(0.9 * nrow)
    g.closure_init(scen.seed)
    epochs = args.conv_epochs
    perm = torch.from_numpy(np.stack([rng.permutation(ntr) for _ in range(epochs)]).astype(np.int32)).to(dev)
    losses, t_train = _timed(lambda: g.closure_train(X[:ntr].contiguous(), Y[:ntr].contiguous(), epochs=epochs,
                                                     batch=4096, lr=1e-3, perm=perm))
    Xv, Yv = X[ntr:].contiguous(), Y[ntr:].contiguous()
    mse_net, mse_win = g.closure_loss(Xv, Yv), g.closure_loss(Xv, Yv, identity=True)
    mse_net_t, mse_win_t = g.closure_loss(Xt, Yt), g.closure_loss(Xt, Yt, identity=True)
    params = g.closure_get()
    g.close()
    del X, Y, perm, Xt, Yt
    torch.cuda.empty_cache()

    # 4. timed runs from the initial state
    thr = max(args.conv_threshold, args.conv_threshold_factor * noise)
    HOLD = 5

    def run(kind, ncycles, n_a=1000):
        h = dig.Solver(scen, dev, closure=1 if kind.startswith("dig_net") else 0, n_a=n_a)
        if kind.startswith("dig_net"):
            h.closure_set(params)
        h.init()
        t, hist, tail, fields = 0.0, [], [], []
        for k in range(ncycles):
            if kind == "plain":
                _, dt = _timed(lambda: h.step(NSC, fl))
            else:
                _, dt = _timed(lambda: cycle(h, kind.startswith("dig_net")))
            t += dt
            prof = profiles(h)
            e = err(prof, ref)
            hist.append((round(t, 3), round(e, 4), (k + 1) * NSC))
            fields.append(prof)
            if k >= ncycles - 20:
                tail.append(prof)
        h.close()
        torch.cuda.empty_cache()

        # converged: the first checkpoint at or below the threshold whose next
        # HOLD checkpoints also average at or below it
        def first_hold(errs):
            for k in range(len(errs) - HOLD + 1):
                if errs[k] <= thr and np.mean(errs[k:k + HOLD]) <= thr:
                    return k
            return None

        k_ref = first_hold([x[1] for x in hist])
        hit = None if k_ref is None else hist[k_ref]
        own = np.mean(tail, axis=0)
        k_own = first_hold([err(f, own) for f in fields[:len(fields) - len(tail)]])
        return {"seconds": None if hit is None else hit[0], "steps": None if hit is None else hit[2],
                "seconds_to_own_final_field": None if k_own is None else hist[k_own][0],
                "own_final_field_error": round(err(own, ref), 4),
                "final_error": hist[-1][1], "mean_error_last_20": round(float(np.mean([x[1] for x in hist[-20:]])), 4),
                "gpu_seconds_run": round(t, 3), "cycles": ncycles,
                "final_profiles": [round(float(x) / Uw, 4) for x in np.mean(tail, axis=0)],
                "error_every_5_cycles": [x[:2] for x in hist[4::5]]}

    na = args.conv_net_na
    res = {"dig_net": run("dig_net", args.conv_cycles, n_a=na), "dig": run("dig", args.conv_cycles),
           f"dig_na{na}": run("dig", args.conv_cycles, n_a=na),
           "dig_net_na1000": run("dig_net", args.conv_cycles, n_a=1000),
           "plain_dsmc": run("plain", args.conv_plain_cycles)}
    sec = res["dig_net"]["seconds"]
    return {
        "metric": "GPU seconds to the converged cavity field", "unit": "s", "higher_is_better": False,
        "value": sec, "workload": scen.name,
        "value_incl_closure_cost": None if sec is None else round(sec + t_data + t_train, 3),
        "methods_config": {"dig_net": f"DIG with the learned closure, n_a = {na}",
                           "dig": "DIG, n_a = 1000", f"dig_na{na}": f"DIG, n_a = {na}",
                           "dig_net_na1000": "DIG with the learned closure, n_a = 1000",
                           "plain_dsmc": "DSMC alone, n_a = 1000"},
        "error": "RMS over the centreline profiles u_x(y) and u_y(x) (moving average, central half of the "
                 "cavity in the other two directions) against the reference profiles, over U_w",
        "threshold": round(thr, 4), "noise_floor": round(noise, 4),
        "reference": f"cumulative average of a separate DIG run of the lid-50 m/s flow over "
                     f"{max(args.conv_ref, nval // 4)} coupling cycles after {args.conv_warm} cycles",
        "reference_profiles": [round(float(x) / Uw, 4) for x in ref],
        "reference_run_error_every_5_cycles": warm_err,
        "methods": res,
        "closure": {"trained_on": [f"lid {u:g} m/s, seed {sd}" for u, sd in train_flows],
                    "train_rows": ntr, "epochs": epochs,
                    "data_gpu_seconds": round(t_data, 3), "train_gpu_seconds": round(t_train, 3),
                    "loss_first_last": [float(losses[0]), float(losses[-1])],
                    "heldout_mse_net": mse_net, "heldout_mse_window_hot": mse_win,
                    "gain_heldout_training_flows": mse_win / max(mse_net, 1e-300),
                    "target_flow_mse_net": mse_net_t, "target_flow_mse_window_hot": mse_win_t,
                    "gain_target_flow": mse_win_t / max(mse_net_t, 1e-300)},
    }


def rconv_experiment(args):
    """The convergence criterion of the 8M-particle Kn = 0.01 cavity (30^3
    hexahedra): plain DSMC for up to 20,000 steps against DIG coupled every
    200 steps (inner solves of N_m = 500, 100 and 50 iterations), each
    sampled into a cumulative average from its first step.
    E_k = |u_k - u_{k-1}|_2 / |u_k|_2 between consecutive 200-step
    checkpoints of the cumulative velocity, over every cell (volume-weighted)
    and over the centreline profiles; a method has converged at the first
    checkpoint where E_k < 1e-3 holds for three checkpoints in a row.
    Returns GPU seconds and steps to that point for each measure (None if
    not reached within 20,000 steps)."""
    import numpy as np

    from paper_2607_08195_gb300 import dig
    from paper_2607_08195_gb300 import workload as W

    scen = W.config_c2()
    vol, profiles, velocity = _cavity_tools(scen)
    NSC, KMAX, TOL, HOLD = 200, args.rconv_checkpoints, 1e-3, 3
    out = {}
    # DIG with the bench's N_m = 500 and with shorter inner solves (the outer
    # iteration does not need the synthetic equations solved far below the
    # noise of their sampled HoT)
    runs = {"plain_dsmc": 500, "dig": 500, "dig_nm100": 100, "dig_nm50": 50}
    for kind, N_m in runs.items():
        g = dig.Solver(scen, "cuda:0", N_m=N_m)
        g.init()
        g.sample(dig.RESET_CUMUL)
        t, prev_u, prev_p, eu, ep, hist = 0.0, None, None, [], [], []
        first = {"field": None, "profiles": None}
        for k in range(KMAX):
            if kind.startswith("dig"):
                _, dt = _timed(lambda: (g.step(NSC, dig.EWMA | dig.WALLFLUX | dig.CUMUL), g.couple()))
            else:
                _, dt = _timed(lambda: g.step(NSC, dig.EWMA | dig.CUMUL))
            t += dt
            u, p = velocity(g, dig.PHI_CUM), profiles(g, dig.PHI_CUM)
            if prev_u is not None:
                eu.append(float(np.sqrt((vol[:, None] * (u - prev_u) ** 2).sum() / (vol[:, None] * u ** 2).sum())))
                ep.append(float(np.linalg.norm(p - prev_p) / np.linalg.norm(p)))
                hist.append((round(t, 3), (k + 1) * NSC, eu[-1], ep[-1]))
                for key, e in (("field", eu), ("profiles", ep)):
                    if first[key] is None and len(e) >= HOLD and all(x < TOL for x in e[-HOLD:]):
                        first[key] = hist[-HOLD]
            prev_u, prev_p = u, p
            if all(v is not None for v in first.values()):
                break
        g.close()
        out[kind] = {"N_m": None if kind == "plain_dsmc" else N_m,
                     "field": None if first["field"] is None else {"seconds": first["field"][0],
                                                                   "steps": first["field"][1]},
                     "profiles": None if first["profiles"] is None else {"seconds": first["profiles"][0],
                                                                         "steps": first["profiles"][1]},
                     "gpu_seconds_run": round(t, 3), "steps_run": hist[-1][1] if hist else 0,
                     "last_E_field": round(eu[-1], 6) if eu else None,
                     "last_E_profiles": round(ep[-1], 6) if ep else None,
                     "E_every_10_checkpoints": [(h[0], h[1], round(h[2], 5), round(h[3], 5)) for h in hist[9::10]]}
    return {"criterion": "E_k = |u_k - u_{k-1}|_2 / |u_k|_2 < 1e-3 on the cumulative velocity at consecutive "
                         "200-step checkpoints, three in a row (field: every cell, volume-weighted; profiles: "
                         "the two centreline profiles)",
            "workload": scen.name, "max_steps": KMAX * NSC, "methods": out}


def closure_timing(args):
    """The learned closure's tensor-core kernels on random rows of a freshly
    initialised network: inference (closure_forward) on n rows, CUDA events
    around 10 launches after 3 warm-up launches; and a training run (20
    epochs of Adam over 2.1M rows, batches of 4096, the convergence
    experiment's shape), timed on the host around the synchronous call.
    Returns the timings."""
    import time

    import numpy as np
    import torch

    from paper_2607_08195_gb300 import dig
    from paper_2607_08195_gb300 import workload as W

    g = dig.Solver(W.config_small(), "cuda:0")
    g.closure_init(3)
    out = []
    flops_row = 2.0 * (13 * 64 + 64 * 64 * 2 + 64 * 8)
    for n in (48_000, 2_000_000, 8_000_000):
        X = torch.randn((n, 13), device="cuda:0")
        Y = torch.empty((n, 8), device="cuda:0")
        for _ in range(3):
            g.closure_forward(X, Y)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(10):
            g.closure_forward(X, Y)
        b.record()
        torch.cuda.synchronize()
        tf = a.elapsed_time(b) / 10
        out.append({"rows": n, "forward_ms": round(tf, 4), "forward_tflops": round(flops_row * n / tf / 1e9, 2)})
    n, ep = 2_100_000, 20
    X = torch.randn((n, 13), device="cuda:0") * 0.5
    Y = torch.randn((n, 8), device="cuda:0") * 0.1
    rng = np.random.default_rng(1)
    perm = torch.from_numpy(np.stack([rng.permutation(n) for _ in range(ep)]).astype(np.int32)).cuda()
    g.closure_train(X, Y, epochs=1, batch=4096, lr=1e-3, perm=perm[:1].contiguous())
    torch.cuda.synchronize()
    t0 = time.time()
    g.closure_train(X, Y, epochs=ep, batch=4096, lr=1e-3, perm=perm)
    torch.cuda.synchronize()
    dt = time.time() - t0
    g.close()
    return {"closure_forward": out,
            "closure_train": {"rows": n, "epochs": ep, "batch": 4096, "seconds": round(dt, 3),
                              "ns_per_row_epoch": round(dt / (n * ep) * 1e9, 2)}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-couple", action="store_true", help="DSMC steps only (no DIG coupling)")
    ap.add_argument("--no-convergence", action="store_true",
                    help="leave the time-to-converged-field experiment out of the default line")
    ap.add_argument("--convergence", action="store_true",
                    help="only the time-to-converged-field experiment (plain DSMC vs DIG vs DIG + learned closure)")
    ap.add_argument("--conv-warm", type=int, default=80)
    ap.add_argument("--conv-train-warm", type=int, default=60,
                    help="cycles each training flow runs before its windows are taken")
    ap.add_argument("--rconv-checkpoints", type=int, default=100,
                    help="200-step checkpoints of the R-conv comparison (100 = 20,000 DSMC steps)")
    ap.add_argument("--no-rconv", action="store_true", help="leave the R-conv comparison out of the default line")
    ap.add_argument("--rconv", action="store_true", help="only the R-conv comparison (plain DSMC vs DIG, 8M cavity)")
    ap.add_argument("--closure-timing", action="store_true",
                    help="only the learned closure's tensor-core inference and training timings")
    ap.add_argument("--conv-windows", type=int, default=44)
    ap.add_argument("--conv-epochs", type=int, default=20)
    ap.add_argument("--conv-cycles", type=int, default=60)
    ap.add_argument("--conv-plain-cycles", type=int, default=160)
    ap.add_argument("--conv-ref", type=int, default=40)
    ap.add_argument("--conv-noise", type=int, default=20)
    ap.add_argument("--conv-workload", default="cavity20", choices=["cavity20", "cavity30"],
                    help="cavity20: Kn 0.001, 50 mean free paths per cell (the experiment); cavity30: Kn 0.01, "
                         "3.3 mean free paths per cell, where plain DSMC is nearly resolved (a check of DIG's field)")
    ap.add_argument("--conv-net-na", type=int, default=50,
                    help="moving-average length n_a of the DIG run with the learned closure")
    ap.add_argument("--conv-threshold", type=float, default=0.02)
    ap.add_argument("--conv-threshold-factor", type=float, default=1.5)
    ap.add_argument("--workload", default="cavity30", choices=["cavity30", "cavity20", "sphere", "capsule"],
                    help="cavity30: 30^3 hexes, Kn 0.01, 8M particles (the benchmark); sphere: Mach 10 argon over a "
                         "sphere, ~2M graded Delaunay tets, 100M particles; capsule: Mach 25 nitrogen over a capsule, "
                         "~8M tets, 1e9 particles; cavity20: 20^3 hexes, "
                         "Kn 0.001, 3M particles (smaller case for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.convergence or args.rconv or args.closure_timing:
        import torch

        torch.cuda.set_device(0)
        fn = convergence_experiment if args.convergence else rconv_experiment if args.rconv else closure_timing
        print(json.dumps(fn(args)), flush=True)
        return 0

    import numpy as np
    import torch

    from paper_2607_08195_gb300 import dig
    from paper_2607_08195_gb300 import workload as W

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    scen = {"cavity30": lambda: W.config_c2(seed=replica_seed(2, rank)),
            "cavity20": lambda: W.config_c3(seed=replica_seed(3, rank)),
            "sphere": lambda: W.config_c4(seed=replica_seed(4, rank)),
            "capsule": lambda: W.config_c5(seed=replica_seed(5, rank))}[args.workload]()
    g = dig.Solver(scen, str(device))
    g.init()
    g.synchronize()
    flags = dig.EWMA | dig.WALLFLUX
    reports = []

    phase_ev = []  # (start, after the DSMC steps, after the coupling) of each timed bench step

    def cycle(timing=0):
        ev = None
        if timing:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(g.stream)
        g.step(N_S, flags | timing)
        if ev:
            ev[1].record(g.stream)
        if not args.no_couple:
            reports.append(g.couple())
        if ev:
            ev[2].record(g.stream)
            phase_ev.append(ev)

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
    value_rate, tmax = replica_rate(pg, float(g.count()) * N_S * args.steps, ms * 1e-3, device)
    ms = tmax * 1e3
    launches = g.launches() - l0
    k_ms, k_n = g.kernel_time()
    N = g.count()
    psteps = N * N_S * args.steps
    value = value_rate
    dsmc_ms = sum(a.elapsed_time(b) for a, b, _ in phase_ev)
    couple_ms = sum(b.elapsed_time(c) for _, b, c in phase_ev)
    phases = {"dsmc_ms_per_bench_step": dsmc_ms / args.steps, "couple_ms_per_bench_step": couple_ms / args.steps,
              "dsmc_particle_steps_per_s": psteps / (dsmc_ms * 1e-3) if dsmc_ms > 0 else None}

    # dominant kernel: the particle pass of one DSMC step (k_order, k_collide,
    # k_move, k_track launched back to back, timed together with CUDA events
    # on the library's stream); algorithmic bytes = read + write of the
    # particle state once per particle-step (x,y,z f64 + vx,vy,vz f32 = 36 B,
    # plus the 4-byte cell id) = 80 B
    alg_bytes_per_pstep = 88.0 if scen.gas.rot_dof > 0 else 80.0  # + I_r (f32) for a diatomic gas
    peak, peak_kind = read_peaks()
    cp_launch_ms = k_ms / max(k_n, 1)
    # passes: n_steps + 1 per dsmc_step call; particle-steps per pass
    psteps_per_launch = psteps / max(k_n, 1)
    achieved = alg_bytes_per_pstep * psteps_per_launch / (cp_launch_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": read_traffic() if args.workload == "cavity30" else None,
                "kernel": "particle pass (k_order+k_collide+k_move+k_track)",
                "peak_kind": peak_kind, "kernel_ms_per_launch": cp_launch_ms, "kernel_share_of_step": k_ms / ms}

    # the coupling: its synthetic solve is bound by the FP64 pipe; executed
    # FP64 FLOPs per cell-iteration (ncu count, committed summary) x cells x
    # the timed couplings' iterations / the couplings' CUDA-event time (S9
    # and S11 included, so slightly low)
    roofline_solve = None
    timed = reports[len(reports) - args.steps:] if reports else []
    fpc = read_solve_flops()
    if timed and couple_ms > 0:
        iters = sum(r["iters"] for r in timed)
        ach = None if fpc is None else fpc * len(scen.mesh.tets) * iters / (couple_ms * 1e-3) / 1e9
        roofline_solve = {"bound": "fp64", "achieved": ach, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                          "frac": None if ach is None else ach / FP64_PEAK_GFLOPS,
                          "peak_kind": "derived: 2 FP64 FMA per SM and cycle x 152 SMs x 2.07 GHz",
                          "flops_per_cell_iteration": fpc, "iterations": iters,
                          "ms_per_iteration": couple_ms / iters if iters else None,
                          "kernel": "synthetic solve (k_cp_*, k_aa_*)"}

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
        e2e_rate, el = replica_rate(pg, float(len(cn)) * N_S * args.steps, t1 - t0, device)
        e2e = {"value": e2e_rate, "unit": "particle-steps/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v_cpu, dt_cpu, st = oracle_sample(scen, steps=3)
        cpu = {"value": v_cpu, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{st} DSMC steps of the {scen.name} workload from its initial state "
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
                       "l2": f"inputs larger than L2 (2 x {40 * scen.n_particles / 1e6:.0f} MB particle buffers)"},
            "roofline": roofline, "roofline_solve": roofline_solve, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "phases": phases,
            "clocks": clk.summary(),
            "couple_last": reports[-1] if reports else None,
        }
    g.close()
    del g
    torch.cuda.empty_cache()
    if rank == 0:
        # the metric's second part: GPU time to the converged cavity field
        # (one GPU, outside the timed region above)
        if world == 1 and args.workload == "cavity30" and not (args.no_convergence or args.no_couple):
            try:
                cv = convergence_experiment(args)
                line["convergence"] = {
                    "metric": cv["metric"], "value": cv["value"], "unit": cv["unit"], "higher_is_better": False,
                    "workload": cv["workload"], "threshold": cv["threshold"], "noise_floor": cv["noise_floor"],
                    "methods": {k: {"config": cv["methods_config"][k], "seconds": r["seconds"], "steps": r["steps"],
                                    "mean_error_last_20": r["mean_error_last_20"]}
                                for k, r in cv["methods"].items()},
                    "value_incl_closure_cost": cv["value_incl_closure_cost"],
                    "closure": {k: cv["closure"][k] for k in ("trained_on", "data_gpu_seconds", "train_gpu_seconds",
                                                              "gain_heldout_training_flows", "gain_target_flow")},
                }
            except Exception as e:  # reported, not fatal for the throughput line
                line["convergence"] = {"error": f"{type(e).__name__}: {e}"}
            if not args.no_rconv:
                try:
                    line["rconv"] = rconv_experiment(args)
                except Exception as e:
                    line["rconv"] = {"error": f"{type(e).__name__}: {e}"}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
