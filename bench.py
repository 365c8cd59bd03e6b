#!/usr/bin/env python3
"""Throughput of the hybrid LB/FD step on GB300.

Workload (default, cube384): the 3D form of the method, D3Q19 on 384^3 sites,
FP32 state (populations stored as deviations from w_i n0), periodic in x and
y, cold walls at z = 0 and 383 (bounce-back, T_w = 0.5), Tc = 1, T0 = 1.1,
b = 1, kappa = -0.025, c = 0.02, Gamma = 0.05, xi = 1e-3, tau = 0.6, phi
i.i.d. uniform in [-0.05, 0.05] (synthetic, seeded).  One benchmark step is
one time step of the method (one lf_step(ctx, 1) call: the three passes of
the 3D step).  The state (2 x 9.5 GB) is far larger than the 129 MB L2.

prec1024 is the 2D precision form (D2Q9, 1024 x 1024, xi = 1e-3, tau = 1, one
fused kernel per step); its state (2 x 44 MiB) fits in L2, so a 256 MiB buffer
is written (and another read) before every timed step.  Each step is timed
alone with CUDA events on the library's stream.

Metric: MLUPS = 1e-6 x sites x steps / s (million lattice-site updates per
second), whole job over all ranks.  --impl reference times the FP64 CPU oracle
on the host cores instead (the only reference this method has).
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

BYTES_PER_SITE = {("fp32", 2): 88, ("fp64", 2): 176, ("fp32", 3): 168, ("fp64", 3): 336}
METRIC = "coupled LB+FD MLUPS"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ranks():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over all ranks (every rank gets it); x itself
    without an initialised process group of more than one rank."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput in millions of units per second: the units of all
    ranks (each rank runs its own replica) over the slowest rank's time."""
    return 1e-6 * units_per_rank * steps * world / seconds


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            import atexit
            atexit.register(self.__exit__)   # never leave the sampler running
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def window(self, t0, t1):
        """keep only the samples taken between t0 and t1 (host clock)."""
        self.lines = [(ts, ln) for ts, ln in self.lines if t0 <= ts <= t1]

    def summary_over(self, timed, run, min_samples=5):
        """Clock summary of the timed window (t0, t1) when it holds at least
        `min_samples` samples, else of the whole GPU run (warm-up, timed
        steps and the end-to-end leg), which short timed regions need."""
        keep = self.lines
        self.window(*timed)
        out = self.summary()
        out["window"] = "timed steps"
        if out["samples"] < min_samples:
            self.lines = [(ts, ln) for ts, ln in keep if run[0] <= ts <= run[1]]
            out = self.summary()
            out["window"] = "whole GPU run (warm-up, timed steps, end-to-end leg)"
        self.lines = keep
        return out

    def __exit__(self, *a):
        if self.proc and self.proc.poll() is None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(nx, ny, xi, seconds=10.0, max_steps=10000, d=2, nz=1, tau=1.0, stencil=0):
    """The FP64 CPU oracle as it stands on a bounded sample: steps of an
    nx x ny (x nz) lattice with the workload's physics, for about `seconds`."""
    from oracle import oracle as O

    cfg = O.make_cfg(d=d, nx=nx, ny=ny, nz=nz, xi=xi, tau=tau, stencil=stencil)
    st = O.init(cfg)
    st = O.run(st, 1)   # warm: compile/load, first touch
    steps, t0 = 0, time.perf_counter()
    chunk = 1
    while time.perf_counter() - t0 < seconds and steps < max_steps:
        st = O.run(st, chunk)
        steps += chunk
        el = time.perf_counter() - t0
        if el < seconds / 4:
            chunk *= 2
    el = time.perf_counter() - t0
    return 1e-6 * nx * ny * nz * steps / el, steps, el, O.threads()


def run_reference(args):
    """The oracle as it stands, on the host cores, on a bounded sample of the
    workload: 256x256 of the 2D quench, 64^3 of the 3D one (same physics and
    stencils)."""
    rank, world, _ = ranks()
    if rank != 0:
        return 0
    if args.workload in ("ens96", "sur256"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle times single lattices; the ensemble and "
                          "surrogate workloads have no CPU reference arm (their baselines are the single-run GPU "
                          "path, reported in their own lines)"}), flush=True)
        return 0
    from oracle import oracle as O

    iso = int(args.stencil == "isotropic")
    if args.workload == "cube384":
        d, nx, ny, nz, tau = 3, 64, 64, 64, 0.6
        full = f"cube384: 3D D3Q19 lamellar quench between cold walls (z), sampled as {nx}x{ny}x{nz} per step"
    else:
        d, nx, ny, nz, tau = 2, 256, 256, 1, 1.0
        full = f"prec1024: 2D D2Q9 lamellar quench between cold walls, sampled as {nx}x{ny} per step"
    if iso:
        full += ", isotropic stencils"
    cfg = O.make_cfg(d=d, nx=nx, ny=ny, nz=nz, xi=args.xi, tau=tau, stencil=iso)
    st = O.init(cfg)
    for _ in range(args.warmup):
        st = O.run(st, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = O.run(st, 1)
    el = time.perf_counter() - t0
    sites = nx * ny * nz
    value = 1e-6 * sites * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": full, "sites_per_step": sites, "grid": [nx, ny, nz][:d], "xi": args.xi, "tau": tau},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": O.threads(), "kind": "oracle",
                         "sample": f"{args.steps} FP64 oracle steps of a {'x'.join(map(str, [nx, ny, nz][:d]))} "
                                   f"lattice (same physics as the full workload), OpenMP over rows"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def traffic_for(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it still
    describes the current kernel source."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        j = json.load(fh)
    ent = j.get(kernel_key)
    if not ent:
        return None
    srcs = ent["source"] if isinstance(ent["source"], list) else [ent["source"]]
    data = b"".join(open(os.path.join(ROOT, s_), "rb").read() for s_ in srcs)
    h = hashlib.sha256(data).hexdigest()[:16]
    return ent["dram_bytes_per_launch"] if h == ent.get("source_sha256_16") else None


def run_ensemble(args):
    """96 independent runs (mixed sizes, xi, tau): batched (one graph-replayed
    persistent launch per step) against the same runs stepped one after
    another by lf_step; identical results, compared at the end."""
    import numpy as np
    import torch

    from paper_1102_3094_gb300 import lf, synth

    rank, world, local = ranks()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:                       # one replica of the whole ensemble per GPU
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    stream = torch.cuda.Stream(dev)
    members = synth.ensemble_members()
    if args.stencil == "isotropic":
        members = [dict(m, stencil="isotropic") for m in members]
    sites = sum(m["nx"] * m["ny"] for m in members)
    with torch.cuda.stream(stream):
        ens = lf.Ensemble(members, stream=stream)
        t0 = time.time()
        ens.tune(reps=5)
        tune_s = time.time() - t0
        singles = [lf.Lattice(precision="fp32", stream=stream, **m) for m in members]
        for r, s_ in enumerate(singles):
            s_.set_variant("march2", ens.rows(r))   # same kernel and row split as the batch
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ens.step(args.warmup)
        for s_ in singles:
            s_.step(args.warmup)
        torch.cuda.synchronize(dev)
        clk = Clocks(local)
        with clk:
            time.sleep(0.5)
            tb = time.time()
            ev[0].record(stream)
            ens.step(args.steps)
            ev[1].record(stream)
            ev[2].record(stream)
            for s_ in singles:
                s_.step(args.steps)
            ev[3].record(stream)
            torch.cuda.synchronize(dev)
            te = time.time()
        clk.window(tb, te + 0.15)
        t_batch = max_over_ranks(ev[0].elapsed_time(ev[1]) / 1e3, dev)
        t_seq = max_over_ranks(ev[2].elapsed_time(ev[3]) / 1e3, dev)
        identical, nonfinite = True, 0
        for r in range(len(members)):
            a = ens.run(r).get("phi", "fp32")
            b = singles[r].get("phi", "fp32")
            identical &= bool(np.array_equal(a, b, equal_nan=True))
            nonfinite += int(not np.isfinite(a).all())
    value = job_rate(sites, args.steps, world, t_batch)
    peak, peak_kind = peaks()
    achieved = 88 * sites * args.steps / t_batch / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_batch / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ens96: 96 independent 2D runs, 24 each of 128^2, 256^2, 384^2, 512^2, xi "
                               "log-uniform in [1e-4, 1], tau in {0.6, 1, 3}, one persistent launch per step "
                               "replayed from a CUDA graph, tuned segment heights"
                               + (", isotropic 9-point stencils (tile items)" if args.stencil == "isotropic" else ""),
                   "sites_per_step": sites, "l2": "inputs (1 GB of state) larger than L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_kind": peak_kind, "algorithmic_bytes_per_site": 88,
                     "kernel": ("k_ens_tile2d_iso" if args.stencil == "isotropic" else "k_ens_march2d")
                               + " (+ k_ens_tsub2d for runs with xi/nsub sub-steps)"},
        "batched_vs_sequential": {"t_batched_s": t_batch, "t_sequential_s": t_seq, "speedup": t_seq / t_batch,
                                  "bit_identical_phi": identical, "tune_s": tune_s,
                                  "runs_nonfinite": nonfinite,
                                  "note": "runs with tau = 0.6 and fast quenches (xi above ~0.05) diverge for the "
                                          "method itself at these parameters (the CPU oracle diverges the same way)"},
        "clocks": clk.summary(),
    }
    if world > 1:
        line["config"]["parallelism"] = f"replicas x{world} (the whole ensemble on every GPU)"
    if rank == 0:
        print(json.dumps(line), flush=True)
    ens.close()
    for s_ in singles:
        s_.close()
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()
    return 0


def run_surrogate(args):
    """Learned surrogate at 256 x 256: trajectories of the plain solver (an
    ensemble, xi log-uniform in [1e-4, 1]) -> (state, state K steps later)
    pairs; training on the tensor-core kernels; then the same number of steps
    of a fresh run done plain-only and interleaved (surrogate windows checked by
    plain shadow windows), time-to-solution and S(k) error compared."""
    import numpy as np
    import torch

    from paper_1102_3094_gb300 import lf

    rank, world, local = ranks()
    if rank != 0:
        return 0        # a single-GPU workload: the other ranks of a multi-GPU launch have no work
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    NY = NX = 256
    K = 50
    rng = np.random.default_rng(2011)
    nruns, nwin, warm = args.sur_runs, args.sur_windows, 400
    members = [dict(nx=NX, ny=NY, xi=float(10 ** rng.uniform(-4, 0)), tau=1.0, seed=500 + i) for i in range(nruns)]
    with torch.cuda.stream(stream):
        t0 = time.time()
        ens = lf.Ensemble(members, stream=stream)
        ens.step(warm)
        xs, ys = [], []

        def snap():
            return [torch.stack([ens.run(r).get(n, "fp32", device=True) for n in ("phi", "T", "ux", "uy")])
                    for r in range(nruns)]
        prev = snap()
        for w in range(nwin):
            ens.step(K)
            cur = snap()
            for r in range(nruns):
                if torch.isfinite(prev[r]).all() and torch.isfinite(cur[r]).all():
                    xs.append(prev[r])
                    ys.append(cur[r])
            prev = cur
        X, Y = torch.stack(xs), torch.stack(ys)
        ens.close()
        # pairs whose velocity left the LB's low-Mach range are diverging runs
        # (fast quenches at these parameters): not training material
        umax = torch.maximum(X[:, 2:].abs().amax(dim=(1, 2, 3)), Y[:, 2:].abs().amax(dim=(1, 2, 3)))
        good = umax < 0.2
        n_dropped = int((~good).sum())
        X, Y = X[good], Y[good]
        # held-out windows: every 8th pair
        hold = torch.zeros(X.shape[0], dtype=torch.bool)
        hold[::8] = True
        Xv, Yv = X[hold.to(dev)], Y[hold.to(dev)]
        X, Y = X[~hold.to(dev)], Y[~hold.to(dev)]
        t_data = time.time() - t0
        # inputs centred on the data mean; every channel scaled by the spread of
        # its K-step change, so all four channels weigh alike in the loss
        offset = X.permute(1, 0, 2, 3).reshape(4, -1).mean(dim=1).cpu().numpy()
        scale = (Y - X).permute(1, 0, 2, 3).reshape(4, -1).std(dim=1).clamp_min(1e-6).cpu().numpy()
        B = 8
        sur = lf.Surrogate(NY, NX, B, scale=scale, offset=offset, seed=7, stream=stream)
        sur.set_clip(1.0)
        npairs = X.shape[0]
        gen = torch.Generator().manual_seed(0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        losses = []
        ev[0].record(stream)
        for it in range(args.sur_iters):
            lr = args.sur_lr * 0.5 * (1 + math.cos(math.pi * it / args.sur_iters))
            idx = torch.randint(0, npairs, (B,), generator=gen).to(dev)
            l = sur.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr)
            if it % 250 == 0 or it == args.sur_iters - 1:
                losses.append((it, l))
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        t_train = ev[0].elapsed_time(ev[1]) / 1e3
        # held-out accuracy against keeping the state unchanged, S(k) by the library
        probe = lf.Lattice(nx=NX, ny=NY, precision="fp32", xi=1e-2, tau=1.0, seed=1, stream=stream, device=dev)

        def sk(phi):
            probe.set("phi", phi)
            d_ = probe.diag()
            return d_["k_peak"], d_["s_peak"]

        def sk_err(a, b):
            (ka, sa), (kb, sb) = sk(a), sk(b)
            return max(abs(ka / kb - 1), abs(sa / sb - 1))
        ho = {"pairs": int(Xv.shape[0]), "phi_l2": [], "sk": [], "persist_phi_l2": [], "persist_sk": []}
        for i in range(Xv.shape[0]):
            yp = sur.predict(Xv[i:i + 1].contiguous())[0]
            yt = Yv[i]
            ho["phi_l2"].append(float((yp[0] - yt[0]).norm() / yt[0].norm()))
            ho["persist_phi_l2"].append(float((Xv[i, 0] - yt[0]).norm() / yt[0].norm()))
            ho["sk"].append(sk_err(yp[0].contiguous(), yt[0].contiguous()))
            ho["persist_sk"].append(sk_err(Xv[i, 0].contiguous(), yt[0].contiguous()))
        probe.close()
        heldout = {k: (float(np.mean(v)) if isinstance(v, list) else v) for k, v in ho.items()}
        heldout.update({k + "_median": float(np.median(v)) for k, v in ho.items() if isinstance(v, list)})
        # evaluation run: fresh state, same physics, xi in the middle of the range
        ev_kw = dict(nx=NX, ny=NY, precision="fp32", xi=1e-2, tau=1.0, seed=9001, stream=stream, device=dev)
        plain = lf.Lattice(**ev_kw)
        hyb = lf.Lattice(**ev_kw)
        plain.step(warm)
        hyb.step(warm)
        torch.cuda.synchronize(dev)
        nsteps = args.sur_eval_windows * K
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        plain.step(nsteps)
        e[1].record(stream)
        torch.cuda.synchronize(dev)
        t_plain = e[0].elapsed_time(e[1]) / 1e3
        t1 = time.time()
        try:
            rep = sur.run(hyb, K, args.sur_eval_windows, args.sur_shadow_every, 0.02)
            run_error = None
        except lf.LFError as ex:      # e.g. the solver diverging after an accepted prediction
            rep, run_error = {}, str(ex)
        t_hyb = time.time() - t1
        dp, dh = plain.diag(), hyb.diag()
        pp, ph = plain.get("phi", "fp32"), hyb.get("phi", "fp32")
        l2 = float(np.linalg.norm(ph - pp) / np.linalg.norm(pp))
    final_sk_err = max(abs(dh["k_peak"] / dp["k_peak"] - 1), abs(dh["s_peak"] / dp["s_peak"] - 1))
    sites = NX * NY
    line = {
        "metric": METRIC + " (surrogate-interleaved time to solution)", "value": 1e-6 * sites * nsteps / t_hyb,
        "unit": "MLUPS", "n_gpus": 1, "steps": nsteps, "warmup": warm, "ms_per_step": 1e3 * t_hyb / nsteps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16/f32", "data": "synthetic",
        "config": {"workload": "sur256: 256x256 lamellar quench, 6-layer 64-channel residual CNN advancing "
                               f"(phi, T, ux, uy) by K={K} steps, trained on {npairs} pairs from {nruns} solver "
                               "trajectories (xi log-uniform in [1e-4, 1]); evaluation at xi = 1e-2",
                   "train_iters": args.sur_iters, "batch": B, "lr": args.sur_lr, "lr_schedule": "cosine",
                   "grad_clip": 1.0, "pairs_dropped_umax": n_dropped,
                   "shadow_every": args.sur_shadow_every, "threshold": 0.02},
        "surrogate": {"t_data_s": t_data, "t_train_s": t_train, "losses": losses, "heldout": heldout,
                      "report": rep, "run_error": run_error,
                      "t_plain_only_s": t_plain, "t_interleaved_wall_s": t_hyb,
                      "speedup_vs_plain": t_plain / t_hyb, "final_phi_rel_l2_vs_plain": l2,
                      "final_sk_peak_err_vs_plain": final_sk_err},
    }
    print(json.dumps(line), flush=True)
    for o in (plain, hyb, sur):
        o.close()
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_1102_3094_gb300 import lf

    rank, world, local = ranks()
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    prec = args.precision
    if args.workload == "cube384":
        d, nx, ny, nz = 3, args.size3, args.size3, args.size3
        tau = 0.6
    else:
        d, nx, ny, nz = 2, args.size, args.size, 1
        tau = 1.0
    sim = lf.Lattice(d=d, nx=nx, ny=ny, nz=nz, precision=prec, xi=args.xi, tau=tau, seed=1 + rank, stream=stream,
                     device=dev)
    variant = args.variant
    if variant == "auto":
        variant = "split3" if d == 3 else ("march2" if prec == "fp32" else "march")
    sim.set_variant(variant, args.tune)
    iso = args.stencil == "isotropic"
    if iso:
        sim.set_stencil("isotropic")        # 2D: the tile kernel; 3D: the variant set (three passes by default)
        if d == 2:
            variant = "tile"
    N = nx * ny * nz
    # The compact 3D step at these parameters goes non-finite after about 150
    # steps (the FP64 oracle too), so the 3D workload restores its initial quench
    # every `restore` steps, between the timed events: every timed step then
    # advances a finite state a few dozen steps after the quench.
    restore = args.restore_every if args.restore_every is not None else (100 if d == 3 else 0)
    state0 = None
    if restore > 0:
        state0 = {k: sim.get(k, device=True) for k in ("pop", "phi", "T")}
        torch.cuda.synchronize(dev)
    n_restores = 0

    def restore_state():
        for k_, v_ in state0.items():
            sim.set(k_, v_)                 # one unpack kernel per field, on the library stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_rd = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev) if args.flush == "write+read" else None
    flush_sum = torch.zeros((), dtype=torch.float32, device=dev)

    def l2_flush(v):
        # evict the state from L2 by writing 256 MiB; with write+read, then
        # read another 256 MiB so the flush's dirty lines are written back
        # before the timed step instead of during it
        flush.fill_(v)
        if flush_rd is not None:
            torch.sum(flush_rd, dim=0, out=flush_sum)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            tdist.barrier()
        torch.cuda.synchronize(dev)

    # nvidia-smi samples the clocks from before the warm-up to the end of the
    # end-to-end leg; the line reports the timed window, or the whole run when
    # the timed window is too short to hold enough samples
    clk = Clocks(local)
    clk.__enter__()
    time.sleep(0.5)                          # let the sampler start
    t_run0 = time.time()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            l2_flush(1.0)
            sim.step(1)
    barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_begin = time.time()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            if restore > 0 and k % restore == 0:
                restore_state()
                n_restores += 1
            l2_flush(float(k))
            starts[k].record(stream)
            sim.step(1)
            ends[k].record(stream)
    barrier()
    t_end = time.time()
    times_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = max_over_ranks(sum(times_ms) / 1e3, dev)
    dg = sim.diag()
    value = job_rate(N, args.steps, world, total_s)
    ms = 1e3 * total_s / args.steps
    bps = BYTES_PER_SITE[(prec, d)]
    peak, peak_kind = peaks()
    passes = 3 if (d == 3 and variant == "split3") else 1
    launches_per_step = passes + (lf.lf_nsub(args.xi, d) - 1 if args.xi not in (0.0, math.inf) else 0)
    # the three-pass 3D step is measured as a whole: algorithmic bytes of the
    # step over the step time
    per_kernel = 1 if passes > 1 else launches_per_step
    kernel_ms = statistics.mean(times_ms) / per_kernel
    achieved = bps * N / (kernel_ms * 1e-3) / 1e9
    if d == 3:
        kname = "k_force3d+k_lb3d+k_phi3d" if variant == "split3" else "k_march3d"
    else:
        kname = {"march": "k_march2d", "march2": "k_march2d_x2", "tile": "k_step2d"}[variant]
    if iso:
        kname += "_iso"                     # the ISO instantiation of the tile / fused kernel
    if kname == "k_march2d_x2" and prec == "fp64":
        kname = "k_march2d"                 # the packed kernel is FP32 only
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_for(f"{kname}_{prec}_{nx}"), "peak_kind": peak_kind,
            "algorithmic_bytes_per_site": bps,
            "kernel": kname + (" (three passes; bytes and time of the whole step)" if passes > 1
                               else " (fused phi-chain + LB + FD)"),
            "kernel_ms_mean": kernel_ms, "kernel_ms_median": statistics.median(times_ms) / per_kernel}

    # ---- end to end through the C ABI with host buffers ---------------------
    e2e = None
    if args.e2e_steps > 0:
        tdt = torch.float32 if prec == "fp32" else torch.float64
        shp = sim.shape
        pop_h = torch.empty((sim.Q,) + shp, dtype=tdt, pin_memory=True)
        phi_h = torch.empty(shp, dtype=tdt, pin_memory=True)
        T_h = torch.empty(shp, dtype=tdt, pin_memory=True)
        out_h = torch.empty(shp, dtype=tdt, pin_memory=True)
        es = pop_h.element_size()
        lf.lf_fields(sim.ctx, lf.FIELDS["pop"], pop_h.data_ptr(), pop_h.numel() * es, False)
        lf.lf_fields(sim.ctx, lf.FIELDS["phi"], phi_h.data_ptr(), phi_h.numel() * es, False)
        lf.lf_fields(sim.ctx, lf.FIELDS["T"], T_h.data_ptr(), T_h.numel() * es, False)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            lf.lf_fields_set(sim.ctx, lf.FIELDS["pop"], pop_h.data_ptr(), pop_h.numel() * es, False)
            lf.lf_fields_set(sim.ctx, lf.FIELDS["phi"], phi_h.data_ptr(), phi_h.numel() * es, False)
            lf.lf_fields_set(sim.ctx, lf.FIELDS["T"], T_h.data_ptr(), T_h.numel() * es, False)
            lf.lf_step(sim.ctx, 1)
            lf.lf_fields(sim.ctx, lf.FIELDS["phi"], out_h.data_ptr(), out_h.numel() * es, False)
        el = max_over_ranks(time.perf_counter() - t0, dev)
        torch.cuda.synchronize(dev)
        e2e = {"value": job_rate(N, args.e2e_steps, world, el), "unit": "MLUPS",
               "h2d_bytes_per_step": (sim.Q + 2) * N * es, "d2h_bytes_per_step": N * es,
               "steps": args.e2e_steps,
               "what": "per step: lf_fields_set of f, phi, T from pinned host, lf_step(1), lf_fields of phi to "
                       "pinned host"}

    t_run1 = time.time()
    clk.__exit__(None, None, None)
    clocks = clk.summary_over((t_begin, t_end + 0.1), (t_run0, t_run1 + 0.1))
    cpu = None
    if rank == 0 and args.cpu_seconds > 0:
        if d == 3:
            rate, steps, el, cores = oracle_rate(64, 64, args.xi, seconds=args.cpu_seconds, d=3, nz=64, tau=tau,
                                                 stencil=int(iso))
            smp = "64x64x64"
        else:
            rate, steps, el, cores = oracle_rate(256, 256, args.xi, seconds=args.cpu_seconds, stencil=int(iso))
            smp = "256x256"
        cpu = {"value": rate, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{steps} FP64 oracle steps of a {smp} lattice with the workload's physics "
                         f"({el:.1f} s)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": (f"prec1024: 2D D2Q9 lamellar quench between cold walls, {nx}x{ny}, "
                                    if d == 2 else
                                    f"cube384: 3D D3Q19 lamellar quench between cold walls (z), {nx}x{ny}x{nz}, ")
                                   + f"{prec.upper()} state (deviation populations), xi={args.xi}, tau={tau}"
                                   + ((", isotropic 9-point stencils" if d == 2 else ", isotropic 19-point stencils")
                                      if iso else ""),
                       "sites": N, "l2": ("flushed before every timed step (256 MiB write"
                                          + (", then a 256 MiB read so no dirty flush lines are written back "
                                             "inside the timed step" if args.flush == "write+read" else "")
                                          + "); each step timed alone with CUDA events on the library stream"),
                       "parallelism": f"replicas x{world} (one independent lattice per GPU)"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps * launches_per_step + 3 * n_restores,
            "restores": ({"every": restore, "count": n_restores, "launches": 3 * n_restores,
                          "what": "lf_fields_set of f, phi, T from a device copy of the initial state, "
                                  "between the timed events"} if restore > 0 else None),
            "clocks": clocks,
            "diag_after": {"mass": dg["mass"], "mach": dg["mach"], "rc": dg["rc"]},
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if dist:
        tdist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["prec1024", "cube384", "ens96", "sur256"], default="cube384")
    ap.add_argument("--sur-runs", type=int, default=32)
    ap.add_argument("--sur-windows", type=int, default=20)
    ap.add_argument("--sur-iters", type=int, default=3000)
    ap.add_argument("--sur-lr", type=float, default=1e-3)
    ap.add_argument("--sur-eval-windows", type=int, default=40)
    ap.add_argument("--sur-shadow-every", type=int, default=4)
    ap.add_argument("--size", type=int, default=1024, help="2D lattice side (prec1024)")
    ap.add_argument("--size3", type=int, default=384, help="3D lattice side (cube384)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--xi", type=float, default=1e-3)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--restore-every", type=int, default=None,
                    help="restore the initial state every R timed steps, outside the timed events "
                         "(default: 100 in 3D, never in 2D; 0 = never)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--variant", choices=["auto", "march", "tile", "march2", "split3"], default="auto",
                    help="step kernel variant (all compute the same step); auto = the library's default "
                         "(2D FP32: march2, 2D FP64: march, 3D: split3)")
    ap.add_argument("--flush", choices=["write", "write+read"], default="write+read",
                    help="L2 eviction between timed steps (2D and 3D single-lattice workloads)")
    ap.add_argument("--tune", type=int, default=0, help="march: rows per CTA segment (0 = automatic)")
    ap.add_argument("--stencil", choices=["compact", "isotropic"], default="compact",
                    help="finite-difference stencils (isotropic: the 2D tile kernel; in 3D the chosen variant)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ens96":
        return run_ensemble(args)
    if args.workload == "sur256":
        return run_surrogate(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
