#!/usr/bin/env python
"""Throughput of the coupled level-set LB step on GB300: MLUPS and HBM roofline.

Workload (default): 3D D3Q19 rising bubble, 128x128x256 base grid, 2 levels
(finest 256x256x512), bubble radius 16 base cells, density ratio 1000,
viscosity ratio 100, Eo 10, Re 35, FP32 storage (``--storage fp16s`` for the
FP16-storage variant).  A step is one coarse time step of the whole method:
collide-stream on both levels (the finest twice), interface bounce-back,
level-set extension / transport / reinitialisation, classification, curvature,
refill, level transfers and the periodic regrid.

MLUPS = leaf cell updates (sum over levels of leaf cells x 2^level) / time.
The state (2 x 19 x 4 B x ~38 M cells) is far larger than the 129 MB L2, so
no flush is needed between steps.  The collide-stream kernel's duration is
measured with CUDA events on the library stream inside the timed region;
its algorithmic bytes are 2 * Q * sizeof(storage) per leaf cell update.

Multi-GPU: the method is not sharded; with torchrun each rank runs an
independent replica ("replicas only") and the value is the sum over ranks.
``--impl reference`` times the FP64 CPU oracle on a bounded sample.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (leaf cell updates / s), 3D D3Q19 rising bubble, 2 AMR levels"
HBM_FALLBACK = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return HBM_FALLBACK, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


def oracle_error(case, s, steps, storage):
    """The CUDA path on the oracle's case for the same number of coarse steps, against the
    oracle's state: per level rel-L2 of u and max |drho| on leaf cells, max |phi| error,
    leaf masks and phases compared bit for bit."""
    from paper_2601_05936_gb300 import lsb
    c = dict(case, storage=storage)
    g = lsb.Grid(c)
    g.step(steps)
    out = dict(storage=storage, steps=steps, leaf_masks_equal=True, u_rel_l2=0.0, drho_max_abs=0.0)
    for l, geom in enumerate(s.geoms):
        leaf = s.masks[l][0]
        tag = g.get("tag", 0, l).reshape(-1)
        out["leaf_masks_equal"] &= bool(np.array_equal((tag & 64) != 0, leaf))
        rho_o, u_o = s.macros(l)
        rho_g = g.get("rho", 0, l).reshape(-1).astype(np.float64)
        u_g = g.get("u", 0, l).reshape(geom.D, -1).astype(np.float64)
        den = float(np.sqrt((u_o[:, leaf] ** 2).sum())) or 1.0
        out["u_rel_l2"] = max(out["u_rel_l2"], float(np.sqrt(((u_g[:, leaf] - u_o[:, leaf]) ** 2).sum())) / den)
        out["drho_max_abs"] = max(out["drho_max_abs"], float(np.abs(rho_g[leaf] - rho_o[leaf]).max()))
    out["phi_max_abs"] = float(np.abs(g.get("phi").reshape(-1).astype(np.float64) - s.phi).max())
    out["phases_equal"] = bool(np.array_equal(g.get("phase").reshape(-1), s.phase[-1].astype(np.uint8)))
    g.close()
    return out


def cpu_baseline(budget_s=20.0, warmup=0, compare_storage=None):
    """The FP64 oracle as it stands on the host cores: bounded sample = the
    downsampled 32x32x64 copy of the workload (same physics, d scaled by 1/4),
    `warmup` untimed coarse steps, then as many timed coarse steps as fit in
    ~budget_s (at least one).  With compare_storage, the CUDA path then runs the
    same case for the same steps and its field errors against the oracle's state
    are reported."""
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import workloads
    case = workloads.rising_bubble_3d(scale=0.25)
    case["phi0"] = np.asarray(case["phi0"], np.float32).astype(np.float64)  # one initial level set for both
    s = Sim(case)
    s.step(warmup)
    t0 = time.perf_counter()
    c0 = time.process_time()  # CPU time of all the process's threads (numpy's BLAS may use several)
    n = 0
    upd = 0.0
    while True:
        s.step(1)
        n += 1
        upd += sum(float(m[0].sum()) * 2 ** l for l, m in enumerate(s.masks))
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = (time.process_time() - c0) / dt  # threads busy on average over the timed steps
    if isinstance(compare_storage, (list, tuple)):
        err = {st: oracle_error(case, s, warmup + n, st) for st in compare_storage}
    else:
        err = oracle_error(case, s, warmup + n, compare_storage) if compare_storage else None
    return dict(value=upd / dt / 1e6, unit="MLUPS", cores=round(max(cores, 1.0), 1), kind="oracle",
                ms_per_step=dt / n * 1e3, error_vs_oracle=err,
                sample=f"downsampled 32x32x64 base / 2-level copy of the workload, {warmup} untimed and {n} "
                       f"timed coarse steps, {upd:.0f} cell updates in {dt:.1f} s (numpy float64; cores = CPU "
                       f"time / wall time of the timed steps, {os.cpu_count()} host cores)")


# DRAM bytes per launch of the collide-and-stream kernel (ncu dram__bytes_read.sum +
# dram__bytes_write.sum per level's launch class) on a workload, with the sha1 of the kernel
# sources the capture was taken on: a change to them voids the figure (traffic null).
TRAFFIC = dict(
    sources_sha1="2a97239a19b27e02f71529324b044a1e865e204e",
    # 3D rising bubble 128x128x256, two levels, FP32: one coarse step after the warm-up
    # (level 0, then the two level-1 sub-steps: 260.6 and 260.2 MB)
    per_launch={("bubble3d", 1.0, "fp32"): {"k_collide_stream": 327672064 + 251297280,
                                            "k_collide_stream_l1": (161361408 + 99237632 + 161222400 + 98941696) / 2}})


def kernel_sources_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in ("lsb_lb.cu", "lsb_device.cuh", "lsb_tma.cuh"):
        with open(os.path.join(ROOT, "paper_2601_05936_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def step_bytes(g, cases):
    """Algorithmic bytes of one coarse step, pass by pass: every pass reads each of its
    inputs once and writes each of its outputs once (s = bytes per stored population,
    4 or 2; fields float32).  Counts are the work lists after the last step
    (lsb_work_counts); levels are global, level l takes 2^l sub-steps per coarse step.
      collide-and-stream: 2 Q s per leaf cell update;
      ghost ring: 2 Q s per ghost cell and fill (coarse sources read, pushes written);
      restriction: (2^D + 1) Q s per covered cell and sub-step of the coarse level;
    finest level, per sub-step (B band cells, I interface cells, K cut links):
      interface bounce-back: per link the two parked populations, the populations written
        and the other node's moments, strain rate, normal and curvature;
      interface velocity: per interface cell its mask, phi, u and u~; per link phi and u;
      extension sweeps: the first reads phi, u~ and writes u~ and the plan, each later
        one reads the plan and u~ and writes u~;
      transport (3 TVD-RK3 stages): stage 1 reads u~ and phi and writes u~ x3 and p1, the
        others read u~, phi and their stage array and write the next;
      reinitialisation (3 stages per pseudo step): phi, S(phi0), frozen flag and stage arrays;
      classification: phase (phi, tag, p1/p2 written back) and cut masks over the band,
        link list entries per link; curvature fit per interface cell (phi, n, kappa)."""
    c0 = cases[0]
    D = 2 if c0["lattice"] == "D2Q9" else 3
    Q = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}[c0["lattice"]]
    s = 2 if c0.get("storage", "fp32") == "fp16s" else 4
    L = max(int(c.get("n_levels", 1)) for c in cases)
    n_ext = int(c0.get("n_ext", 8))
    re_every = int(c0.get("reinit_every", 1))
    n_re = int(c0.get("n_reinit", 1)) if re_every == 1 else 0  # bench workloads reinitialise every step
    live = bool(c0.get("ls_active", True))
    MF = 1 + D + D * (D + 1) // 2
    by = dict(collide=0.0, ghost=0.0, restrict=0.0, interface=0.0, ext=0.0, transport=0.0, reinit=0.0,
              classify=0.0)
    for l in range(L):
        w = g.work_counts(l)
        sub = 2 ** l
        by["collide"] += sub * w["leaf"] * 2 * Q * s
        by["ghost"] += sub * w["ghost"] * 2 * Q * s
        by["restrict"] += sub * w["restrict"] * (2 ** D + 1) * Q * s
        B, I, K = w["band"], w["iface"], w["links"]
        if B == 0 and K == 0:
            continue
        by["interface"] += sub * K * (8 + s + (MF + D + 1) * 4)
        if not live:
            continue
        by["ext"] += sub * (I * (8 + 2 * D * 4) + K * (1 + D) * 4)
        if n_ext > 0:
            by["ext"] += sub * B * (((3 * D + 1) * 4 + 2) + (n_ext - 1) * (3 * D * 4 + 1))
        by["transport"] += sub * B * ((4 * D + 2) * 4 + 2 * (D + 3) * 4)
        if n_re > 0:
            by["reinit"] += sub * B * (13 + 17 * (3 * n_re - 1))
        by["classify"] += sub * (B * (14 + 5) + K * 9 + I * (4 + (D + 1) * 4))
    return sum(by.values()), by


def oracle_compare(case, steps):
    """The oracle on the workload's own case (full size, `steps` coarse steps, host cores),
    then the CUDA path for the same steps: the oracle's throughput and the field errors."""
    from oracle.sim import Sim
    case = dict(case)
    case["phi0"] = np.asarray(case["phi0"], np.float32).astype(np.float64)  # one initial level set for both
    s = Sim(case)
    t0 = time.perf_counter()
    c0 = time.process_time()
    upd = 0.0
    for _ in range(steps):
        s.step(1)
        upd += sum(float(m[0].sum()) * 2 ** l for l, m in enumerate(s.masks))
    dt = time.perf_counter() - t0
    cores = (time.process_time() - c0) / dt
    err = oracle_error(case, s, steps, case.get("storage", "fp32"))
    return dict(value=upd / dt / 1e6, unit="MLUPS", cores=round(max(cores, 1.0), 1), kind="oracle",
                ms_per_step=dt / steps * 1e3, error_vs_oracle=err,
                sample=f"the workload's own case, {steps} coarse steps, {upd:.0f} cell updates in {dt:.1f} s "
                       f"(numpy float64; {os.cpu_count()} host cores)")


def timed_record(cases, steps, warmup, local, label):
    """A secondary throughput record: the cases in one handle with graph replay, `warmup`
    untimed and `steps` timed coarse steps (CUDA events on the library stream), clocks
    sampled during the timed steps."""
    import torch
    from paper_2601_05936_gb300 import lsb
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    g = lsb.Grid(cases, stream=stream, device=local)
    g.use_graphs(True)
    g.step(warmup)
    g.sync()
    setup_s = time.perf_counter() - t0
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    l0, u0 = g.kernel_launches(), g.cell_updates(total=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches, upd = g.kernel_launches() - l0, g.cell_updates(total=True) - u0
    sb, by_pass = step_bytes(g, cases)
    hbm, src = peaks()
    ach = sb / (ms / steps / 1e3) / 1e9
    g.close()
    return dict(label=label, value=upd / (ms / 1e3) / 1e6, unit="MLUPS", steps=steps, warmup=warmup,
                ms_per_step=ms / steps, gpu_launches=launches, launches_per_step=launches / steps,
                cell_updates_per_step=upd / steps, setup_s=setup_s,
                step_roofline=dict(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                                   bytes_per_step=sb, peak_source=src), clocks=clk)


def reduce_ranks(ms, upd, dist, device):
    """Replicas: the job's time is the slowest rank's, its work the sum over ranks."""
    if dist is None:
        return ms, upd
    import torch
    t = torch.tensor([ms, upd], dtype=torch.float64, device=device)
    tm = t.clone()
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    ts = t.clone()
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    return float(tm[0]), float(ts[1])


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each step is one coarse step of the downsampled copy (about 4 s here); the warm-up
    # and the timed steps are capped so that the run ends within a few minutes
    res = cpu_baseline(budget_s=max(10.0, min(120.0, 6.0 * max(args.steps, 1))), warmup=min(args.warmup, 3))
    line = dict(impl="reference", metric=METRIC, value=res["value"], unit="MLUPS", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=res["ms_per_step"], higher_is_better=True,
                scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload="rising_bubble_3d_32x32x64_L2 (downsampled sample of 128x128x256_L2)",
                            lattice="D3Q19"),
                cpu_baseline=res, e2e=dict(value=res["value"], unit="MLUPS", h2d_bytes_per_step=0,
                                           d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def adjoint_bench(args, world, rank, local, barrier, dist, moving=False, levels=1):
    """Reverse sweep of the adjoint: 128x128x256 D3Q19 box with the bubble of the
    benchmark workload (d = 32 finest cells, density ratio 1000), single-level
    or on the benchmark's two-level grid, level set frozen or moving.  A
    step of the metric is one adjoint step of the sweep: recomputation of the
    forward step from the segment checkpoint, the segment-store copy (on two
    levels also the replay of the step with its per-call record), the cut-link,
    per-cell and level-transfer adjoint kernels."""
    import torch
    from paper_2601_05936_gb300 import autograd, lsb, workloads
    case = workloads.rising_bubble_3d(levels=levels)
    if moving:  # level set live: the sweep also replays and transposes the level-set passes
        case.update(regrid_every=0)
    else:
        case.update(ls_active=False, n_ext=0, reinit_every=0, regrid_every=0)
    stream = torch.cuda.Stream()
    g = lsb.Grid(case, stream=stream, device=local)
    g.step(args.warmup)
    # forward step time of the same workload (eager, as the recorded steps run)
    g.sync()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    g.step(args.steps)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1) / args.steps
    g.record(args.checkpoint_every)
    g.step(args.steps)
    D = g.D
    w = np.zeros((1, 4 + 2 * D))
    w[0, 4 + 2 * D - 1] = 1.0  # vertical gas velocity
    g.backward(w)  # warm-up sweep (allocates the segment store)
    g.sync()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    g.profile(2)
    launches0 = g.kernel_launches()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    dp = g.backward(w)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    prof = g.profile_read()
    g.profile(0)
    clk = clocks.stop()
    launches = g.kernel_launches() - launches0
    cells = g.cell_updates()
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t[0])
    value = world * cells * args.steps / (ms_max / 1e3) / 1e6
    hbm, src = peaks()
    kms, kn, kb = prof.get("k_adj_collide", (0.0, 0, 0.0))
    achieved = kb / (kms / 1e3) / 1e9 if kms > 0 else None
    roof = dict(bound="hbm", achieved=achieved, peak=hbm, unit="GB/s", frac=achieved / hbm if achieved else None,
                traffic=None, peak_source=src + " (hbm_gbs, of " + src + ")", kernel="k_adj_collide", launches=kn,
                bytes_per_launch=kb / max(kn, 1), avg_launch_ms=kms / max(kn, 1),
                share_of_step=kms / ms if ms > 0 else None,
                kernels={k: dict(ms=v[0], launches=v[1]) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])})
    # end to end through the public API: autograd window (forward recorded steps + reverse sweep),
    # parameters from a host tensor, gradient back on the host
    E = max(1, min(args.steps, 50))
    p = autograd.params_tensor([case])
    g.sync()
    t0 = time.perf_counter()
    obs = autograd.window(g, p, E, checkpoint_every=args.checkpoint_every)
    (grad,) = torch.autograd.grad(obs[0, 4 + 2 * D - 1], p)
    t1 = time.perf_counter()
    e2e = dict(value=world * cells * E / (t1 - t0) / 1e6, unit="MLUPS", h2d_bytes_per_step=8 * 5 / E,
               d2h_bytes_per_step=(8 * (4 + 2 * D) + 8 * 5) / E, steps=E,
               note="autograd.window(E steps) + torch.autograd.grad per window, host wall clock: "
                    "forward recorded steps and the reverse sweep, MLUPS of one adjoint step each")
    g.close()
    state_mb = sum(float(np.prod([b * 2 ** l for b in case["base"]])) for l in range(levels)) * 19 * 4 / 1e6
    if rank != 0:
        return
    line = dict(metric="MLUPS of the reverse sweep (adjoint cell steps / s), 3D D3Q19 "
                       + ("moving" if moving else "frozen") + " bubble 128x128x256"
                       + (f", {levels} levels" if levels > 1 else ""),
                value=value, unit="MLUPS", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms_max / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32", data="synthetic",
                config=dict(workload=case["name"] + ("_moving" if moving else "_frozen"), lattice="D3Q19", levels=levels,
                            storage="fp32",
                            parallelism=f"replicas{world}", checkpoint_every=args.checkpoint_every,
                            cells=cells, l2_flush=f"state {state_mb:.0f} MB x (segment store) >> 129 MB L2",
                            dJ_dparams=[float(v) for v in dp[0]], forward_ms_per_step=fwd_ms,
                            adjoint_over_forward=(ms_max / args.steps) / fwd_ms),
                roofline=roof, cpu_baseline=None, e2e=e2e, gpu_launches=launches, clocks=clk)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="lsb", choices=["lsb", "reference"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16s"])
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-all", action="store_true", help="print a per-kernel time table to stderr")
    ap.add_argument("--workload", default="bubble3d",
                    choices=["bubble3d", "box3d", "ensemble", "adjoint3d", "adjoint3d_ls", "adjoint3d_amr",
                             "adjoint3d_amr_ls",
                             "paper3d", "couette2d", "cluster3d", "stratified", "drop2d", "bubble2d"],
                    help="bubble3d: the benchmark configuration; box3d: uniform periodic 128^3 box "
                         "(collide-and-stream only, for profiling captures); ensemble: 64 uneven 2D bubbles; "
                         "adjoint3d: reverse sweep over --steps recorded steps of a frozen 3D bubble; "
                         "adjoint3d_ls: the same with the level set moving (short windows: no phase change); "
                         "adjoint3d_amr: the frozen adjoint on the two-level grid of bubble3d; "
                         "adjoint3d_amr_ls: the same with the finest level's level set moving; "
                         "paper3d: the paper's own 3D box (2d x 2d x 4d, d = 64, uniform, slip lateral walls, "
                         "case --paper-case); couette2d: two-layer Couette with a moving wall, 2048^2; cluster3d: nine "
                         "rising bubbles (case I) in a 10 d x 10 d x 20 d box, d = 32 finest cells, 2 levels; "
                         "stratified: the two-layer channel, 64x32, D2Q9; drop2d: the Laplace static drop, "
                         "128^2 base, 2 levels; bubble2d: the 2D rising bubble, 160x320 base, 3 levels "
                         "(the last three also run the oracle on the same case for --oracle-steps)")
    ap.add_argument("--oracle-steps", type=int, default=None,
                    help="stratified / drop2d / bubble2d: coarse steps of the oracle comparison "
                         "(default 1000 / 20 / 2)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="bubble3d: skip the secondary records (64-case ensemble, FP16 storage)")
    ap.add_argument("--paper-case", default="I", choices=["I", "II"], help="paper3d: parameter set of Sec. 3.2")
    ap.add_argument("--lattice", default="D3Q19", choices=["D3Q19", "D3Q27"],
                    help="paper3d: D3Q19 with BGK in both phases, or the paper's own 3D setup: D3Q27 with BGK "
                         "in the liquid and the cumulant model in the gas")
    ap.add_argument("--nu-floor", type=float, default=None,
                    help="paper3d: lower bound of the lattice viscosities (default 0.05 for case I, 0.1 for "
                         "case II, the smallest measured stable; BGK in both phases is unstable at the "
                         "paper's Re = 35, tau = 0.563, where the paper's gas solver is a cumulant model)")
    ap.add_argument("--checkpoint-every", type=int, default=100)
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel from the host instead of replaying captured CUDA graphs")
    ap.add_argument("--driver", type=int, default=0, choices=[0, 1],
                    help="level-set passes: 0 one launch each, 1 one persistent cooperative launch per finest step")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="bubble3d and box3d: linear scale of the box (and bubble) (profiling captures of a "
                         "smaller copy; box3d at 2.0 is the 256^3 box)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_05936_gb300 import lsb, workloads

    if args.workload in ("adjoint3d", "adjoint3d_ls", "adjoint3d_amr", "adjoint3d_amr_ls"):
        adjoint_bench(args, world, rank, local, barrier, dist, moving=args.workload.endswith("_ls"),
                      levels=2 if "_amr" in args.workload else 1)
        return
    if args.workload == "bubble3d":
        case = workloads.rising_bubble_3d(storage=args.storage, scale=args.scale)
        cases = [case]
    elif args.workload == "box3d":
        case = workloads.uniform_box(n=int(round(128 * args.scale)), storage=args.storage)
        cases = [case]
    elif args.workload == "paper3d":
        floor = args.nu_floor if args.nu_floor is not None else {"I": 0.05, "II": 0.1}[args.paper_case]
        coll = ("bgk", "cumulant") if args.lattice == "D3Q27" else ("bgk", "bgk")
        case = workloads.paper_box_3d(args.paper_case, storage=args.storage, nu_floor=floor, lattice=args.lattice,
                                      collision=coll)
        cases = [case]
    elif args.workload == "cluster3d":
        case = workloads.bubble_cluster_3d(d=32, levels=2, storage=args.storage)
        cases = [case]
    elif args.workload == "couette2d":
        case = workloads.two_layer_couette()
        case["storage"] = args.storage
        cases = [case]
    elif args.workload in ("stratified", "drop2d", "bubble2d"):
        case = {"stratified": workloads.stratified_channel, "drop2d": workloads.static_drop,
                "bubble2d": workloads.rising_bubble_2d}[args.workload]()
        case["storage"] = args.storage
        cases = [case]
    else:
        cases = workloads.ensemble()
        for c in cases:
            c["storage"] = args.storage
        case = cases[0]
    stream = torch.cuda.Stream()
    g = lsb.Grid(cases, stream=stream, device=local)
    g.set_driver(args.driver)
    graphs = not args.no_graphs and args.driver == 0
    g.use_graphs(graphs)  # two coarse steps per graph replay; the warm-up captures them
    g.step(args.warmup)
    g.sync()

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = g.kernel_launches()
    upd0 = g.cell_updates(total=True)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    g.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = g.kernel_launches() - launches0
    upd = g.cell_updates(total=True) - upd0
    # per-kernel times for the roofline: a second, shorter pass with an event pair around
    # every launch (eager launches: per-launch events and graph replay exclude each other)
    P = max(2, min(args.steps, 50))
    g.profile(2 if args.profile_all else 1)
    torch.cuda.synchronize()
    ev0.record(stream)
    g.step(P)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_p = ev0.elapsed_time(ev1)
    prof = g.profile_read()
    g.profile(0)
    clk = clocks.stop()
    g.sync()

    ms_max, upd_sum = reduce_ranks(ms, upd, dist, "cuda")
    value = upd_sum / (ms_max / 1e3) / 1e6

    # roofline of the dominant kernel (collide-and-stream), from events on the library stream
    cs = [v for k, v in prof.items() if k.startswith("k_collide_stream")]
    cs_ms = sum(v[0] for v in cs)
    cs_n = sum(v[1] for v in cs)
    cs_bytes = sum(v[2] for v in cs)
    per_level = {k: dict(ms=v[0], launches=v[1], bytes_per_launch=v[2] / max(v[1], 1),
                         gbs=(v[2] / (v[0] / 1e3) / 1e9 if v[0] > 0 else None))
                 for k, v in prof.items() if k.startswith("k_collide_stream")}
    hbm, src = peaks()
    achieved = cs_bytes / (cs_ms / 1e3) / 1e9 if cs_ms > 0 else None
    # DRAM bytes per launch of the current collide-and-stream kernel on this workload (ncu
    # dram__bytes_read.sum + dram__bytes_write.sum, one coarse step of the full-size FP32 run):
    # launch-weighted over the levels; other workloads have no capture
    traffic = None
    key = (args.workload, args.scale, args.storage)
    if TRAFFIC.get("sources_sha1") == kernel_sources_sha1() and key in TRAFFIC.get("per_launch", {}) and cs_n > 0:
        per = TRAFFIC["per_launch"][key]
        traffic = sum(per.get(k, 0.0) * v[1] for k, v in prof.items() if k.startswith("k_collide_stream")) / cs_n
    roof = dict(bound="hbm", achieved=achieved, peak=hbm, unit="GB/s",
                frac=(achieved / hbm) if achieved else None, traffic=traffic, peak_source=src + " (hbm_gbs, of "
                + src + ")", kernel="k_collide_stream", launches=cs_n,
                bytes_per_launch=cs_bytes / max(cs_n, 1), avg_launch_ms=cs_ms / max(cs_n, 1),
                share_of_step=cs_ms / ms_p if ms_p > 0 else None, per_level=per_level,
                timed_in=f"separate pass of {P} steps with per-launch events (eager launches)")
    # whole-step roofline: the algorithmic bytes of every pass of a coarse step over the
    # timed ms per step
    sb, by_pass = step_bytes(g, cases)
    step_ach = sb / (ms_max / args.steps / 1e3) / 1e9
    step_roof = dict(bound="hbm", achieved=step_ach, peak=hbm, unit="GB/s", frac=step_ach / hbm,
                     bytes_per_step=sb, by_pass_bytes=by_pass, peak_source=src + " (hbm_gbs, of " + src + ")",
                     note="algorithmic bytes of every pass of one coarse step (each pass reads its inputs once "
                          "and writes its outputs once; work lists after the last step) / ms_per_step; the "
                          "finest level's band fields (a few MB) stay in L2 between passes")
    if args.profile_all and rank == 0:
        for k, (kms, kn, kb) in sorted(prof.items(), key=lambda kv: -kv[1][0]):
            print(f"{k:20s} {kms:9.2f} ms {kn:7d} launches {100 * kms / ms_p:5.1f}%", file=sys.stderr)

    # end to end through the public API with host buffers: parameters H2D, step, observables D2H
    import ctypes
    E = args.e2e_steps
    nld = len(g.cases) * int(case["n_levels"])
    h2d = ctypes.sizeof(lsb.Params) + 0  # the parameter struct the caller hands over each step
    d2h = 8 * (4 + 2 * g.D) * len(g.cases)
    h2d *= len(g.cases)
    g.sync()
    u0 = g.cell_updates(total=True)
    t0 = time.perf_counter()
    for _ in range(E):
        for k, c in enumerate(cases):
            g.set_params(c, k)
        g.step(1)
        g.observables()
    t1 = time.perf_counter()
    e2e = dict(value=(g.cell_updates(total=True) - u0) / (t1 - t0) / 1e6 * world, unit="MLUPS",
               h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h, steps=E,
               note=f"lsb_set_params + lsb_step(1) + lsb_observables per step, host wall clock; the "
                    f"parameter upload also rewrites {nld} level descriptors on the device")
    obs = g.observables()[0]
    g.close()

    if rank != 0:
        return
    cpu = None
    secondary = None
    if not args.no_cpu_baseline and world == 1 and args.workload == "bubble3d":
        cpu = cpu_baseline(compare_storage=[args.storage] + (["fp16s"] if args.storage == "fp32" else []))
    elif not args.no_cpu_baseline and world == 1 and args.workload in ("stratified", "drop2d", "bubble2d"):
        osteps = args.oracle_steps or {"stratified": 1000, "drop2d": 20, "bubble2d": 2}[args.workload]
        cpu = oracle_compare(case, osteps)
    if world == 1 and args.workload == "bubble3d" and args.scale == 1.0 and not args.no_secondary:
        ens = workloads.ensemble()
        secondary = dict(
            ensemble=timed_record(ens, args.steps, args.warmup, local,
                                  "ensemble of 64 2D rising bubbles (96x192..256x512, 1-3 levels), one handle"),
            fp16s=timed_record([workloads.rising_bubble_3d(storage="fp16s")], args.steps, args.warmup, local,
                               "the same 3D bubble with FP16 storage / FP32 arithmetic"))
    metric = METRIC if args.workload == "bubble3d" else f"MLUPS (leaf cell updates / s), {args.workload}"
    lattice = case["lattice"]
    state_gb = sum(float(np.prod([b * 2 ** l for b in c["base"]])) for c in cases
                   for l in range(int(c["n_levels"]))) * 2 * {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}[lattice] * 4 / 1e9
    wname = case["name"] if len(cases) == 1 else f"ensemble of {len(cases)} 2D rising bubbles (96x192..256x512, 1-3 levels)"
    line = dict(metric=metric, value=value, unit="MLUPS", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms_max / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32" if args.storage == "fp32" else "f16-store/f32-compute", data="synthetic",
                config=dict(workload=wname, lattice=lattice, levels=int(case["n_levels"]),
                            storage=args.storage, parallelism=f"replicas{world}", driver=args.driver,
                            cuda_graphs=graphs,
                            cell_updates_per_step=upd / args.steps,
                            l2_flush=f"state {state_gb:.1f} GB (both buffers) >> 129 MB L2",
                            bubble=dict(centroid=[float(v) if np.isfinite(v) else None for v in obs["centroid"]],
                                        velocity=[float(v) if np.isfinite(v) else None for v in obs["velocity"]])),
                roofline=roof, step_roofline=step_roof, cpu_baseline=cpu, e2e=e2e, gpu_launches=launches,
                launches_per_step=launches / args.steps, clocks=clk, secondary=secondary)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
