"""Terminal rise velocity against the refinement distance d_ref (the paper's AMR study of
the 3D case II, Sec. 3.2: base d/dx = 32 refined to 64 with the signed level-set sensor,
compared with the uniform d/dx = 64 grid).

Runs on the GPU through the library only:

    python -m paper_2601_05936_gb300.study_dref --tstar 3 --drefs 0.5 1 1.5 2 2.5 3

Time is t* = t sqrt(g / L), L = 2 d the box width (the paper's normalisation); the terminal
velocity is the mean vertical gas velocity over the last fifth of the run.  One JSON line per
run, then a summary line with each deviation from the uniform run.
"""
import argparse
import json
import time

import numpy as np


def run(case, tstar, chunk):
    from . import lsb
    g = lsb.Grid(case)
    d = 64
    grav = abs(case["gravity"][2])
    r = 2 ** (int(case["n_levels"]) - 1)  # finest steps per coarse step
    rate = np.sqrt(grav / (2 * d))         # t* per finest step
    steps = int(round(tstar / rate / r))   # coarse steps
    t0 = time.perf_counter()
    ts, us = [], []
    done = 0
    diverged = None
    while done < steps:
        n = min(chunk, steps - done)
        try:
            g.step(n)
            obs = g.observables()[0]
        except lsb.LsbError as e:  # non-finite state: report when, keep what was measured
            diverged = dict(tstar=(done + n) * r * rate, error=str(e))
            break
        done += n
        ts.append(done * r * rate)
        us.append(float(obs["velocity"][2]))
    cells = g.cell_updates()
    g.close()
    ts, us = np.array(ts), np.array(us)
    if diverged or len(ts) == 0:
        return dict(steps=steps, diverged=diverged, wall_s=time.perf_counter() - t0, cell_updates_per_step=cells,
                    terminal_velocity=None, u_peak=float(us.max()) if len(us) else None, history=[])
    tail = ts >= 0.8 * ts[-1]
    return dict(steps=steps, diverged=None, wall_s=time.perf_counter() - t0, cell_updates_per_step=cells,
                terminal_velocity=float(us[tail].mean()), u_peak=float(us.max()),
                history=[[round(float(t), 4), u] for t, u in zip(ts[::max(1, len(ts) // 40)], us[::max(1, len(us) // 40)])])


def main():
    from . import workloads
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="II", choices=["I", "II"])
    ap.add_argument("--tstar", type=float, default=3.0)
    ap.add_argument("--drefs", type=float, nargs="+", default=[0.5, 1.0, 1.5, 2.0, 2.5, 3.0])
    ap.add_argument("--nu-floor", type=float, default=0.1)
    ap.add_argument("--Ma", type=float, default=0.02)
    ap.add_argument("--uniform-only", action="store_true")
    ap.add_argument("--chunk", type=int, default=200)
    args = ap.parse_args()
    out = {}
    uni = workloads.paper_box_3d(args.case, d=64, levels=1, nu_floor=args.nu_floor, Ma=args.Ma)
    out["uniform"] = run(uni, args.tstar, args.chunk)
    print(json.dumps(dict(run="uniform d/dx=64", **out["uniform"])), flush=True)
    if args.uniform_only or out["uniform"]["terminal_velocity"] is None:
        return
    for dr in args.drefs:
        c = workloads.paper_box_3d(args.case, d=64, levels=2, nu_floor=args.nu_floor, Ma=args.Ma, sensor="signed",
                                   refine_dist=dr * 64)
        out[dr] = run(c, args.tstar, args.chunk)
        print(json.dumps(dict(run=f"amr d_ref/d = {dr}", **out[dr])), flush=True)
    ut = out["uniform"]["terminal_velocity"]
    print(json.dumps(dict(summary={str(dr): dict(terminal_velocity=out[dr]["terminal_velocity"],
                                                 deviation=out[dr]["terminal_velocity"] / ut - 1.0,
                                                 cell_updates_per_step=out[dr]["cell_updates_per_step"])
                                   for dr in args.drefs if out[dr]["terminal_velocity"] is not None},
                          uniform=ut)), flush=True)


if __name__ == "__main__":
    main()
