"""Autotuner of the two-site update's schedule.

For every (values per site, precision, chi_max) of the grid below it times whole time
steps of an ensemble of synthetic states at full bond dimension under candidate
schedules (the lt_config fields theta_path and env_ctas_per_sm) with CUDA
events, by coordinate search from the default schedule, and keeps the fastest.  It
writes the table as JSON and as the C header the library compiles in
(csrc/lt_schedule_table.h), which lt_create consults for every field left at 0.

    python -m paper_2609_18841_b300.autotune --out DIR     (on the GPU)

The header and JSON written to DIR are then copied over csrc/lt_schedule_table.h and
schedules.json, and the library is rebuilt.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

# (values per site, chi_max grid); trajectories (2) and the vectorised density matrix (4)
GRID = {2: (16, 32, 64, 128, 256), 4: (16, 32, 64, 128)}


def full_dims(L, chi, d):
    return [min(d ** min(b + 1, 30), d ** min(L - 1 - b, 30), chi) for b in range(L - 1)]


def time_steps(lt, torch, d, precision, chi, sched, n_traj, L, steps):
    """Device time per step of n_traj synthetic full-dimension chains under `sched`."""
    method = lt.LT_TRAJ if d == 2 else lt.LT_MPDO
    kw = dict(method=method, precision=precision, init="neel", dt=0.02, gamma_loss=0.1,
              fermionic_jumps=1 if d == 2 else 0, svd_cut=1e-6 if precision == lt.LT_MIXED else 1e-12,
              seed=3, **sched)
    if d == 4:
        kw.update(gamma_gain=0.05)
    mps = [workloads.synthetic_mps(L, chi, seed=500 + t, d=d, dims=full_dims(L, chi, d))
           for t in range(min(4, n_traj))]
    packed = lt.pack_state(mps, L, chi, d=d)
    with lt.Ensemble(L, chi, n_traj, **kw) as e:
        for t0 in range(0, n_traj, len(mps)):
            m = min(len(mps), n_traj - t0)
            lt.lt_set_state(e.ctx, t0, packed[0][:m], packed[1][:m], packed[2][:m])
        lt.lt_step(e.ctx, 1)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.ExternalStream(lt.lt_stream(e.ctx))
        a.record(stream)
        lt.lt_step(e.ctx, steps)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps


def tune_one(lt, torch, d, precision, chi, log):
    L = 32 if d == 2 else 12
    slow = chi >= 128 and (precision == lt.LT_FP64 or d == 4)
    n_traj = 8 if slow else (48 if chi <= 64 else 16)
    steps = 1 if slow else 2
    knobs = []
    if precision == lt.LT_MIXED and d == 2:
        knobs.append(("theta_path", (1, 2)))
    knobs.append(("env_ctas_per_sm", (8, 4, 2, 1)))
    best = {"theta_path": 1, "env_ctas_per_sm": 8}
    t_default = time_steps(lt, torch, d, precision, chi, best, n_traj, L, steps)
    t_best = t_default
    tried = {json.dumps(best, sort_keys=True): t_default}
    for name, values in knobs:
        for v in values:
            cand = dict(best, **{name: v})
            key = json.dumps(cand, sort_keys=True)
            if key not in tried:
                tried[key] = time_steps(lt, torch, d, precision, chi, cand, n_traj, L, steps)
            if tried[key] < t_best * 0.99:  # keep a change only for a clear gain
                best, t_best = cand, tried[key]
    entry = {"d": d, "precision": "mixed" if precision == lt.LT_MIXED else "fp64", "chi_max": chi,
             "L": L, "n_traj": n_traj, "steps": steps, "schedule": best,
             "ms_per_step_default": t_default, "ms_per_step_tuned": t_best,
             "candidates": {k: v for k, v in tried.items()}}
    log(json.dumps({k: entry[k] for k in ("d", "precision", "chi_max", "schedule",
                                          "ms_per_step_default", "ms_per_step_tuned")}))
    return entry


def header(entries, gpu):
    lines = ["// Tuned schedules of the two-site update, written by paper_2609_18841_b300/autotune.py",
             "// from timings on the device (%s); no entry: the defaults of lindtebd.h." % gpu,
             "#pragma once", "", "struct LtSchedule {",
             "  int d, precision, chi_max;          // values per site, lt_precision, chi_max",
             "  int theta_path, env_ctas_per_sm;", "};", "",
             "static const LtSchedule kLtSchedules[] = {"]
    for e in entries:
        s = e["schedule"]
        lines.append("    {%d, %d, %d, %d, %d},  // %.1f -> %.1f ms per step" % (
            e["d"], 1 if e["precision"] == "mixed" else 0, e["chi_max"], s["theta_path"],
            s["env_ctas_per_sm"], e["ms_per_step_default"], e["ms_per_step_tuned"]))
    lines += ["};", ""]
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    import torch
    from paper_2609_18841_b300 import lindtebd as lt
    os.makedirs(args.out, exist_ok=True)
    entries = []
    t0 = time.time()
    for d, chis in GRID.items():
        for precision in (lt.LT_MIXED, lt.LT_FP64):
            for chi in chis:
                entries.append(tune_one(lt, torch, d, precision, chi, print))
                sys.stdout.flush()
    gpu = torch.cuda.get_device_name(0)
    with open(os.path.join(args.out, "schedules.json"), "w") as f:
        json.dump({"gpu": gpu, "seconds": time.time() - t0, "entries": entries}, f, indent=1)
    with open(os.path.join(args.out, "lt_schedule_table.h"), "w") as f:
        f.write(header(entries, gpu))


if __name__ == "__main__":
    main()
