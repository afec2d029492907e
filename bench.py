#!/usr/bin/env python
"""Benchmark of the GB300 multigrid xCFC solver.

One step = one full xCFC solve (Steps 1-6 of Sec. 2.6: the X, psi, alpha-psi
and shift equations, each by FAS V(2,2) cycles to a relative residual of
1e-10) from the flat initial guess, on the uniformly rotating n = 1
polytrope on the 3D spherical 128 x 64 x 64 grid (r <= 100), inputs
resident in HBM.  The metric is smoother cell-updates per second
(sum over levels of cells x sweeps x components, per second of device time).

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
instead (a bounded sample of the same workload on the host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_GRID = (128, 64, 64)
R_MAX = 100.0
TOL = 1e-10
METRIC = "V-cycle Gcell-updates/s"
UNIT = "Gcell-updates/s"
WORKLOAD = "xCFC full system (X, psi, alpha*psi, beta), 3D spherical 128x64x64, r<=100, rotating n=1 polytrope"


def aggregate_ranks(dist, total_ms, updates, device):
    """Whole-job numbers over the ranks: the slowest rank's timed milliseconds
    and the cell updates of all ranks (each rank solves its own replica, weak
    scaling).  dist is torch.distributed or None (one rank)."""
    if dist is None:
        return total_ms, float(updates)
    import torch
    t = torch.tensor([total_ms, float(updates)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1])


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--max-cycles", type=int, default=1000)
    p.add_argument("--accel", type=int, default=16, help="Anderson mixing depth (0: plain V-cycles)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-divb", action="store_true", help="skip the 256^3 div-B cleaning measurement")
    p.add_argument("--no-serve", action="store_true", help="skip the request-serving measurement")
    p.add_argument("--serve-sweep", action="store_true",
                   help="serving at arrival rates 250..4000/s, 1000 requests each, mixed and FP64 (minutes)")
    p.add_argument("--no-batch", action="store_true", help="skip the 512-solve batch measurement")
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 solve beside the mixed one")
    p.add_argument("--fp64-steps", type=int, default=3, help="timed FP64 solves (each ~1 s)")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def sources():
    from paper_2012_07322_gb300 import inputs
    return inputs.rotating_polytrope_sph3d(N_GRID, R_MAX)


def level_cells():
    """Cells per level of the hierarchy (halving while all dims even, >= 4)."""
    n = list(N_GRID)
    out = []
    while True:
        out.append(n[0] * n[1] * n[2])
        if any(x < 4 or x % 2 for x in n):
            break
        n = [x // 2 for x in n]
    return out


# Algorithmic bytes per cell one launch of each profiled kernel class
# processes, from the bytes the method itself must move: one red-black sweep
# streams s (2 n_u + n_in) bytes per cell (read and write each of the n_u
# unknowns, read each of the n_in per-cell inputs; s = 8 FP64, 4 FP32), and a
# colour pass, which updates half of the cells for one component, carries
# 1 / (2 n_comp) of it, i.e. s (2 n_u + n_in) / n_comp per updated cell:
#   colour pass, scalar (n_u = 1, n_in = 2: U and A2 of eq. psi, c and f of a
#     linear equation, or f32 and K of the FP32 correction) -> 4 s
#   colour pass, vector (n_u = 3, n_in = 3 right-hand sides) -> 3 s
#   one-launch red-black sweep (Cartesian scalar: u and f, and c)
#                                                   -> 3 s per cell (4 s with c)
# (the finest residuals are FP64-pipe bound: FLOPS_PER_CELL below).
BYTES_PER_CELL = {"smooth64_scalar": 4 * 8, "smooth64_vec": 3 * 8, "smooth32_scalar": 4 * 4,
                  "smooth32_vec": 3 * 4, "resid64_scalar": 4 * 8, "resid64_psi": 4 * 8, "resid64_vec": 9 * 8,
                  "sweep64_fused": 3 * 8, "sweep32_fused": 3 * 4}

# The finest FP64 residuals are bound by the FP64 pipe (GB300 issues 2 FP64
# FMA per SM and clock, 1/64 of its FP32 rate), not by memory.  Algorithmic
# FP64 flops per cell of the spherical operators as the kernels evaluate them
# (+, -, x count one, a multiply-add two; the Newton diagonal excluded):
#   vector, from per-(i, j) stencil coefficients (3 components: 34 + 29 + 29,
#   and f - L: 3); vec_op as written costs 220
#   scalar, linear (flux-form Laplacian 18, - c u, f - L): 22
#   eq. psi, p = 1 + u (the Laplacian 18; p and 1 / p 2, the division
#   counted as one; p^-2, p^-7, p^-8 6; the source S = -(2 pi U p^-1 +
#   A2 p^-7 / 8) 5; L = lap - S and f - L 2; the linearisation K = 2 pi U
#   p^-2 + 7/8 A2 p^-8 of the FP32 correction 4): 37
FLOPS_PER_CELL = {"resid64_vec": 95, "resid64_scalar": 22, "resid64_psi": 37}
FP64_FMA_PER_SM_CLK = 2

# DRAM bytes of one launch (dram__bytes_read.sum + dram__bytes_write.sum)
# from one ncu capture of the current kernel version (cold caches): the
# level-0 FP32 vector colour pass (ghost push included) and the FP64 vector
# residual of the 128x64x64 spherical solve, and the 256^3 one-launch FP32
# sweep.  A kernel changed since its capture has none.
TRAFFIC_PER_LAUNCH = {"smooth32_vec": 9.82e6, "resid64_vec": 29.80e6, "sweep32_fused": 188.61e6}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        self.fh = os.fdopen(fd, "w")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_id), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            self.fh.close()
            os.unlink(self.path)
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def divb_measurement(mg, torch, stream, steps, precision, peak, variant="compact"):
    """Secondary measurement: elliptic div-B cleaning on the 256^3 Cartesian
    cube (the HBM-bound workload: every level-0 array is 128 MB in FP64),
    device-resident B, L2 flushed between cleanings.  variant "exact": the
    exact projection (div_c grad_c Phi = b as 8 parity-class solves of
    128^3); its line also gives the largest deviation of the cleaned
    divergence from its parity-class constants."""
    from paper_2012_07322_gb300 import inputs
    n = 256
    B0 = [torch.from_numpy(b).cuda() for b in inputs.divb_field(n=n)]
    B = [b.clone() for b in B0]
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    desc = mg.grid_desc("cart", [n] * 3, [-1.0] * 3, [1.0] * 3, precision=precision, tol=TOL, max_cycles=200,
                        stall_window=0, divb=variant)
    h = mg.Hierarchy(desc, stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def clean():
        for b, b0 in zip(B, B0):
            b.copy_(b0)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = mg.mg_clean_divB(h, B, phi)
        e1.record(stream)
        torch.cuda.synchronize()
        return rep, e0.elapsed_time(e1)

    clean()
    ms, ups, rep = 0.0, 0, None
    for _ in range(steps):
        rep, t = clean()
        ms += t
        ups += rep["solve"]["cell_updates"]
    class_dev = None
    if variant == "exact":
        # central divergence of the cleaned field (the library's kernel)
        # minus its parity-class means
        div = torch.empty_like(phi)
        mg.mg_divergence(h, B, div)
        class_dev = max(float((div[c::2, b::2, a::2] - div[c::2, b::2, a::2].mean()).abs().max())
                        for a in (0, 1) for b in (0, 1) for c in (0, 1))
        h.close()
        return {"workload": "exact-projection div-B cleaning (div_c grad_c Phi = b, 8 parity-class Neumann "
                            "solves of 128^3), 3D Cartesian 256^3, same field", "precision": precision,
                "value": ups / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_cleaning": ms / steps,
                "cycles_max_class": rep["solve"]["cycles"], "rel": rep["solve"]["rel"],
                "max_div_before": rep["max_div_before"], "max_div_after": rep["max_div_after"],
                "max_div_after_minus_class_means": class_dev}
    mg.mg_profile_enable(h, True)
    clean()
    prof = mg.mg_profile_read(h)
    mg.mg_profile_enable(h, False)
    h.close()
    key = "sweep32_fused" if precision == "mixed" else "sweep64_fused"
    nl, kms, kcells = prof[key]
    bpl = kcells * BYTES_PER_CELL[key] / max(nl, 1)
    ach = bpl / (kms / max(nl, 1) * 1e-3) / 1e9 if nl else 0.0
    return {"workload": "elliptic div-B cleaning, 3D Cartesian 256^3 on [-1,1]^3, curl of 32 seeded modes + "
                        "1e-3 noise, Neumann Poisson", "precision": precision,
            "value": ups / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_cleaning": ms / steps,
            "cycles": rep["solve"]["cycles"], "rel": rep["solve"]["rel"],
            "max_div_before": rep["max_div_before"], "max_div_after": rep["max_div_after"],
            "l2_div_before": rep["l2_div_before"], "l2_div_after": rep["l2_div_after"],
            "roofline": {"bound": "hbm", "kernel": key, "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "traffic": TRAFFIC_PER_LAUNCH.get(key),
                         "avg_launch_us": kms / max(nl, 1) * 1e3,
                         "algorithmic_bytes_per_launch": bpl, "launches": nl}}


# Schedules the batch's autotuner tries per shape class (nu1, nu2,
# accel_depth): the paper's V(2, 2) with mixing depths 16, 8 and none, and
# V(1, 1) with depth 16.
BATCH_CANDIDATES = [(2, 2, 16), (2, 2, 8), (2, 2, 0), (1, 1, 16)]


def batch_measurement(mg, torch, count=512, slots=16, tune=True, rotating=False):
    """Batched solves: 512 uneven 2D static stars (seed 2; half spherical,
    half cylindrical, 32 grid shapes) submitted at once to worker slots that
    overlap their kernels on the device; hierarchies and CUDA graphs are
    cached per shape (warmed once), inputs resident in HBM; and all 512 in
    one persistent launch (mg_solve_cfc_batch, one hierarchy per problem).
    Run with the default schedule (V(2, 2), mixing depth 16) and, with tune,
    with the schedule the autotuner picked per shape class (tuning time
    reported apart)."""
    import time
    from paper_2012_07322_gb300 import autotune, inputs
    batch = (inputs.batch_static_stars_2d(count=count, seed=2, axis_ratio=0.8, omega=0.02) if rotating else
             inputs.batch_static_stars_2d(count=count, seed=2))
    dev = lambda a: torch.from_numpy(np.array(a, copy=True)).cuda()
    items = []
    for (g, n, lo, hi, U, S, Si) in batch:
        desc = mg.grid_desc(g, n, lo, hi, precision="mixed", tol=TOL, max_cycles=800, accel_depth=16,
                            stall_window=0)
        items.append((desc, dev(U), dev(S), [dev(x) for x in Si], g, tuple(n)))
    cells = sum(int(np.prod(it[5])) for it in items)

    def fields(U):
        psi = torch.ones(U.shape, dtype=torch.float64, device="cuda")
        return (psi, torch.ones_like(psi), [torch.zeros_like(psi) for _ in range(3)],
                [torch.zeros_like(psi) for _ in range(3)])

    def run(descs):
        srv = mg.Server(hbm_budget=64 << 30, max_slots=slots, max_queue=2 * count)
        seen = set()
        for d, (_, U, S, Si, g, n) in zip(descs, items):  # one solve per shape: hierarchies and graphs
            if (g, n) in seen:
                continue
            seen.add((g, n))
            srv.wait(srv.submit_cfc(d, U, S, Si, *fields(U)))
        outs = [fields(it[1]) for it in items]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = [srv.submit_cfc(d, U, S, Si, *f) for d, (_, U, S, Si, _, _), f in zip(descs, items, outs)]
        res = [srv.wait(t) for t in tickets]
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        srv.close()
        lat = sorted(r["latency_ms"] for r in res)
        ups = sum(sum(r["cfc"][k]["cell_updates"] for k in ("X", "psi", "alphapsi", "beta")) for r in res)
        cyc = [r["cfc"]["psi"]["cycles"] + r["cfc"]["alphapsi"]["cycles"] for r in res]
        return {"solves_per_s": count / wall, "wall_ms": wall * 1e3, "value": ups / wall / 1e9, "unit": UNIT,
                "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                "ok": sum(r["status"] == "ok" for r in res), "shapes": len(seen),
                "cycles_psi_plus_alphapsi": {"min": min(cyc), "median": sorted(cyc)[len(cyc) // 2],
                                             "max": max(cyc)}}

    def run_persistent(descs, reps=3, launch=None):
        """All solves in one persistent launch (mg_solve_cfc_batch): one
        hierarchy per problem, created once; each timed call starts from the
        flat guess.  Wall time of the call (descriptor upload, the launch,
        the reports back), best of reps; latency = the time from the launch's
        first problem start to the problem's end."""
        hs = [mg.Hierarchy(d) for d in descs]
        outs = [fields(it[1]) for it in items]
        probs = [(h, U, S, Si) + tuple(f) for h, (_, U, S, Si, _, _), f in zip(hs, items, outs)]

        def reset():
            for f in outs:
                f[0].fill_(1.0)
                f[1].fill_(1.0)
        tuned = None
        if launch == "tune":
            t0 = time.perf_counter()
            tuned = autotune.tune_launch(mg, torch, probs, reset)
            tuned["tuning_s"] = time.perf_counter() - t0
        shape = {"team": tuned["team"], "team_cells": tuned["team_cells"]} if tuned else {}
        best = None
        for r in range(reps + 1):  # the first call builds the coarsest operators and mixing storage
            reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res, b = mg.mg_solve_cfc_batch(probs, **shape)
            wall = time.perf_counter() - t0
            if r > 0 and (best is None or wall < best[0]):
                best = (wall, res, b)
        for h in hs:
            h.close()
        wall, res, b = best
        lat = sorted(x["ms"] for x in res)
        ups = sum(sum(x[k]["cell_updates"] for k in ("X", "psi", "alphapsi", "beta")) for x in res)
        cyc = [x["psi"]["cycles"] + x["alphapsi"]["cycles"] for x in res]
        line = {"solves_per_s": count / wall, "wall_ms": wall * 1e3, "kernel_ms": b["kernel_ms"],
                "value": ups / wall / 1e9, "unit": UNIT, "blocks": b["blocks"], "team": b["team"],
                "persistent": b["persistent"],
                "general": b["general"], "p50_ms": lat[len(lat) // 2],
                "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                "ok": sum(x["psi"]["status"] == "ok" and x["alphapsi"]["status"] == "ok" for x in res),
                "cycles_psi_plus_alphapsi": {"min": min(cyc), "median": sorted(cyc)[len(cyc) // 2],
                                             "max": max(cyc)}}
        if tuned:
            line["launch_tuned"] = tuned
        return line

    out = {"workload": "%d uneven 2D %s (seed 2): spherical N_r 32..256 x N_theta 16..128, cylindrical "
                       "N_R 32..256 x N_z 64..512, rho_c ~ U[5e-4, 2e-3], R ~ U[8, 14]; full xCFC system, mixed "
                       "precision; worker slots (%d) and one persistent launch"
                       % (count, "rotating stars (Omega = 0.02, axis ratio 0.8)" if rotating else "static stars",
                          slots), "cells": cells}
    out["default_schedule"] = run([it[0] for it in items])
    out["persistent"] = run_persistent([it[0] for it in items])
    if tune:
        t0 = time.perf_counter()
        table = autotune.tune(mg, torch, [(it[0], (it[1], it[2], it[3])) for it in items],
                              candidates=BATCH_CANDIDATES, repeats=1)
        tuning_s = time.perf_counter() - t0
        tuned = run([autotune.tuned(mg, it[0], table) for it in items])
        picks = {}
        for k, e in table.items():
            key = "nu%d%d_m%d" % (e["nu1"], e["nu2"], e["accel_depth"])
            picks[key] = picks.get(key, 0) + 1
        tuned.update({"tuning_s": tuning_s, "schedules_picked": picks})
        out["autotuned"] = tuned
        out["persistent_autotuned"] = run_persistent([autotune.tuned(mg, it[0], table) for it in items],
                                                     launch="tune")
    return out


# The serving mix: request kinds of the metric streams (geometry, grid) and
# their shares.  The largest uniform grid is the 3D spherical 128 x 64 x 64
# one: the solver needs power-of-two grids, and 192 x 96 x 96 is not one.
# The "amr" kinds are eq. psi on a two-level composite grid refined 2x for
# r < r_max / 4 (static stars; the composite path solves the scalar
# equations); the others the full xCFC system on uniform grids.
SERVE_KINDS = [(("sph", [64, 32], [0.0, 0.0], [100.0, np.pi]), 0.25),
               (("sph", [128, 64], [0.0, 0.0], [100.0, np.pi]), 0.15),
               (("cyl", [64, 128], [0.0, -100.0], [100.0, 100.0]), 0.15),
               (("sph", [32, 16, 16], [0.0, 0.0, 0.0], [100.0, np.pi, 2 * np.pi]), 0.15),
               (("sph", [64, 32, 32], [0.0, 0.0, 0.0], [100.0, np.pi, 2 * np.pi]), 0.10),
               (("sph", [128, 64, 64], [0.0, 0.0, 0.0], [100.0, np.pi, 2 * np.pi]), 0.05),
               (("amr", [64, 32, 32], [0.0, 0.0, 0.0], [100.0, np.pi, 2 * np.pi]), 0.15)]
SERVE_STREAMS = 24
SERVE_STEPS = 4   # source variants per stream: consecutive "time steps" of a slowly changing star


class UtilSampler:
    """nvidia-smi utilization.gpu samples (share of time a kernel ran) while
    requests are served."""

    def __init__(self, gpu_id):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        self.fh = os.fdopen(fd, "w")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_id), "--query-gpu=utilization.gpu",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.fh.close()
        vals = []
        for line in open(self.path):
            try:
                vals.append(float(line.strip()))
            except ValueError:
                pass
        os.unlink(self.path)
        return statistics.median(vals) if vals else None


def serving_setup(mg, torch, precision):
    """Resident inputs of the serving mix: SERVE_STREAMS warm-started xCFC
    streams (seed 3), each with SERVE_STEPS source variants (rho_c grows by
    0.2 % per step), and two div-B fields."""
    from paper_2012_07322_gb300 import inputs
    rng = np.random.default_rng(3)
    dev = lambda a: torch.from_numpy(np.array(a)).cuda()
    shares = np.array([w for _, w in SERVE_KINDS])
    streams = []
    for sid in range(SERVE_STREAMS):
        geom, n, lo, hi = SERVE_KINDS[int(rng.choice(len(SERVE_KINDS), p=shares / shares.sum()))][0]
        rho_c, R = rng.uniform(5e-4, 2e-3), rng.uniform(8.0, 14.0)
        if geom == "amr":
            # base grid and the patch over base cells r < r_max / 4
            box = ([0, 0, 0], [n[0] // 4, n[1], n[2]])
            steps = []
            for t in range(SERVE_STEPS):
                rc = rho_c * (1.0 + 0.002 * t)
                U = inputs.static_polytrope_sph3d(tuple(n), 100.0, rc, R)
                Up = inputs.static_polytrope_sph3d((n[0] // 2, 2 * n[1], 2 * n[2]), 25.0, rc, R)
                steps.append((dev(U), dev(np.zeros_like(U)), dev(Up), dev(np.zeros_like(Up))))
            desc = mg.grid_desc("sph", n, lo, hi, tol=TOL, max_cycles=800, accel_depth=16, stall_window=0)
            streams.append((desc, steps, "amr_sph%s" % "x".join(map(str, n)), box))
            continue
        steps = []
        for t in range(SERVE_STEPS):
            rc = rho_c * (1.0 + 0.002 * t)
            if geom == "cyl":
                U, S, Si = inputs.rotating_polytrope_cyl(n, 100.0, rc, R)
            elif len(n) == 2:
                U, S, Si = inputs.rotating_polytrope_sph2d(n[0], n[1], 100.0, rc, R)
            else:
                U, S, Si = inputs.rotating_polytrope_sph3d(tuple(n), 100.0, rc, R)
            steps.append((dev(U), dev(S), [dev(x) for x in Si]))
        desc = mg.grid_desc(geom, n, lo, hi, precision=precision, tol=TOL, max_cycles=800, accel_depth=16,
                            stall_window=0)
        streams.append((desc, steps, "%s%s" % (geom, "x".join(map(str, n))), None))
    divbs = []
    for n in (32, 64):
        B = inputs.divb_field(n=n, n_modes=16, k_max=6)
        desc = mg.grid_desc("cart", [n] * 3, [-1.0] * 3, [1.0] * 3, precision=precision, tol=TOL, max_cycles=200,
                            stall_window=0)
        divbs.append((desc, [dev(b) for b in B]))
    return streams, divbs


def serving_measurement(mg, torch, precision="mixed", rate=2000.0, n_requests=400, slots=8, gpu_id=None,
                        setup=None):
    """Request serving (continuous batching through mg_submit / mg_poll):
    Poisson arrivals (mean `rate` per second, seed 3) of xCFC solves (80 %,
    SERVE_KINDS; each request of a stream is its next time step, warm-started
    from the stream's resident previous solution) and div-B cleanings (20 %,
    32^3 and 64^3).  Requests are admitted into `slots` worker slots as they
    free up; their kernels overlap on the device.  Reports solves/s, p50 and
    p99 latency (submission to completion), the mean number of requests in
    service (summed service time / wall time) and the median GPU utilization
    (share of time a kernel ran) while serving."""
    import time
    rng = np.random.default_rng(3)
    streams, divbs = setup if setup is not None else serving_setup(mg, torch, precision)
    plan = []
    t = 0.0
    for q in range(n_requests):
        t += rng.exponential(1.0 / rate)
        plan.append((t, "divb" if rng.uniform() < 0.2 else "cfc", int(rng.integers(0, len(streams))),
                     int(rng.integers(0, 2))))
    srv = mg.Server(hbm_budget=96 << 30, max_slots=slots, max_queue=4 * n_requests)

    def fields(U):
        psi = torch.ones(U.shape, dtype=torch.float64, device="cuda")
        return (psi, torch.ones_like(psi), [torch.zeros_like(psi) for _ in range(3)],
                [torch.zeros_like(psi) for _ in range(3)])

    def submit_stream(sid, t):
        desc, steps, name, box = streams[sid]
        if box is not None:
            U, A2, Up, A2p = steps[t % SERVE_STEPS]
            return srv.submit_amr(desc, box[0], box[1], U, A2, Up, A2p, torch.zeros_like(U), torch.zeros_like(Up))
        U, S, Si = steps[t % SERVE_STEPS]
        return srv.submit_cfc(desc, U, S, Si, *fields(U), stream_id=sid + 1)

    # warm the hierarchy cache and the resident streams (first time step)
    for sid in range(len(streams)):
        srv.wait(submit_stream(sid, 0))
    for desc, B in divbs:
        srv.wait(srv.submit_divb(desc, [b.clone() for b in B]))
    torch.cuda.synchronize()
    step_of = [1] * len(streams)
    pending, lat, service, statuses, kinds_done = {}, [], [], [], {}
    util = UtilSampler(gpu_id) if gpu_id is not None else None

    def collect(tk):
        done, res = srv.poll(tk)
        if done:
            lat.append(res["latency_ms"])
            service.append(res["latency_ms"] - res["queue_ms"])
            statuses.append(res["status"])
            k = pending.pop(tk)
            kinds_done.setdefault(k, []).append(res["latency_ms"])
        return done

    t0 = time.perf_counter()
    for (ta, kind, sid, which) in plan:
        while time.perf_counter() - t0 < ta:
            for tk in list(pending):
                collect(tk)
        if kind == "cfc":
            name = streams[sid][2]
            tk = submit_stream(sid, step_of[sid])
            step_of[sid] += 1
        else:
            desc, B = divbs[which]
            name = "divb%d" % desc.n[0]
            tk = srv.submit_divb(desc, [b.clone() for b in B])
        pending[tk] = name
    while pending:
        for tk in list(pending):
            collect(tk)
    wall = time.perf_counter() - t0
    gpu_util = util.stop() if util else None
    srv.close()
    lat.sort()
    pct = lambda a, q: a[min(len(a) - 1, int(q * len(a)))]
    return {"precision": precision, "rate_per_s": rate, "requests": n_requests, "slots": slots,
            "solves_per_s": n_requests / wall, "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99),
            "wall_s": wall, "ok": sum(1 for x in statuses if x == "ok"),
            "mean_in_service": sum(service) / (wall * 1e3), "gpu_util_pct": gpu_util,
            "p50_ms_by_kind": {k: sorted(v)[len(v) // 2] for k, v in sorted(kinds_done.items())}}


def serving_block(mg, torch, gpu_id, sweep):
    """The serving measurement of the bench line: mixed precision at 2000
    requests/s (the serving workload's rate, beyond the server's capacity:
    the queue grows) and at 30/s (below it), 300 requests each; with sweep,
    1000 requests per point at 15 ... 400/s in mixed precision and 5 ... 80/s
    in FP64, across the capacity of each."""
    work = ("Poisson arrivals (seed 3): 80%% metric requests on %d streams (each request the next of %d "
            "time steps of a star; xCFC on uniform grids, warm-started, and eq. psi on two-level AMR grids "
            "refined 2x for r < r_max/4; grids %s), 20%% div-B (32^3, 64^3); continuous admission into "
            "worker slots"
            % (SERVE_STREAMS, SERVE_STEPS, ", ".join("%s %s" % (k[0], "x".join(map(str, k[1])))
                                                      for k, _ in SERVE_KINDS)))
    if not sweep:
        setup = serving_setup(mg, torch, "mixed")
        return {"workload": work,
                "points": [serving_measurement(mg, torch, "mixed", rate, 300, gpu_id=gpu_id, setup=setup)
                           for rate in (2000.0, 30.0)]}
    points = []
    for precision, rates in (("mixed", (15.0, 30.0, 60.0, 100.0, 150.0, 400.0)),
                             ("fp64", (5.0, 10.0, 20.0, 30.0, 80.0))):
        setup = serving_setup(mg, torch, precision)
        for rate in rates:
            points.append(serving_measurement(mg, torch, precision, rate, 1000, gpu_id=gpu_id, setup=setup))
    return {"workload": work, "sweep": points}


def fp64_arm(mg, torch, stream, Ud, Sd, Sid, shp, steps, warmup, accel, max_cycles, mixed_fields):
    """The plain FP64 GPU solve of the same workload (every kernel FP64), timed
    like the headline (L2 flushed between solves), and the per-field
    difference of the mixed-precision solution from it: max |mixed - fp64| /
    max |fp64| for psi, alpha, beta_i and X_i.  The FP64 GPU path matches the
    FP64 oracle to 1e-9 on every field (parity tests), so it stands in for the
    oracle at this size."""
    desc = mg.grid_desc("sph", list(N_GRID), hi=[R_MAX, np.pi, 2 * np.pi], precision="fp64", tol=TOL,
                        max_cycles=max_cycles, accel_depth=accel, stall_window=0)
    h = mg.Hierarchy(desc, stream)
    psi = torch.ones(shp, dtype=torch.float64, device="cuda")
    alpha = torch.ones_like(psi)
    beta = [torch.zeros_like(psi) for _ in range(3)]
    X = [torch.zeros_like(psi) for _ in range(3)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def reset():
        psi.fill_(1.0)
        alpha.fill_(1.0)
        for t in beta + X:
            t.zero_()

    for _ in range(warmup):
        reset()
        mg.mg_solve_cfc(h, Ud, Sd, Sid, psi, alpha, beta, X)
    ms, ups, rep = [], 0, None
    for _ in range(steps):
        reset()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = mg.mg_solve_cfc(h, Ud, Sd, Sid, psi, alpha, beta, X)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        ups += sum(rep[k]["cell_updates"] for k in ("X", "psi", "alphapsi", "beta"))
    h.close()
    # scalars relative to their own maximum, vector components relative to
    # the vector's largest component (as the parity tests measure them): the
    # r and theta components of X and beta vanish in the axisymmetric limit,
    # and their own maxima are iteration noise
    names = ["psi", "alpha", "beta_r", "beta_theta", "beta_phi", "X_r", "X_theta", "X_phi"]
    ref = [psi, alpha] + beta + X
    scale_b = max(float(t.abs().max()) for t in beta)
    scale_x = max(float(t.abs().max()) for t in X)
    err = {}
    for q, (nm, a, b) in enumerate(zip(names, mixed_fields, ref)):
        den = float(b.abs().max()) if q < 2 else (scale_b if q < 5 else scale_x)
        num = float((a - b).abs().max())
        err[nm] = num / den if den > 0 else num
    err["delta_psi"] = float((mixed_fields[0] - psi).abs().max()) / float((psi - 1).abs().max())
    err["delta_alpha"] = float((mixed_fields[1] - alpha).abs().max()) / float((alpha - 1).abs().max())
    lat = sorted(ms)
    return {"precision": "fp64", "value": ups / (sum(ms) * 1e-3) / 1e9, "unit": UNIT,
            "ms_per_solve": sum(ms) / len(ms), "solves_per_s": 1e3 * len(ms) / sum(ms),
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "solves": len(ms), "cycles": {k: rep[k]["cycles"] for k in ("X", "psi", "alphapsi", "beta")},
            "rel": {k: rep[k]["rel"] for k in ("X", "psi", "alphapsi", "beta")}}, err


def oracle_sample(threads):
    """Bounded sample of the workload on the CPU oracle: 2 V-cycles of the X
    (vector) equation and 2 of the psi equation on the full grid.  Returns
    (cell updates, seconds)."""
    os.environ["OMP_NUM_THREADS"] = str(threads)
    import oracle.oracle as orc
    U, S, Si = sources()
    d = orc.desc("sph", list(N_GRID), [0, 0, 0], [R_MAX, np.pi, 2 * np.pi], tol=1e-30, max_cycles=2,
                 stall_window=0)
    cells = level_cells()
    per_cycle = sum(cells[:-1]) * 4          # nu1 + nu2 sweeps on every non-coarsest level
    f = [8 * np.pi * x for x in Si]
    V = [np.zeros(U.shape) for _ in range(3)]
    t0 = time.perf_counter()
    rv = orc.solve_vector(d, "dirichlet", f, V)
    u = np.zeros(U.shape)
    rs = orc.solve_scalar(d, "psi", "robin", u, U=U, A2=np.zeros(U.shape))
    dt = time.perf_counter() - t0
    updates = (rv["cycles"] * 3 + rs["cycles"]) * per_cycle
    return updates, dt


def reference_arm(args):
    """The oracle as the reference arm (rank 0 only under torchrun)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_sample(threads)
    ups, secs = 0, 0.0
    for _ in range(args.steps):
        u, s = oracle_sample(threads)
        ups += u
        secs += s
    value = ups / secs / 1e9
    sample = "2 V-cycles of eq. X (3 components) + 2 of eq. psi on the full 128x64x64 grid per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(N_GRID), "precision": "fp64", "tol": TOL,
                       "cycle": "FAS V(2,2) red-black NGS", "l2": "oracle on host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
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
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2012_07322_gb300 import mg
    mg.lib()

    U, S, Si = sources()
    shp = U.shape
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Ud, Sd, Sid = dev(U), dev(S), [dev(x) for x in Si]
    stream = torch.cuda.current_stream()
    desc = mg.grid_desc("sph", list(N_GRID), hi=[R_MAX, np.pi, 2 * np.pi], precision=args.precision, tol=TOL,
                        max_cycles=args.max_cycles, accel_depth=args.accel, stall_window=0)
    h = mg.Hierarchy(desc, stream)
    psi = torch.ones(shp, dtype=torch.float64, device="cuda")
    alpha = torch.ones_like(psi)
    beta = [torch.zeros_like(psi) for _ in range(3)]
    X = [torch.zeros_like(psi) for _ in range(3)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def reset():
        psi.fill_(1.0)
        alpha.fill_(1.0)
        for t in beta + X:
            t.zero_()

    def solve():
        return mg.mg_solve_cfc(h, Ud, Sd, Sid, psi, alpha, beta, X)

    for _ in range(args.warmup):
        reset()
        solve()
    torch.cuda.synchronize()

    # ---------------------------------------------------------- device-timed
    props = torch.cuda.get_device_properties(local)
    gpu_id = ("GPU-" + str(props.uuid)) if hasattr(props, "uuid") else str(local)
    sampler = ClockSampler(gpu_id)
    ms_steps, updates = [], 0
    launches0 = mg.mg_kernel_launches()
    reps = []
    for _ in range(args.steps):
        reset()
        flush.fill_(1.0)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = solve()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_steps.append(e0.elapsed_time(e1))
        updates += sum(rep[k]["cell_updates"] for k in ("X", "psi", "alphapsi", "beta"))
        reps.append(rep)
    launches = mg.mg_kernel_launches() - launches0
    clocks = sampler.stop()
    # Per-kernel device time: one more identical solve with CUDA events around
    # every finest-level smoother / residual launch on the solver's stream
    # (the timed solves replay CUDA graphs; this one launches directly).
    reset()
    flush.fill_(1.0)
    mg.mg_profile_enable(h, True)
    prof_rep = solve()
    prof = mg.mg_profile_read(h)
    mg.mg_profile_enable(h, False)
    prof_step_ms = prof_rep["ms"]
    total_ms, all_updates = aggregate_ranks(dist, sum(ms_steps), updates, "cuda")
    fp64, mixed_vs_fp64 = None, None
    if args.precision == "mixed" and not args.no_fp64:
        # the mixed solution of the last timed solve (the profiled solve ran
        # the same arithmetic from the same start)
        fp64, mixed_vs_fp64 = fp64_arm(mg, torch, stream, Ud, Sd, Sid, shp, args.fp64_steps, 1, args.accel,
                                       args.max_cycles, [psi, alpha] + beta + X)
    value = all_updates / (total_ms * 1e-3) / 1e9

    # ------------------------------------------------------------------ e2e
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        Uh, Sh, Sih = pin(U), pin(S), [pin(x) for x in Si]
        ph, ah = pin(np.ones(shp)), pin(np.ones(shp))
        bh = [pin(np.zeros(shp)) for _ in range(3)]
        xh = [pin(np.zeros(shp)) for _ in range(3)]
        e2e_ms, e2e_up = 0.0, 0
        for _ in range(args.steps):
            ph.fill_(1.0)
            ah.fill_(1.0)
            for t in bh + xh:
                t.zero_()
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rep = mg.mg_solve_cfc(h, Uh, Sh, Sih, ph, ah, bh, xh, host=True)
            e1.record(stream)
            torch.cuda.synchronize()
            e2e_ms += e0.elapsed_time(e1)
            e2e_up += sum(rep[k]["cell_updates"] for k in ("X", "psi", "alphapsi", "beta"))
        nb = 8 * int(np.prod(shp))
        e2e_ms, e2e_up = aggregate_ranks(dist, e2e_ms, e2e_up, "cuda")
        e2e = {"value": e2e_up / (e2e_ms * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": 13 * nb,
               "d2h_bytes_per_step": 8 * nb}

    # ------------------------------------------------------------ roofline
    peak, peak_kind = load_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    fpeak = FP64_FMA_PER_SM_CLK * 2 * sms * mhz * 1e6 / 1e9

    def class_roofline(name, nl, kms, kcells):
        launch_s = kms / max(nl, 1) * 1e-3
        if name in FLOPS_PER_CELL:
            # FP64-pipe bound: peak from the unit count and the maximum SM clock
            flops_launch = kcells * FLOPS_PER_CELL[name] / max(nl, 1)
            achieved = flops_launch / launch_s / 1e9 if nl else 0.0
            return {"bound": "alu", "achieved": achieved, "peak": fpeak, "unit": "GFLOP/s (FP64)",
                    "frac": achieved / fpeak, "traffic": TRAFFIC_PER_LAUNCH.get(name),
                    "algorithmic_flops_per_launch": flops_launch,
                    "peak_source": "derived: %d FP64 FMA/SM/clock x 2 x %d SMs x %.0f MHz"
                                   % (FP64_FMA_PER_SM_CLK, sms, mhz)}
        bytes_launch = kcells * BYTES_PER_CELL[name] / max(nl, 1)
        achieved = bytes_launch / launch_s / 1e9 if nl else 0.0
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": TRAFFIC_PER_LAUNCH.get(name), "algorithmic_bytes_per_launch": bytes_launch,
                "peak_source": peak_kind}

    # the dominant kernel among the classes of one kernel each (the coarse
    # colour passes, the mixing kernels and the one-block cycle are reported
    # beside them as a breakdown of the step, without a roofline)
    dom = max(((k, v) for k, v in prof.items() if k in BYTES_PER_CELL or k in FLOPS_PER_CELL),
              key=lambda kv: kv[1][1])
    name, (nl, kms, kcells) = dom
    classes = {}
    for k, v in prof.items():
        classes[k] = {"launches": v[0], "ms": v[1]}
        if v[0]:
            classes[k]["avg_launch_us"] = v[1] / v[0] * 1e3
            if k in BYTES_PER_CELL or k in FLOPS_PER_CELL:
                cr = class_roofline(k, *v)
                classes[k].update({"bound": cr["bound"], "frac": cr["frac"]})
    roofline = dict(class_roofline(name, nl, kms, kcells),
                    kernel=name, launches=nl, avg_launch_us=kms / max(nl, 1) * 1e3,
                    share_of_step_time=kms / prof_step_ms if prof_step_ms else None,
                    measured="CUDA events around each finest-level launch of this kernel during one profiled "
                             "solve right after the timed steps (direct launches instead of graph replay)",
                    kernel_classes=classes)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        # repeated samples until about 10 s of oracle time (a bounded share of
        # the workload; the rate is per cell update)
        ups, secs, reps_cpu = 0, 0.0, 0
        while secs < 10.0 and reps_cpu < 64:
            u, t = oracle_sample(threads)
            ups, secs, reps_cpu = ups + u, secs + t, reps_cpu + 1
        cpu = {"value": ups / secs / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d x (2 V-cycles of eq. X (3 components) + 2 of eq. psi) on the full grid, %.1f s"
                         % (reps_cpu, secs)}

    divb = divb_exact = None
    if not args.no_divb:
        divb = divb_measurement(mg, torch, stream, args.steps, args.precision, peak)
        divb_exact = divb_measurement(mg, torch, stream, args.steps, args.precision, peak, variant="exact")
    serving = None
    if not args.no_serve and world == 1:
        serving = serving_block(mg, torch, gpu_id, args.serve_sweep)
    batch = batch_rot = None
    if not args.no_batch and world == 1:
        batch = batch_measurement(mg, torch)
        batch_rot = batch_measurement(mg, torch, tune=False, rotating=True)

    r0 = reps[-1]
    if rank == 0:
        lat = sorted(ms_steps)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(N_GRID), "precision": args.precision, "tol": TOL,
                       "cycle": "FAS V(2,2) red-black NGS", "accel_depth": args.accel,
                       "l2": "flushed between steps (256 MB write)",
                       "cycles": {k: r0[k]["cycles"] for k in ("X", "psi", "alphapsi", "beta")},
                       "rel": {k: r0[k]["rel"] for k in ("X", "psi", "alphapsi", "beta")},
                       "solves_per_s": 1e3 * args.steps * world / total_ms,
                       "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                       "parallelism": "replicas (independent solves per GPU)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "fp64": fp64, "mixed_vs_fp64_err": mixed_vs_fp64,
            "divb_256": divb, "divb_256_exact": divb_exact, "serving": serving, "batch_2d": batch,
            "batch_2d_rotating": batch_rot,
        }
        print(json.dumps(line))
    h.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
