"""Autotuner of cycle schedules per grid shape class.

A batch of uneven solves (many grids of a few shapes) spends most of its
time in the cycle loop of each solve.  The schedule that reaches the
tolerance fastest depends on the shape: on spherical grids the point
smoother contracts slowly near the axis and Anderson mixing pays, on small
cylindrical grids the mixing step costs more than the cycles it saves, and
the pre/post smoothing counts trade cycles against work per cycle.  The
tuner solves one representative of each shape class (geometry, grid,
precision) with every candidate schedule through the library's own entry
point, keeps the fastest that converges, and records it in a JSON table
that later runs reuse.

Every candidate is the same multigrid (Sec. 2.7) with the same stopping
rule, so the tuned solves reach the same tolerance; only the route there
changes (V(nu1, nu2) counts and the mixing depth).

tune_launch picks the launch shape of the persistent batch kernel for a
given batch: the cluster size that runs one large grid and the grid size
from which a cluster takes a problem (the rest run one block each), by the
measured time of the whole batch per candidate.
"""
from __future__ import annotations

import json
import os
import time

# Candidate schedules: (nu1, nu2, accel_depth).  V(2, 2) is the paper's
# smoothing; accel_depth 0 its plain iteration.
CANDIDATES = [(2, 2, 16), (2, 2, 8), (2, 2, 4), (2, 2, 0), (1, 1, 16), (1, 1, 8), (2, 1, 16), (3, 3, 16)]


def shape_key(desc) -> str:
    """Key of a descriptor's shape class: geometry, cells per dimension,
    precision."""
    nd = desc.ndim
    return "g%d_n%s_p%d" % (desc.geom, "x".join(str(desc.n[k]) for k in range(nd)), desc.precision)


def with_schedule(mg, desc, sched):
    """A copy of desc with the schedule (nu1, nu2, accel_depth) applied."""
    d = mg.mg_grid_desc()
    for name, _ in mg.mg_grid_desc._fields_:
        v = getattr(desc, name)
        if hasattr(v, "_length_"):
            arr = getattr(d, name)
            for k in range(len(v)):
                arr[k] = v[k]
        else:
            setattr(d, name, v)
    d.nu1, d.nu2, d.accel_depth = sched
    return d


def load(path):
    if path and os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def save(path, table):
    if not path:
        return
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_solve(mg, torch, desc, src, repeats):
    """Wall milliseconds of one xCFC solve (the median of repeats after one
    warm-up solve that builds the hierarchy's graphs), its status and the
    psi + alpha-psi cycles."""
    U, S, Si = src
    h = mg.Hierarchy(desc)
    try:
        def fields():
            psi = torch.ones(U.shape, dtype=torch.float64, device="cuda")
            return (psi, torch.ones_like(psi), [torch.zeros_like(psi) for _ in range(3)],
                    [torch.zeros_like(psi) for _ in range(3)])
        allow = (mg.MG_OK, mg.MG_ERR_NOCONV, mg.MG_ERR_STALLED)
        mg.mg_solve_cfc(h, U, S, Si, *fields(), allow=allow)
        ms, rep = [], None
        for _ in range(repeats):
            f = fields()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = mg.mg_solve_cfc(h, U, S, Si, *f, allow=allow)
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t0) * 1e3)
        ok = all(rep[k]["status"] == "ok" for k in ("X", "psi", "alphapsi", "beta"))
        return sorted(ms)[len(ms) // 2], ok, rep["psi"]["cycles"] + rep["alphapsi"]["cycles"]
    finally:
        h.close()


def tune(mg, torch, items, path=None, candidates=CANDIDATES, repeats=2):
    """Tune the schedule of every shape class among items, a list of
    (desc, (U, S, Si)) with device tensors; classes already in the table at
    path are kept.  Returns the table {key: {"nu1", "nu2", "accel_depth",
    "ms", "cycles", "tried"}}."""
    table = load(path)
    seen = {}
    for desc, src in items:
        seen.setdefault(shape_key(desc), (desc, src))
    for key, (desc, src) in seen.items():
        if key in table:
            continue
        best, tried = None, []
        for sched in candidates:
            ms, ok, cyc = _time_solve(mg, torch, with_schedule(mg, desc, sched), src, repeats)
            tried.append({"nu1": sched[0], "nu2": sched[1], "accel_depth": sched[2], "ms": ms, "ok": ok,
                          "cycles": cyc})
            if ok and (best is None or ms < best[0]):
                best = (ms, sched, cyc)
        if best is None:
            continue
        table[key] = {"nu1": best[1][0], "nu2": best[1][1], "accel_depth": best[1][2], "ms": best[0],
                      "cycles": best[2], "tried": tried}
    save(path, table)
    return table


def tuned(mg, desc, table):
    """desc with its shape class's tuned schedule (unchanged if untuned)."""
    e = table.get(shape_key(desc))
    if not e:
        return desc
    return with_schedule(mg, desc, (e["nu1"], e["nu2"], e["accel_depth"]))


# Candidate launch shapes of the persistent batch: (team, team_cells).
LAUNCH_CANDIDATES = [(2, 16384), (2, 32768), (2, 8192), (4, 16384), (4, 32768), (8, 32768), (1, 0)]


def tune_launch(mg, torch, problems, reset, candidates=LAUNCH_CANDIDATES, repeats=1):
    """The fastest launch shape for a batch.  problems: the tuple list
    mg.mg_solve_cfc_batch takes; reset(): restores the initial guesses.
    Each candidate runs once untimed (the problems' cycle history orders the
    queue) and then repeats timed times; returns {"team", "team_cells",
    "ms", "tried"}."""
    best, tried = None, []
    for team, cells in candidates:
        ms = []
        for r in range(repeats + 1):
            reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps, b = mg.mg_solve_cfc_batch(problems, reports=False, team=team, team_cells=cells,
                                            allow=(mg.MG_OK, mg.MG_ERR_NOCONV, mg.MG_ERR_STALLED))
            if r > 0:
                ms.append((time.perf_counter() - t0) * 1e3)
        t = sorted(ms)[len(ms) // 2]
        ok = b["status"] == "ok"
        tried.append({"team": team, "team_cells": cells, "ms": t, "ok": ok, "blocks": b["blocks"]})
        if ok and (best is None or t < best[0]):
            best = (t, team, cells)
    if best is None:
        return {"team": 0, "team_cells": 0, "ms": None, "tried": tried}
    return {"team": best[1], "team_cells": best[2], "ms": best[0], "tried": tried}
