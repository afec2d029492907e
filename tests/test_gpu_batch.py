"""The persistent batched xCFC solve (mg_solve_cfc_batch): uneven 2D static
stars solved in one launch, one thread block per problem at a time.

Parity: every field within 1e-9 of the FP64 oracle at a converged relative
residual of 1e-10 (the bar of the mixed-precision solves), X = beta = 0
exactly for static stars, cycle counts close to the launched mixed path's,
for static and rotating stars.  A problem's result does not depend on the
batch it runs in (one block runs it with the same instructions)."""
import numpy as np
import pytest

import oracle.oracle as o
from paper_2012_07322_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PI = np.pi


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_07322_gb300 import mg as m
    m.lib()
    return m


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.float64, copy=True)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


# (geom, n, rho_c, R): the whole correction cycle in one block (2048 cells),
# and grids whose finest levels run the block-strided phases (8192, 16384
# and 32768 cells)
STARS = [("sph", [64, 32], 1.28e-3, 10.0), ("cyl", [32, 64], 9e-4, 12.0), ("sph", [128, 64], 1.6e-3, 9.0),
         ("cyl", [64, 128], 7e-4, 13.0), ("sph", [64, 128], 1.1e-3, 11.0), ("cyl", [32, 512], 1.9e-3, 8.5)]


def star(geom, n, rho_c, R, omega=0.0):
    if geom == "sph":
        U, S, Si = inputs.rotating_polytrope_sph2d(n[0], n[1], 100.0, rho_c, R, axis_ratio=1.0, omega=omega)
        return U, S, Si, [0.0, 0.0], [100.0, PI]
    U, S, Si = inputs.rotating_polytrope_cyl(n, 100.0, rho_c, R, axis_ratio=1.0, omega=omega)
    return U, S, Si, [0.0, -100.0], [100.0, 100.0]


def problem(mg, geom, n, rho_c, R, accel=16, omega=0.0, **kw):
    U, S, Si, lo, hi = star(geom, n, rho_c, R, omega)
    d = mg.grid_desc(geom, n, lo, hi, precision="mixed", tol=1e-10, max_cycles=800, accel_depth=accel,
                     stall_window=0, **kw)
    h = mg.Hierarchy(d)
    shp = U.shape
    f = (torch.ones(shp, dtype=torch.float64, device="cuda"), torch.ones(shp, dtype=torch.float64, device="cuda"),
         [torch.zeros(shp, dtype=torch.float64, device="cuda") for _ in range(3)],
         [torch.zeros(shp, dtype=torch.float64, device="cuda") for _ in range(3)])
    return {"h": h, "desc": d, "np": (U, S, Si, lo, hi), "dev": (dev(U), dev(S), [dev(x) for x in Si]), "f": f,
            "geom": geom, "n": n}


def as_tuple(p):
    U, S, Si = p["dev"]
    psi, alpha, beta, X = p["f"]
    return (p["h"], U, S, Si, psi, alpha, beta, X)


def close(ps):
    for p in ps:
        p["h"].close()


def test_batch_matches_oracle(mg):
    """Six uneven static stars in one launch against the FP64 oracle's xCFC
    solve: psi and alpha within 1e-9, residual 1e-10, X and beta exactly 0."""
    ps = [problem(mg, *s) for s in STARS]
    reps, b = mg.mg_solve_cfc_batch([as_tuple(p) for p in ps])
    assert b["status"] == "ok" and b["persistent"] == len(ps) and b["general"] == 0, b
    for p, r in zip(ps, reps):
        U, S, Si, lo, hi = p["np"]
        d = o.desc(p["geom"], p["n"], lo, hi, tol=1e-10, max_cycles=1000, stall_window=0, accel_depth=16)
        shp = U.shape
        psi, alpha = np.ones(shp), np.ones(shp)
        beta = [np.zeros(shp) for _ in range(3)]
        X = [np.zeros(shp) for _ in range(3)]
        ro = o.solve_cfc(d, U, S, Si, psi, alpha, beta, X)
        for k in ("psi", "alphapsi"):
            assert ro[k]["status"] == "ok" and r[k]["status"] == "ok", (p["n"], k, r[k]["status"])
            assert r[k]["rel"] <= 1e-10 and r[k]["cycles"] > 0
            assert r[k]["hist"][-1] == r[k]["rel"] and len(r[k]["hist"]) == r[k]["cycles"] + 1
        for k in ("X", "beta"):
            assert r[k]["status"] == "ok" and r[k]["cycles"] == 0 and r[k]["rel"] == 0.0
        gp, ga = host(p["f"][0]), host(p["f"][1])
        errs = {"psi": relerr(gp, psi), "dpsi": relerr(gp - 1, psi - 1), "alpha": relerr(ga, alpha),
                "dalpha": relerr(ga - 1, alpha - 1)}
        assert max(errs.values()) < 1e-9, (p["geom"], p["n"], errs)
        assert all((host(x) == 0).all() for x in p["f"][2] + p["f"][3])
        assert r["ms"] > 0
    close(ps)


def test_batch_cycles_close_to_launched_path(mg):
    """The same problems through mg_solve_cfc (launched kernels, CUDA
    graphs): the persistent solve runs the same iteration, so its cycle
    counts differ only through the rounding order of the mixing sums."""
    ps = [problem(mg, *s) for s in STARS]
    reps, _ = mg.mg_solve_cfc_batch([as_tuple(p) for p in ps])
    for s, p, r in zip(STARS, ps, reps):
        q = problem(mg, *s)
        ra = mg.mg_solve_cfc(*as_tuple(q))
        for k in ("psi", "alphapsi"):
            c0, c1 = ra[k]["cycles"], r[k]["cycles"]
            assert abs(c0 - c1) <= max(2, 0.15 * c0), (p["n"], k, c0, c1)
        for a, b in [(q["f"][0], p["f"][0]), (q["f"][1], p["f"][1])]:
            assert relerr(host(b), host(a)) < 2e-9
        q["h"].close()
    close(ps)


def test_batch_result_independent_of_the_mix(mg):
    """One block runs a problem from start to end with the same
    instructions whatever else the launch holds: a problem solved alone
    (a batch of one) and inside the batch gives bitwise the same fields,
    and so does a second run of the whole batch."""
    ps = [problem(mg, *s) for s in STARS]
    mg.mg_solve_cfc_batch([as_tuple(p) for p in ps])
    first = [(p["f"][0].clone(), p["f"][1].clone()) for p in ps]
    for p in ps:
        p["f"][0].fill_(1.0)
        p["f"][1].fill_(1.0)
    mg.mg_solve_cfc_batch([as_tuple(p) for p in reversed(ps)])
    for p, (a, b) in zip(ps, first):
        assert torch.equal(p["f"][0], a) and torch.equal(p["f"][1], b)
    alone = problem(mg, *STARS[3])
    mg.mg_solve_cfc_batch([as_tuple(alone)])
    assert torch.equal(alone["f"][0], first[3][0]) and torch.equal(alone["f"][1], first[3][1])
    close(ps + [alone])


def test_batch_psi_only_and_no_mixing(mg):
    """Eq. psi alone (MG_CFC_PSI_ONLY), and plain cycles without mixing,
    against the oracle."""
    for accel, psi_only, stars in [(0, False, STARS[:2]), (16, True, STARS[:4])]:
        ps = [problem(mg, *s, accel=accel) for s in stars]
        reps, b = mg.mg_solve_cfc_batch([as_tuple(p) for p in ps], psi_only=psi_only)
        assert b["status"] == "ok"
        for p, r in zip(ps, reps):
            U, S, Si, lo, hi = p["np"]
            d = o.desc(p["geom"], p["n"], lo, hi, tol=1e-10, max_cycles=1000, stall_window=0, accel_depth=accel)
            psi, alpha = np.ones(U.shape), np.ones(U.shape)
            z = [np.zeros(U.shape) for _ in range(3)]
            o.solve_cfc(d, U, S, Si, psi, alpha, z, [x.copy() for x in z], psi_only=psi_only)
            assert r["psi"]["status"] == "ok" and r["psi"]["rel"] <= 1e-10
            assert relerr(host(p["f"][0]) - 1, psi - 1) < 1e-9
            if psi_only:
                assert (host(p["f"][1]) == 1).all() and r["alphapsi"]["cycles"] == 0
            else:
                assert relerr(host(p["f"][1]) - 1, alpha - 1) < 1e-9
        close(ps)


ROTATING = [("sph", [64, 32], 1.28e-3, 10.0), ("cyl", [32, 64], 9e-4, 12.0), ("sph", [32, 16], 1.6e-3, 9.0),
            ("cyl", [64, 128], 1.1e-3, 11.0), ("sph", [128, 64], 1.3e-3, 10.5)]


def test_batch_rotating_stars_match_oracle(mg):
    """Rotating stars (S_i != 0) in the launch with static ones: the kernel
    solves all four equations (X and beta by the vector V-cycle), every
    field within 1e-9 of the FP64 oracle's xCFC solve (vector components
    scaled by the vector's maximum), residual 1e-10 in every equation."""
    ps = [problem(mg, *STARS[0])] + [problem(mg, *s, omega=0.02) for s in ROTATING] + [problem(mg, *STARS[1])]
    reps, b = mg.mg_solve_cfc_batch([as_tuple(p) for p in ps])
    assert b["persistent"] == len(ps) and b["general"] == 0 and b["status"] == "ok", b
    for p, r in zip(ps, reps):
        U, S, Si, lo, hi = p["np"]
        d = o.desc(p["geom"], p["n"], lo, hi, tol=1e-10, max_cycles=1000, stall_window=0, accel_depth=16)
        shp = U.shape
        psi, alpha = np.ones(shp), np.ones(shp)
        beta = [np.zeros(shp) for _ in range(3)]
        X = [np.zeros(shp) for _ in range(3)]
        ro = o.solve_cfc(d, U, S, Si, psi, alpha, beta, X)
        moving = any(np.abs(x).max() > 0 for x in Si)
        for k in ("X", "psi", "alphapsi", "beta"):
            assert ro[k]["status"] == "ok" and r[k]["status"] == "ok", (p["n"], k, r[k]["status"])
            assert r[k]["rel"] <= 1e-10 and len(r[k]["hist"]) == r[k]["cycles"] + 1
            if k in ("X", "beta"):
                assert (r[k]["cycles"] > 0) == moving, (p["n"], k, r[k]["cycles"])
        got = {"psi": host(p["f"][0]), "alpha": host(p["f"][1])}
        errs = {"psi": relerr(got["psi"], psi), "dpsi": relerr(got["psi"] - 1, psi - 1),
                "alpha": relerr(got["alpha"], alpha), "dalpha": relerr(got["alpha"] - 1, alpha - 1)}
        for name, want, t in (("beta", beta, p["f"][2]), ("X", X, p["f"][3])):
            scale = max(np.abs(x).max() for x in want)
            errs[name] = max(np.abs(host(g) - w).max() for g, w in zip(t, want)) / (scale or 1.0)
        assert max(errs.values()) < 1e-9, (p["geom"], p["n"], errs)
    close(ps)


def test_batch_rotating_stars_close_to_launched_path(mg):
    """The same rotating stars through mg_solve_cfc: the same iteration, so
    the fields agree within the rounding of the mixing sums and the cycle
    counts within 15 %."""
    ps = [problem(mg, *s, omega=0.02) for s in ROTATING]
    reps, _ = mg.mg_solve_cfc_batch([as_tuple(p) for p in ps])
    for s, p, r in zip(ROTATING, ps, reps):
        q = problem(mg, *s, omega=0.02)
        ra = mg.mg_solve_cfc(*as_tuple(q))
        for k in ("X", "psi", "alphapsi", "beta"):
            c0, c1 = ra[k]["cycles"], r[k]["cycles"]
            assert abs(c0 - c1) <= max(2, 0.15 * c0), (p["n"], k, c0, c1)
        for a, c in zip([q["f"][0], q["f"][1]], [p["f"][0], p["f"][1]]):
            assert relerr(host(c), host(a)) < 2e-9
        for name in (2, 3):
            scale = max(np.abs(host(x)).max() for x in q["f"][name])
            assert max(np.abs(host(c) - host(a)).max() for a, c in zip(q["f"][name], p["f"][name])) < 2e-9 * scale
        q["h"].close()
    close(ps)


def test_batch_3d_grids_match_oracle(mg):
    """3D grids in the launch (the kernel's passes are dimension- and
    geometry-generic): rotating stars on a spherical 32 x 16 x 16, a
    cylindrical 16 x 32 x 8 and a Cartesian 16^3 grid beside a 2D static
    star, every field within 1e-9 of the oracle."""
    cases = [("sph", [32, 16, 16], [0.0, 0.0, 0.0], [100.0, PI, 2 * PI]),
             ("cyl", [16, 32, 8], [0.0, -100.0, 0.0], [100.0, 100.0, 2 * PI]),
             ("cart", [16, 16, 16], [-30.0] * 3, [30.0] * 3)]
    ps, srcs = [], []
    for geom, n, lo, hi in cases:
        if geom == "sph":
            U, S, Si = inputs.rotating_polytrope_sph3d(tuple(n), 100.0)
        elif geom == "cyl":
            U, S, Si = inputs.rotating_polytrope_cyl(n, 100.0)
        else:
            U, S, Si = inputs.rotating_polytrope_cart3d(tuple(n), 30.0)
        d = mg.grid_desc(geom, n, lo, hi, precision="mixed", tol=1e-10, max_cycles=800, accel_depth=16,
                         stall_window=0)
        shp = U.shape
        f = (torch.ones(shp, dtype=torch.float64, device="cuda"), torch.ones(shp, dtype=torch.float64, device="cuda"),
             [torch.zeros(shp, dtype=torch.float64, device="cuda") for _ in range(3)],
             [torch.zeros(shp, dtype=torch.float64, device="cuda") for _ in range(3)])
        ps.append({"h": mg.Hierarchy(d), "dev": (dev(U), dev(S), [dev(x) for x in Si]), "f": f})
        srcs.append((geom, n, lo, hi, U, S, Si))
    ps.append(problem(mg, *STARS[2]))
    reps, b = mg.mg_solve_cfc_batch([as_tuple(p) for p in ps])
    assert b["status"] == "ok" and b["persistent"] == 4 and b["general"] == 0, b
    for p, r, (geom, n, lo, hi, U, S, Si) in zip(ps, reps, srcs):
        d = o.desc(geom, n, lo, hi, tol=1e-10, max_cycles=1000, stall_window=0, accel_depth=16)
        shp = U.shape
        psi, alpha = np.ones(shp), np.ones(shp)
        beta = [np.zeros(shp) for _ in range(3)]
        X = [np.zeros(shp) for _ in range(3)]
        ro = o.solve_cfc(d, U, S, Si, psi, alpha, beta, X)
        for k in ("X", "psi", "alphapsi", "beta"):
            assert ro[k]["status"] == "ok" and r[k]["status"] == "ok", (n, k, r[k]["status"])
            assert r[k]["rel"] <= 1e-10 and r[k]["cycles"] > 0
        errs = {"psi": relerr(host(p["f"][0]) - 1, psi - 1), "alpha": relerr(host(p["f"][1]) - 1, alpha - 1)}
        for name, want, t in (("beta", beta, p["f"][2]), ("X", X, p["f"][3])):
            scale = max(np.abs(x).max() for x in want)
            errs[name] = max(np.abs(host(g) - w).max() for g, w in zip(t, want)) / (scale or 1.0)
        assert max(errs.values()) < 1e-9, (geom, n, errs)
    close(ps)


@pytest.mark.parametrize("team,team_cells", [(1, 0), (4, 8192), (8, 8192)])
def test_batch_launch_shapes(mg, team, team_cells):
    """Single blocks only, and clusters of 4 and 8 blocks taking every grid
    of 8192 cells and more: the same iteration, so the fields agree with the
    default launch's within the rounding of the mixing sums, every solve
    converges, and three runs give the same fields bit for bit."""
    ps = [problem(mg, *s) for s in STARS]
    ref, _ = mg.mg_solve_cfc_batch([as_tuple(p) for p in ps])
    want = [(host(p["f"][0]), host(p["f"][1])) for p in ps]
    for p in ps:
        p["f"][0].fill_(1.0)
        p["f"][1].fill_(1.0)
    runs = []
    for _ in range(3):
        for p in ps:
            p["f"][0].fill_(1.0)
            p["f"][1].fill_(1.0)
        reps, b = mg.mg_solve_cfc_batch([as_tuple(p) for p in ps], team=team, team_cells=team_cells)
        assert b["status"] == "ok" and b["team"] == team, b
        for p, r, r0, (a, c) in zip(ps, reps, ref, want):
            for k in ("psi", "alphapsi"):
                assert r[k]["status"] == "ok" and r[k]["rel"] <= 1e-10
                assert abs(r[k]["cycles"] - r0[k]["cycles"]) <= max(2, 0.15 * r0[k]["cycles"])
            assert relerr(host(p["f"][0]), a) < 2e-9 and relerr(host(p["f"][1]), c) < 2e-9
        runs.append(([p["f"][0].clone() for p in ps], [(r["psi"]["cycles"], r["alphapsi"]["cycles"]) for r in reps]))
    # a team's blocks meet at the same barriers and reduce in a fixed order:
    # the runs agree bit for bit
    for fields, cycles in runs[1:]:
        assert cycles == runs[0][1]
        assert all(torch.equal(x, y) for x, y in zip(fields, runs[0][0]))
    close(ps)


def test_batch_rejects_bad_arguments(mg):
    """Before any work: the same hierarchy twice, a cluster of 3 blocks, an
    FP64 hierarchy, and FMG cycles."""
    a, b = problem(mg, *STARS[0]), problem(mg, *STARS[1])
    with pytest.raises(mg.MgError):
        mg.mg_solve_cfc_batch([as_tuple(a), as_tuple(a)])
    with pytest.raises(mg.MgError):
        mg.mg_solve_cfc_batch([as_tuple(a), as_tuple(b)], team=3)
    for kw in [{"precision": "fp64"}, {"cycle": "fmg"}]:
        U, S, Si, lo, hi = b["np"]
        args = dict(precision="mixed", tol=1e-10, max_cycles=800, accel_depth=16)
        args.update(kw)
        d = mg.grid_desc(b["geom"], b["n"], lo, hi, **args)
        h = mg.Hierarchy(d)
        t = as_tuple(b)
        with pytest.raises(mg.MgError):
            mg.mg_solve_cfc_batch([as_tuple(a), (h,) + t[1:]])
        h.close()
    # nothing was written: the guesses are untouched
    assert (host(a["f"][0]) == 1).all() and (host(b["f"][0]) == 1).all()
    close([a, b])
