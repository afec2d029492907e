"""Fixed workloads for kernel profiling (ncu), run from the repository root:

    python -m paper_2012_07322_gb300.profile_cases divb256   # mixed 256^3 div-B cleaning, twice
    python -m paper_2012_07322_gb300.profile_cases xeq       # 10 mixed cycles of eq. X, 128x64x64
    python -m paper_2012_07322_gb300.profile_cases xcfc      # one full mixed xCFC solve, 128x64x64
    python -m paper_2012_07322_gb300.profile_cases batch24   # 24 static stars in one persistent launch, twice

Each case runs through the C ABI and exits 0 on success, so the same command
can be profiled after it has run once without a profiler.  Every case
switches the library's event timing on, which makes every cycle run as
direct launches under a host loop (no CUDA graphs): a profiler does not see
the kernels of a graph that holds a conditional (while) node, which is how
the library otherwise runs the cycle loop.  The batch case is one kernel
launch per batch and needs no such switch.
"""
import sys

import numpy as np


def divb256(precision="mixed"):
    import torch
    from . import inputs, mg
    n = 256
    B = [torch.from_numpy(b).cuda() for b in inputs.divb_field(n=n)]
    h = mg.Hierarchy(mg.grid_desc("cart", [n] * 3, [-1.0] * 3, [1.0] * 3, precision=precision, tol=1e-10,
                                  max_cycles=200, stall_window=0))
    rep = None
    mg.mg_profile_enable(h, True)
    for _ in range(2):
        rep = mg.mg_clean_divB(h, [b.clone() for b in B])
    h.close()
    print("divb256", precision, rep["solve"]["cycles"], rep["max_div_before"], rep["max_div_after"])


def xeq(precision="mixed"):
    import torch
    from . import inputs, mg
    n = (128, 64, 64)
    U, S, Si = inputs.rotating_polytrope_sph3d(n, 100.0)
    h = mg.Hierarchy(mg.grid_desc("sph", list(n), hi=[100.0, np.pi, 2 * np.pi], precision=precision, tol=1e-10,
                                  max_cycles=10, stall_window=0, accel_depth=16))
    f = [torch.from_numpy(8 * np.pi * x).cuda() for x in Si]
    V = [torch.zeros(U.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    mg.mg_profile_enable(h, True)
    rep = mg.mg_solve_vector(h, "dirichlet", f, V, allow=(mg.MG_OK, mg.MG_ERR_NOCONV))
    h.close()
    print("xeq", precision, rep["status"], rep["cycles"], rep["rel"])


def xcfc(precision="mixed"):
    import torch
    from . import inputs, mg
    n = (128, 64, 64)
    U, S, Si = inputs.rotating_polytrope_sph3d(n, 100.0)
    h = mg.Hierarchy(mg.grid_desc("sph", list(n), hi=[100.0, np.pi, 2 * np.pi], precision=precision, tol=1e-10,
                                  max_cycles=400, stall_window=0, accel_depth=16))
    dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (U, S)]
    Sid = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in Si]
    psi = torch.ones(U.shape, dtype=torch.float64, device="cuda")
    alpha = torch.ones_like(psi)
    beta = [torch.zeros_like(psi) for _ in range(3)]
    X = [torch.zeros_like(psi) for _ in range(3)]
    mg.mg_profile_enable(h, True)
    rep = mg.mg_solve_cfc(h, dev[0], dev[1], Sid, psi, alpha, beta, X)
    prof = mg.mg_profile_read(h)
    h.close()
    print("xcfc", precision, {k: rep[k]["cycles"] for k in ("X", "psi", "alphapsi", "beta")})
    for k, (n, ms, cells) in prof.items():
        if n:
            print("  %-16s %6d launches %9.3f ms %8.2f us/launch" % (k, n, ms, ms / n * 1e3))


def batch24(precision="mixed"):
    import torch
    from . import inputs, mg
    dev = lambda a: torch.from_numpy(np.array(a, copy=True)).cuda()
    probs = []
    for (g, n, lo, hi, U, S, Si) in inputs.batch_static_stars_2d(count=24, seed=2):
        h = mg.Hierarchy(mg.grid_desc(g, n, lo, hi, precision=precision, tol=1e-10, max_cycles=800, accel_depth=16,
                                      stall_window=0))
        z = lambda: torch.zeros(U.shape, dtype=torch.float64, device="cuda")
        probs.append((h, dev(U), dev(S), [dev(x) for x in Si], z() + 1, z() + 1, [z() for _ in range(3)],
                      [z() for _ in range(3)]))
    for _ in range(2):
        for p in probs:
            p[4].fill_(1.0)
            p[5].fill_(1.0)
        reps, b = mg.mg_solve_cfc_batch(probs)
        print("batch24", b, sum(r["psi"]["status"] == "ok" and r["alphapsi"]["status"] == "ok" for r in reps))
    for p in probs:
        p[0].close()


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "divb256"
    prec = sys.argv[2] if len(sys.argv) > 2 else "mixed"
    {"divb256": divb256, "xeq": xeq, "xcfc": xcfc, "batch24": batch24}[case](prec)
