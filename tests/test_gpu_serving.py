"""Request serving (mg_submit / mg_poll): continuous admission into worker
slots whose kernels overlap on the device, hierarchy reuse, resident warm
starts per stream, admission by HBM budget.

Each result must be the same alone and in the mix: the solver's arithmetic
does not depend on what runs beside it (fixed reduction orders, per-request
hierarchies), so results are compared bit for bit."""
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


def cfc_case(kind, seed):
    """(desc args, U, S, Si) of a jittered rotating star."""
    rng = np.random.default_rng(seed)
    rho_c, R = rng.uniform(8e-4, 1.6e-3), rng.uniform(8.0, 12.0)
    if kind == "sph2d":
        U, S, Si = inputs.rotating_polytrope_sph2d(64, 32, 100.0, rho_c, R)
        return ("sph", [64, 32], [0.0, 0.0], [100.0, PI]), U, S, Si
    if kind == "sph3d":
        U, S, Si = inputs.rotating_polytrope_sph3d((32, 16, 16), 100.0, rho_c, R)
        return ("sph", [32, 16, 16], [0.0, 0.0, 0.0], [100.0, PI, 2 * PI]), U, S, Si
    U, S, Si = inputs.rotating_polytrope_cyl([32, 64], 100.0, rho_c, R)
    return ("cyl", [32, 64], [0.0, -100.0], [100.0, 100.0]), U, S, Si


def fields(shape):
    psi = torch.ones(shape, dtype=torch.float64, device="cuda")
    return psi, torch.ones_like(psi), [torch.zeros_like(psi) for _ in range(3)], [torch.zeros_like(psi) for _ in range(3)]


def desc_of(mg, args, accel=8):
    geom, n, lo, hi = args
    return mg.grid_desc(geom, n, lo, hi, tol=1e-10, max_cycles=600, accel_depth=accel, stall_window=0)


def test_results_identical_alone_and_in_the_mix(mg):
    cases = [("sph2d", 1), ("sph3d", 2), ("cyl2d", 3), ("sph2d", 4), ("sph3d", 5), ("cyl2d", 6)]
    reqs = []
    for kind, seed in cases:
        args, U, S, Si = cfc_case(kind, seed)
        reqs.append(("cfc", args, [dev(U), dev(S), [dev(x) for x in Si]]))
    for n, seed in [(32, 7), (16, 8)]:
        B = inputs.divb_field(n=n, n_modes=8, k_max=4, seed_modes=seed, seed_noise=seed + 1)
        reqs.append(("divb", ("cart", [n] * 3, [-1.0] * 3, [1.0] * 3), [dev(b) for b in B]))
    # alone: one hierarchy per request, direct calls
    alone = []
    for kind, args, data in reqs:
        h = mg.Hierarchy(desc_of(mg, args))
        if kind == "cfc":
            psi, alpha, beta, X = fields(data[0].shape)
            mg.mg_solve_cfc(h, data[0], data[1], data[2], psi, alpha, beta, X)
            alone.append([psi, alpha] + beta + X)
        else:
            B = [b.clone() for b in data]
            mg.mg_clean_divB(h, B)
            alone.append(B)
        h.close()
    # in the mix: everything submitted at once, twice over, to 4 slots
    srv = mg.Server(hbm_budget=8 << 30, max_slots=4, max_queue=64)
    tickets, outs = [], []
    for rep in range(2):
        for kind, args, data in reqs:
            if kind == "cfc":
                psi, alpha, beta, X = fields(data[0].shape)
                t = srv.submit_cfc(desc_of(mg, args), data[0], data[1], data[2], psi, alpha, beta, X)
                outs.append([psi, alpha] + beta + X)
            else:
                B = [b.clone() for b in data]
                t = srv.submit_divb(desc_of(mg, args), B)
                outs.append(B)
            tickets.append(t)
    results = [srv.wait(t) for t in tickets]
    srv.close()
    assert all(r["status"] == "ok" for r in results)
    for q, out in enumerate(outs):
        ref = alone[q % len(reqs)]
        for a, b in zip(out, ref):
            assert torch.equal(a, b), q
    # the first request (2D spherical 64 x 32), the same alone and in the
    # mix, is also the oracle's solution
    args, U, S, Si = cfc_case("sph2d", 1)
    geom, n, lo, hi = args
    d = o.desc(geom, n, lo, hi, tol=1e-10, max_cycles=600, accel_depth=8, stall_window=0)
    psi, alpha = np.ones(U.shape), np.ones(U.shape)
    beta, X = [np.zeros(U.shape) for _ in range(3)], [np.zeros(U.shape) for _ in range(3)]
    ro = o.solve_cfc(d, U, S, Si, psi, alpha, beta, X)
    assert ro["status"] == "ok"
    got = [t.cpu().numpy() for t in outs[0]]
    for a, b in zip(got[:2], [psi, alpha]):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()
    for lo_, hi_ in ((2, 5), (5, 8)):
        want = (beta if lo_ == 2 else X)
        scale = max(np.abs(w).max() for w in want)
        assert max(np.abs(a - b).max() for a, b in zip(got[lo_:hi_], want)) <= 1e-9 * scale


def test_warm_start_of_a_stream(mg):
    """The second request of a stream starts from the first one's resident
    solution: with unchanged sources it is converged at cycle 0."""
    args, U, S, Si = cfc_case("sph2d", 11)
    d = desc_of(mg, args)
    srv = mg.Server(hbm_budget=2 << 30, max_slots=2, max_queue=8)
    Ud, Sd, Sid = dev(U), dev(S), [dev(x) for x in Si]
    f1 = fields(U.shape)
    r1 = srv.wait(srv.submit_cfc(d, Ud, Sd, Sid, *f1, stream_id=42))
    f2 = fields(U.shape)
    r2 = srv.wait(srv.submit_cfc(d, Ud, Sd, Sid, *f2, stream_id=42))
    srv.close()
    assert r1["status"] == "ok" and r2["status"] == "ok"
    assert not r1["warm_started"] and r2["warm_started"]
    assert r1["cfc"]["psi"]["cycles"] > 0
    assert all(r2["cfc"][k]["cycles"] == 0 for k in ("X", "psi", "alphapsi", "beta"))
    assert torch.equal(f1[0], f2[0])


def test_admission_by_budget_and_queue(mg):
    args, U, S, Si = cfc_case("sph3d", 12)
    d = desc_of(mg, args)
    need = mg.mg_hierarchy_bytes(d)
    # a request larger than the whole budget is refused at submission
    small = mg.Server(hbm_budget=need // 2, max_slots=1, max_queue=4)
    Ud, Sd, Sid = dev(U), dev(S), [dev(x) for x in Si]
    st = small.submit_cfc(d, Ud, Sd, Sid, *fields(U.shape), allow=(mg.MG_OK, mg.MG_ERR_OOM))
    assert st is None
    small.close()
    # a full queue refuses with MG_ERR_BUSY; everything admitted completes
    srv = mg.Server(hbm_budget=need + (64 << 20), max_slots=1, max_queue=2)
    tickets, busy = [], 0
    for _ in range(8):
        t = srv.submit_cfc(d, Ud, Sd, Sid, *fields(U.shape), allow=(mg.MG_OK, mg.MG_ERR_BUSY))
        if t is None:
            busy += 1
        else:
            tickets.append(t)
    results = [srv.wait(t) for t in tickets]
    srv.close()
    assert busy > 0
    assert all(r["status"] == "ok" for r in results)


def test_eviction_keeps_results_correct(mg):
    """A budget for one hierarchy at a time: alternating grids evict and
    recreate hierarchies; each result still equals the direct solve."""
    a_args, Ua, Sa, Sia = cfc_case("sph2d", 21)
    b_args, Ub, Sb, Sib = cfc_case("cyl2d", 22)
    da, db = desc_of(mg, a_args), desc_of(mg, b_args)
    budget = max(mg.mg_hierarchy_bytes(da), mg.mg_hierarchy_bytes(db)) + (1 << 20)
    srv = mg.Server(hbm_budget=budget, max_slots=1, max_queue=16)
    outs, tickets = [], []
    for q in range(4):
        d, U, S, Si = (da, Ua, Sa, Sia) if q % 2 == 0 else (db, Ub, Sb, Sib)
        f = fields(U.shape)
        tickets.append(srv.submit_cfc(d, dev(U), dev(S), [dev(x) for x in Si], *f))
        outs.append(f)
    res = [srv.wait(t) for t in tickets]
    srv.close()
    assert all(r["status"] == "ok" for r in res)
    assert torch.equal(outs[0][0], outs[2][0]) and torch.equal(outs[1][0], outs[3][0])


def test_uneven_2d_batch_identical_alone_and_batched(mg):
    """A batch of uneven 2D static stars (spherical and cylindrical grids of
    different sizes, mixed precision) through the worker slots: every result
    is bitwise the one of its own solve."""
    batch = inputs.batch_static_stars_2d(count=10, seed=5)
    descs = [mg.grid_desc(g, n, lo, hi, precision="mixed", tol=1e-10, max_cycles=800, accel_depth=8,
                          stall_window=0) for (g, n, lo, hi, _, _, _) in batch]
    data = [(dev(U), dev(S), [dev(x) for x in Si]) for (_, _, _, _, U, S, Si) in batch]
    alone = []
    for d, (U, S, Si) in zip(descs, data):
        h = mg.Hierarchy(d)
        f = fields(U.shape)
        rep = mg.mg_solve_cfc(h, U, S, Si, *f)
        h.close()
        assert rep["psi"]["cycles"] > 0
        alone.append([f[0], f[1]] + f[2] + f[3])
    srv = mg.Server(hbm_budget=8 << 30, max_slots=4, max_queue=64)
    outs, tickets = [], []
    for d, (U, S, Si) in zip(descs, data):
        f = fields(U.shape)
        tickets.append(srv.submit_cfc(d, U, S, Si, *f))
        outs.append([f[0], f[1]] + f[2] + f[3])
    res = [srv.wait(t) for t in tickets]
    srv.close()
    assert all(r["status"] == "ok" for r in res)
    for q, (a, b) in enumerate(zip(outs, alone)):
        for x, y in zip(a, b):
            assert torch.equal(x, y), q


def test_resident_solutions_are_evicted_before_waiting(mg):
    """A budget of the largest hierarchy plus half a resident solution.  Two
    warm-started streams leave their solutions resident; a third grid then
    fits only once those are evicted (their streams have nothing in flight).
    Every request completes within the host timeout, and the third result
    equals its direct solve."""
    a_args, Ua, Sa, Sia = cfc_case("sph2d", 31)
    b_args, Ub, Sb, Sib = cfc_case("cyl2d", 32)
    c_args, Uc, Sc, Sic = cfc_case("sph3d", 33)
    da, db, dc = desc_of(mg, a_args), desc_of(mg, b_args), desc_of(mg, c_args)
    need = [mg.mg_hierarchy_bytes(d) for d in (da, db, dc)]
    warm_a = 8 * 8 * Ua.size
    assert need[2] == max(need)
    srv = mg.Server(hbm_budget=need[2] + warm_a // 2, max_slots=1, max_queue=8)
    outs, tickets = [], []
    for d, U, S, Si, sid in [(da, Ua, Sa, Sia, 1), (db, Ub, Sb, Sib, 2), (dc, Uc, Sc, Sic, 0),
                             (da, Ua, Sa, Sia, 1)]:
        f = fields(U.shape)
        tickets.append(srv.submit_cfc(d, dev(U), dev(S), [dev(x) for x in Si], *f, stream_id=sid))
        outs.append(f)
    res = [srv.wait(t, timeout_s=120.0) for t in tickets]
    srv.close()
    assert all(r["status"] == "ok" for r in res)
    assert not res[3]["warm_started"]  # stream 1's solution made room for the third grid
    h = mg.Hierarchy(dc)
    f = fields(Uc.shape)
    mg.mg_solve_cfc(h, dev(Uc), dev(Sc), [dev(x) for x in Sic], *f)
    h.close()
    for x, y in zip([outs[2][0], outs[2][1]] + outs[2][2] + outs[2][3], [f[0], f[1]] + f[2] + f[3]):
        assert torch.equal(x, y)



def test_requests_with_wrong_shapes_are_refused(mg):
    """The server reads and writes a request's arrays through raw device
    pointers: the binding refuses arrays whose shape differs from the grid's
    before anything is queued."""
    args, U, S, Si = cfc_case("sph2d", 51)
    d = desc_of(mg, args)
    srv = mg.Server(hbm_budget=1 << 30, max_slots=1, max_queue=4)
    small = fields((16, 32))
    with pytest.raises(ValueError):
        srv.submit_cfc(d, dev(U), dev(S), [dev(x) for x in Si], *small)
    with pytest.raises(ValueError):
        srv.submit_divb(mg.grid_desc("cart", [16] * 3, [-1.0] * 3, [1.0] * 3),
                        [torch.zeros((8, 16, 16), dtype=torch.float64, device="cuda")] * 3)
    srv.close()


def _amr_case(n=(32, 16, 16), seed=61):
    """A static star on a 3D spherical grid refined for r < r_max / 4 (the
    serving workload's two-level AMR): base and patch U~ at their own cell
    centres."""
    rng = np.random.default_rng(seed)
    rho_c, R = rng.uniform(8e-4, 1.6e-3), rng.uniform(8.0, 12.0)
    a, b = [0, 0, 0], [n[0] // 4, n[1], n[2]]
    U = inputs.static_polytrope_sph3d(n, 100.0, rho_c, R)
    Up = inputs.static_polytrope_sph3d((2 * b[0], 2 * n[1], 2 * n[2]), 100.0 / 4, rho_c, R)
    return a, b, U, Up


def test_amr_requests_identical_alone_and_in_the_mix(mg):
    """Composite-grid requests (eq. psi, patch r < r_max / 4) served beside
    xCFC requests give bitwise the result of the direct composite solve."""
    n = (32, 16, 16)
    a, b, U, Up = _amr_case(n)
    desc = mg.grid_desc("sph", list(n), hi=[100.0, PI, 2 * PI], tol=1e-10, max_cycles=600, accel_depth=8,
                        stall_window=0)
    z, zp = np.zeros_like(U), np.zeros_like(Up)
    h = mg.Hierarchy(desc)
    u0, up0 = dev(z), dev(zp)
    rep = mg.mg_solve_scalar_amr(h, a, b, "psi", "robin", u0, up0, U=dev(U), A2=dev(z), Up=dev(Up), A2p=dev(zp))
    h.close()
    assert rep["status"] == "ok" and rep["cycles"] > 0
    srv = mg.Server(hbm_budget=8 << 30, max_slots=4, max_queue=64)
    outs, tickets = [], []
    for q in range(6):
        if q % 2 == 0:
            u, up = dev(z), dev(zp)
            tickets.append(srv.submit_amr(desc, a, b, dev(U), dev(z), dev(Up), dev(zp), u, up))
            outs.append((u, up))
        else:
            args, Uc, Sc, Sic = cfc_case("sph3d", 70 + q)
            tickets.append(srv.submit_cfc(desc_of(mg, args), dev(Uc), dev(Sc), [dev(x) for x in Sic],
                                          *fields(Uc.shape)))
            outs.append(None)
    res = [srv.wait(t) for t in tickets]
    srv.close()
    assert all(r["status"] == "ok" for r in res)
    for q, o_ in enumerate(outs):
        if o_ is None:
            continue
        assert res[q]["cfc"]["psi"]["cycles"] == rep["cycles"]
        assert torch.equal(o_[0], u0) and torch.equal(o_[1], up0)
