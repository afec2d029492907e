"""Two-level composite grid (block AMR of ratio 2) on the GPU against the
oracle: the composite operator (coarse-fine ghosts, flux matching at the
interface) element by element, and composite FAS solves (fields within
1e-9, cycle counts within one) in Cartesian, cylindrical and spherical
geometry, through the C ABI."""
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
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


GRIDS = {
    "cart2d": ("cart", [32, 16], [-1.0, -0.5], [1.0, 0.5], [8, 4], [24, 12]),
    "cart3d": ("cart", [16, 16, 16], [-1.0] * 3, [1.0] * 3, [4, 4, 8], [12, 12, 16]),
    "cyl2d": ("cyl", [32, 32], [0.0, -1.0], [2.0, 1.0], [0, 8], [8, 24]),
    "cyl3d": ("cyl", [16, 16, 8], [0.0, -1.0, 0.0], [2.0, 1.0, 2 * PI], [0, 4, 0], [8, 12, 8]),
    "sph2d": ("sph", [32, 16], [0.0, 0.0], [3.0, PI], [0, 0], [8, 16]),
    "sph3d": ("sph", [16, 8, 8], [0.0, 0.0, 0.0], [3.0, PI, 2 * PI], [0, 0, 0], [4, 8, 8]),
}


@pytest.mark.parametrize("kind,bc", [("lin", "robin"), ("lin", "neumann"), ("psi", "robin"), ("lin", "dirichlet")])
@pytest.mark.parametrize("grid", list(GRIDS))
def test_composite_operator_parity(mg, grid, kind, bc):
    geom, n, lo, hi, a, b = GRIDS[grid]
    d = o.desc(geom, n, lo, hi)
    rng = np.random.default_rng(17)
    shp, pshp = o.shape(d), o.patch_shape(d, a, b)
    u = rng.uniform(-0.3, 0.3, shp)
    up = rng.uniform(-0.3, 0.3, pshp)
    kw = {}
    if kind == "psi":
        kw = dict(U=rng.uniform(0, 0.01, shp), A2=rng.uniform(0, 0.01, shp), Up=rng.uniform(0, 0.01, pshp),
                  A2p=rng.uniform(0, 0.01, pshp))
    else:
        kw = dict(c=rng.uniform(0.1, 0.5, shp), cp=rng.uniform(0.1, 0.5, pshp))
    want, wantp = o.apply_amr(d, a, b, kind, bc, u, up, **kw)
    h = mg.Hierarchy(mg.grid_desc(geom, n, lo, hi))
    out = torch.zeros(shp, dtype=torch.float64, device="cuda")
    outp = torch.zeros(pshp, dtype=torch.float64, device="cuda")
    mg.mg_apply_amr(h, a, b, kind, bc, dev(u), dev(up), out, outp, **{k: dev(v) for k, v in kw.items()})
    h.close()
    scale = max(np.abs(want).max(), np.abs(wantp).max())
    assert np.abs(host(out) - want).max() <= 1e-12 * scale
    assert np.abs(host(outp) - wantp).max() <= 1e-12 * scale


def _polytrope(n, a, b, geom, lo, hi, rho_c=1.28e-3, R=1.0):
    """U of a static n = 1 polytrope of radius R at the cell centres of the
    base grid and of the patch (spherical grids)."""
    def at(nn, llo, hhi):
        r = llo[0] + (np.arange(nn[0]) + 0.5) * (hhi[0] - llo[0]) / nn[0]
        x = PI * r / R
        rho = np.where(r < R, rho_c * np.sin(x) / x, 0.0)
        shape = tuple(reversed(nn))
        return np.ascontiguousarray(np.broadcast_to(rho + 100.0 * rho ** 2, shape))
    hh = [(hi[k] - lo[k]) / n[k] for k in range(len(n))]
    pn = [2 * (b[k] - a[k]) for k in range(len(n))]
    plo = [lo[k] + a[k] * hh[k] for k in range(len(n))]
    phi = [lo[k] + b[k] * hh[k] for k in range(len(n))]
    return at(n, lo, hi), at(pn, plo, phi)


@pytest.mark.parametrize("case", ["cart2d_lin", "cart3d_lin", "cyl2d_lin", "cyl3d_lin", "sph2d_psi", "sph3d_psi",
                                  "sph2d_psi_64"])
def test_composite_solve_parity(mg, case):
    """Composite FAS solves: every field within 1e-9 of the oracle, cycles
    within one (Anderson depth 8 on curvilinear grids, plain V-cycles on
    Cartesian ones)."""
    grid, kind = case.rsplit("_", 1)[0], case.split("_")[1]
    if case == "sph2d_psi_64":
        geom, n, lo, hi, a, b = "sph", [64, 32], [0.0, 0.0], [100.0, PI], [0, 0], [16, 32]
    else:
        geom, n, lo, hi, a, b = GRIDS[grid]
    accel = 0 if geom == "cart" else 8
    d = o.desc(geom, n, lo, hi, tol=1e-10, max_cycles=500, accel_depth=accel, stall_window=0)
    gd = mg.grid_desc(geom, n, lo, hi, tol=1e-10, max_cycles=500, accel_depth=accel, stall_window=0)
    shp, pshp = o.shape(d), o.patch_shape(d, a, b)
    rng = np.random.default_rng(23)
    if kind == "psi":
        R = 10.0 if case == "sph2d_psi_64" else 0.6
        U, Up = _polytrope(n, a, b, geom, lo, hi, R=R, rho_c=1.28e-3 if R > 1 else 0.05)
        kw = dict(U=U, A2=np.zeros(shp), Up=Up, A2p=np.zeros(pshp))
    else:
        kw = dict(c=rng.uniform(0.1, 0.5, shp), cp=rng.uniform(0.1, 0.5, pshp), f=rng.standard_normal(shp),
                  fp=rng.standard_normal(pshp))
    bc = "dirichlet" if geom == "cart" and kind == "lin" else "robin"
    u, up = np.zeros(shp), np.zeros(pshp)
    ro = o.solve_scalar_amr(d, a, b, kind, bc, u, up, **kw)
    assert ro["status"] == "ok"
    h = mg.Hierarchy(gd)
    ut = torch.zeros(shp, dtype=torch.float64, device="cuda")
    upt = torch.zeros(pshp, dtype=torch.float64, device="cuda")
    rg = mg.mg_solve_scalar_amr(h, a, b, kind, bc, ut, upt, **{k: dev(v) for k, v in kw.items()})
    h.close()
    assert rg["status"] == "ok" and rg["rel"] <= 1e-10
    assert abs(rg["cycles"] - ro["cycles"]) <= 1, (rg["cycles"], ro["cycles"])
    scale = max(np.abs(u).max(), np.abs(up).max())
    assert np.abs(host(upt) - up).max() <= 1e-9 * scale
    assert np.abs(host(ut) - u).max() <= 1e-9 * scale


def test_composite_box_rules(mg):
    """Boxes the composite grid rejects with MG_ERR_INVALID: outside the
    grid, patch sizes not powers of two, a spherical patch short of theta."""
    h = mg.Hierarchy(mg.grid_desc("sph", [32, 16], [0.0, 0.0], [3.0, PI]))
    shp = (16, 32)
    u = torch.zeros(shp, dtype=torch.float64, device="cuda")
    z = torch.zeros(shp, dtype=torch.float64, device="cuda")
    for a, b in (([0, 0], [40, 16]), ([0, 0], [6, 16]), ([0, 0], [8, 8])):
        up = torch.zeros(tuple(2 * (b[k] - a[k]) for k in (1, 0)), dtype=torch.float64, device="cuda")
        st = mg.lib().mg_solve_scalar_amr(h.handle, mg.C.byref(mg._box3(a)), mg.C.byref(mg._box3(b)), mg.MG_EQ_PSI,
                                          mg.MG_BC_ROBIN, z.data_ptr(), z.data_ptr(), None, None, up.data_ptr(),
                                          up.data_ptr(), None, None, u.data_ptr(), up.data_ptr(), None)
        assert st == mg.MG_ERR_INVALID, (a, b)
    h.close()
