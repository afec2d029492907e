"""Pins of the oracle's two-level composite grid (block AMR of ratio 2).

The composite operator and its FAS iteration are readings (the paper's
multigrid on block-AMR grids lives in the library it cites); these tests tie
them to facts fixed by the discretisation and the mathematics: exact
conservation of the composite operator (the fine fluxes through the
coarse-fine interface are the coarse cell's), second-order convergence on
closed-form solutions, the multigrid fixed point against a direct sparse
solve of the same composite equations, and the reduction to the uniform fine
grid when the patch covers the whole domain."""
import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.linalg

import oracle.oracle as o

PI = np.pi

# (name, geom, n, lo, hi, patch a, patch b)
GRIDS = [
    ("cart2d", "cart", [16, 8], [-1.0, -0.5], [1.0, 0.5], [4, 2], [12, 6]),
    ("cart3d", "cart", [8, 8, 8], [-1.0] * 3, [1.0] * 3, [2, 2, 4], [6, 4, 8]),
    ("cyl2d", "cyl", [16, 16], [0.0, -1.0], [2.0, 1.0], [0, 4], [4, 12]),
    ("cyl3d", "cyl", [8, 8, 4], [0.0, -1.0, 0.0], [2.0, 1.0, 2 * PI], [0, 2, 0], [4, 6, 4]),
    ("sph2d", "sph", [16, 8], [0.0, 0.0], [3.0, PI], [0, 0], [4, 8]),
    ("sph3d", "sph", [8, 8, 4], [0.0, 0.0, 0.0], [3.0, PI, 2 * PI], [0, 0, 0], [2, 8, 4]),
]
IDS = [g[0] for g in GRIDS]


def _centres(n, lo, hi):
    return [lo[k] + (np.arange(n[k]) + 0.5) * (hi[k] - lo[k]) / n[k] for k in range(len(n))]


def _pseudo_volume(geom, n, lo, hi):
    """Cell measure of the printed operators' flux form: prod h times 1, R or
    r^2 sin(theta) at the cell centre; numpy shape (.., n1, n0)."""
    c = _centres(n, lo, hi)
    h = np.prod([(hi[k] - lo[k]) / n[k] for k in range(len(n))])
    w = np.ones(tuple(reversed(n)))
    if geom == "cyl":
        w = w * c[0]
    if geom == "sph":
        w = w * (c[0] ** 2) * np.sin(c[1])[:, None]
    return h * w


def _patch_desc(n, lo, hi, a, b):
    h = [(hi[k] - lo[k]) / n[k] for k in range(len(n))]
    return [2 * (b[k] - a[k]) for k in range(len(n))], [lo[k] + a[k] * h[k] for k in range(len(n))], \
        [lo[k] + b[k] * h[k] for k in range(len(n))]


def _covered(n, a, b):
    m = np.zeros(tuple(reversed(n)), bool)
    m[tuple(slice(a[k], b[k]) for k in reversed(range(len(n))))] = True
    return m


@pytest.mark.parametrize("grid", GRIDS, ids=IDS)
def test_composite_operator_is_conservative(grid):
    """With Neumann outer ghosts (zero flux through the domain boundary;
    the origin, axis and pole faces have zero area, phi is periodic) the
    composite Laplacian summed with the cell measures vanishes for ANY field:
    every interior face flux cancels, including the coarse-fine faces where
    the coarse cell takes the sum of the fine fluxes.  Replacing the fine
    fluxes by the coarse one would leave O(1)."""
    name, geom, n, lo, hi, a, b = grid
    d = o.desc(geom, n, lo, hi)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(o.shape(d))
    up = rng.standard_normal(o.patch_shape(d, a, b))
    out, outp = o.apply_amr(d, a, b, "lin", "neumann", u, up)
    pn, plo, phi = _patch_desc(n, lo, hi, a, b)
    vb = _pseudo_volume(geom, n, lo, hi)
    vp = _pseudo_volume(geom, pn, plo, phi)
    cov = _covered(n, a, b)
    assert np.all(out[cov] == 0.0)
    total = (vb * out).sum() + (vp * outp).sum()
    scale = np.abs(vb * out).sum() + np.abs(vp * outp).sum()
    assert abs(total) < 1e-12 * scale, (total, scale)


def _solve_amr_mms(n, with_patch=True):
    """Dirichlet Poisson on the unit square, u* = sin(pi x) sin(pi y), with a
    centred patch over base cells n/4 .. 3n/4."""
    d = o.desc("cart", [n, n], [0, 0], [1, 1], tol=1e-12, max_cycles=300)
    a, b = [n // 4, n // 4], [3 * n // 4, 3 * n // 4]
    x = (np.arange(n) + 0.5) / n
    us = np.sin(PI * x)[None, :] * np.sin(PI * x)[:, None]
    xp = (a[0] + (np.arange(2 * (b[0] - a[0])) + 0.5) / 2) / n
    ups = np.sin(PI * xp)[None, :] * np.sin(PI * xp)[:, None]
    u, up = np.zeros_like(us), np.zeros_like(ups)
    rep = o.solve_scalar_amr(d, a, b, "lin", "dirichlet", u, up, f=-2 * PI ** 2 * us, fp=-2 * PI ** 2 * ups)
    assert rep["status"] == "ok"
    cov = _covered([n, n], a, b)
    return np.abs(u - us)[~cov].max(), np.abs(up - ups).max()


def test_composite_poisson_converges_at_second_order():
    """Closed-form Dirichlet Poisson problem: the composite solution's error
    falls by ~4 per refinement on the uncovered base cells and on the patch
    (the O(h) truncation error at the interface cells does not spoil the
    second order of the solution), and the patch lowers the error of the
    uniform base grid."""
    eb, ep = zip(*[_solve_amr_mms(n) for n in (16, 32, 64)])
    for e in (eb, ep):
        rates = [np.log2(e[i] / e[i + 1]) for i in range(2)]
        assert min(rates) > 1.85, (e, rates)
    d = o.desc("cart", [64, 64], [0, 0], [1, 1], tol=1e-12, max_cycles=300)
    x = (np.arange(64) + 0.5) / 64
    us = np.sin(PI * x)[None, :] * np.sin(PI * x)[:, None]
    u = np.zeros_like(us)
    o.solve_scalar(d, "lin", "dirichlet", u, f=-2 * PI ** 2 * us)
    assert max(eb[-1], ep[-1]) < 0.6 * np.abs(u - us).max()


def test_composite_polytrope_second_order():
    """The Newtonian n = 1 polytrope (lap delta = -2 pi rho, closed form
    delta = -Phi_N / 2, Robin outer condition exact for the exterior 1/r) on
    a spherical grid refined for r < r_max / 4 (the star): outside the star
    the error falls at second order on the patch and on the base cells."""
    rho_c, R, rmax = 1.28e-3, 10.0, 40.0
    k, M = PI / R, 4 * rho_c * R ** 3 / PI

    def profile(r):
        kr = k * r
        rho = np.where(r < R, rho_c * np.sin(kr) / kr, 0.0)
        phi = np.where(r < R, -(4 * rho_c * R ** 2 / PI) * (1 + np.sin(kr) / kr), -M / r)
        return rho, phi

    eb, ep = [], []
    for nr, nt in [(32, 8), (64, 16), (128, 32)]:
        d = o.desc("sph", [nr, nt], [0, 0], [rmax, PI], tol=1e-11, max_cycles=400, accel_depth=8, stall_window=0)
        a, b = [0, 0], [nr // 4, nt]
        r = (np.arange(nr) + 0.5) * rmax / nr
        rp = (np.arange(2 * b[0]) + 0.5) * rmax / nr / 2
        rho, phi = profile(r)
        rhop, phip = profile(rp)
        f = np.ascontiguousarray(np.broadcast_to(-2 * PI * rho, (nt, nr)))
        fp = np.ascontiguousarray(np.broadcast_to(-2 * PI * rhop, (2 * nt, 2 * b[0])))
        u, up = np.zeros((nt, nr)), np.zeros((2 * nt, 2 * b[0]))
        rep = o.solve_scalar_amr(d, a, b, "lin", "robin", u, up, f=f, fp=fp)
        assert rep["status"] == "ok", rep["status"]
        eb.append(np.abs(u - (-phi / 2)[None, :])[:, b[0]:].max())
        ep.append(np.abs(up - (-phip / 2)[None, :])[:, rp > R].max() if (rp > R).any() else 0.0)
    rates = [np.log2(eb[i] / eb[i + 1]) for i in range(2)]
    assert min(rates) > 1.9, (eb, rates)
    assert eb[-1] < 2e-5 * M


def _composite_matrix(d, a, b, kind, bc, c, cp):
    """Matrix of the composite linear operator over the composite unknowns
    (patch cells, then uncovered base cells), applied column by column."""
    nb = o.shape(d)
    pshape = o.patch_shape(d, a, b)
    cov = _covered([d.n[k] for k in range(d.ndim)], a, b)
    idx_b = np.flatnonzero(~cov.ravel())
    npatch = int(np.prod(pshape))
    N = npatch + len(idx_b)
    cols = []
    for m in range(N):
        u = np.zeros(nb)
        up = np.zeros(pshape)
        if m < npatch:
            up.flat[m] = 1.0
        else:
            u.flat[idx_b[m - npatch]] = 1.0
        out, outp = o.apply_amr(d, a, b, kind, bc, u, up, c=c, cp=cp)
        cols.append(np.concatenate([outp.ravel(), out.ravel()[idx_b]]))
    return scipy.sparse.csc_matrix(np.array(cols).T), idx_b, npatch


@pytest.mark.parametrize("grid", GRIDS, ids=IDS)
def test_composite_fixed_point_equals_direct_solve(grid):
    """lap u - c u = f on the composite grid (Robin outer condition): the
    composite FAS iteration converges to the direct sparse solution of the
    composite equations."""
    name, geom, n, lo, hi, a, b = grid
    d = o.desc(geom, n, lo, hi, tol=1e-12, max_cycles=400, accel_depth=8, stall_window=0)
    rng = np.random.default_rng(3)
    c = rng.uniform(0.1, 0.5, o.shape(d))
    cp = rng.uniform(0.1, 0.5, o.patch_shape(d, a, b))
    f = rng.standard_normal(o.shape(d))
    fp = rng.standard_normal(o.patch_shape(d, a, b))
    A, idx_b, npatch = _composite_matrix(d, a, b, "lin", "robin", c, cp)
    x = scipy.sparse.linalg.spsolve(A, np.concatenate([fp.ravel(), f.ravel()[idx_b]]))
    u, up = np.zeros(o.shape(d)), np.zeros(o.patch_shape(d, a, b))
    rep = o.solve_scalar_amr(d, a, b, "lin", "robin", u, up, c=c, f=f, cp=cp, fp=fp)
    assert rep["status"] == "ok"
    got = np.concatenate([up.ravel(), u.ravel()[idx_b]])
    np.testing.assert_allclose(got, x, rtol=0, atol=1e-9 * np.abs(x).max())


@pytest.mark.parametrize("geom,n,lo,hi", [("cart", [8, 8], [-1.0, -1.0], [1.0, 1.0]),
                                          ("sph", [8, 4], [0.0, 0.0], [3.0, PI])])
def test_full_patch_equals_uniform_fine_grid(geom, n, lo, hi):
    """A patch over the whole domain has no coarse-fine interface: the
    composite solution on it is the solution of the uniform fine grid (eq.
    psi with a source), the base hierarchy serving only as coarse grids."""
    nd = len(n)
    d = o.desc(geom, n, lo, hi, tol=1e-12, max_cycles=400, accel_depth=8, stall_window=0)
    a, b = [0] * nd, list(n)
    nf = [2 * x for x in n]
    df = o.desc(geom, nf, lo, hi, tol=1e-12, max_cycles=400, accel_depth=8, stall_window=0)
    rng = np.random.default_rng(4)
    Up = rng.uniform(0, 0.05, o.shape(df))
    A2p = rng.uniform(0, 0.01, o.shape(df))
    U = np.zeros(o.shape(d))
    A2 = np.zeros(o.shape(d))
    u, up = np.zeros(o.shape(d)), np.zeros(o.shape(df))
    rep = o.solve_scalar_amr(d, a, b, "psi", "robin", u, up, U=U, A2=A2, Up=Up, A2p=A2p)
    assert rep["status"] == "ok"
    uf = np.zeros(o.shape(df))
    ru = o.solve_scalar(df, "psi", "robin", uf, U=Up, A2=A2p)
    assert ru["status"] == "ok"
    np.testing.assert_allclose(up, uf, rtol=0, atol=1e-10 * np.abs(uf).max())


@pytest.mark.parametrize("nd", [2, 3])
def test_composite_operator_exact_on_quadratics(nd):
    """The coarse-fine ghosts are quadratic in both directions (the reading
    of the interface): for a quadratic field sampled at every cell centre the
    ghosts equal the field at their own centres, so the composite Laplacian is
    the exact Laplacian (2 sum of the squared coefficients' diagonal) on every
    composite cell whose stencil stays away from the domain boundary, the
    interface cells of both levels included.  Linear interpolation in either
    direction would leave O(1) there."""
    n = [8] * nd
    lo, hi = [-1.0] * nd, [1.0] * nd
    a, b = [2] * nd, [6] * nd
    if nd == 3:
        a[2], b[2] = 3, 5
    d = o.desc("cart", n, lo, hi)
    coef = np.array([[1.0, 0.3, -0.2], [0.3, -0.7, 0.5], [-0.2, 0.5, 0.4]])[:nd, :nd]
    lin = np.array([0.2, -0.1, 0.3])[:nd]

    def q(centres):
        X = np.meshgrid(*reversed(centres), indexing="ij")[::-1]  # X[k] varies along dim k
        return sum(coef[i, j] * X[i] * X[j] for i in range(nd) for j in range(nd)) + sum(
            lin[i] * X[i] for i in range(nd)) + 1.0

    pn, plo, phi = _patch_desc(n, lo, hi, a, b)
    u = q(_centres(n, lo, hi))
    up = q(_centres(pn, plo, phi))
    out, outp = o.apply_amr(d, a, b, "lin", "dirichlet", u, up)
    exact = 2.0 * np.trace(coef)
    cov = _covered(n, a, b)
    inner = np.zeros_like(cov)
    inner[(slice(1, -1),) * nd] = True
    np.testing.assert_allclose(out[inner & ~cov], exact, rtol=0, atol=1e-11)
    np.testing.assert_allclose(outp, exact, rtol=0, atol=1e-11)
