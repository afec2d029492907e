"""Seeded synthetic inputs for the solver and for its CPU oracle.

This module only samples source fields on the cell centres of a grid; it
holds none of the solver's arithmetic.  The paper's own sources (rotating
neutron stars from XNS initial data, Sec. 3.3.2) are not available, so
analytic Gamma = 2 polytropes stand in for them (G = c = M_sun = 1):

    rho(xi) = rho_c sin(pi xi) / (pi xi) for xi < 1, else 0,
    p = K rho^2 (K = 100), eps = K rho, h = 1 + eps + p / rho = 1 + 2 K rho.

Arrays are float64 numpy arrays, dimension 0 fastest: shape (n1, n0) in 2D,
(n2, n1, n0) in 3D.
"""
from __future__ import annotations

import numpy as np

K_POLY = 100.0


def cell_centres(n, lo, hi):
    """1D cell-centre coordinates per dimension."""
    return [lo[d] + (np.arange(n[d]) + 0.5) * (hi[d] - lo[d]) / n[d] for d in range(len(n))]


def _lane_emden_n1(xi, rho_c):
    rho = np.zeros_like(xi)
    m = xi < 1.0
    x = np.pi * xi[m]
    rho[m] = rho_c * np.where(x > 0, np.sin(x) / np.where(x > 0, x, 1.0), 1.0)
    return rho


def static_polytrope_sph2d(n_r=64, n_theta=32, r_max=100.0, rho_c=1.28e-3, R=10.0):
    """Static star on a 2D axisymmetric spherical grid (r, theta in [0, pi]).

    Returns U~ = rho (1 + eps) = rho + K rho^2 (W = 1), the conformal energy
    density of the psi equation."""
    r, th = cell_centres([n_r, n_theta], [0.0, 0.0], [r_max, np.pi])
    rr = np.broadcast_to(r[None, :], (n_theta, n_r))
    rho = _lane_emden_n1(rr / R, rho_c)
    return np.ascontiguousarray(rho + K_POLY * rho * rho)


def static_polytrope_sph3d(n=(64, 32, 32), r_max=100.0, rho_c=1.28e-3, R=10.0):
    """The static star of :func:`static_polytrope_sph2d` on a 3D spherical
    grid (r in [0, r_max], theta in [0, pi], phi in [0, 2 pi)): U~ = rho +
    K rho^2, K = 100, shaped (n_phi, n_theta, n_r).  A patch refined over
    r < r_max' is the same star on the grid of r_max' with its own cells."""
    U2 = static_polytrope_sph2d(n[0], n[1], r_max, rho_c, R)
    return np.ascontiguousarray(np.broadcast_to(U2[None, :, :], (n[2], n[1], n[0])))


def rotating_polytrope_sph3d(n=(128, 64, 64), r_max=100.0, rho_c=1.28e-3, R=10.0, axis_ratio=0.8,
                             omega=0.02):
    """Uniformly rotating oblate polytrope on a 3D spherical grid.

    xi = sqrt((varpi / R)^2 + (z / (axis_ratio R))^2), v_phi = omega varpi,
    W = (1 - v^2)^-1/2.  Returns (U~, S~, [S~_r, S~_theta, S~_phi]) with
    U~ = rho h W^2 - p, S~_phi = rho h W^2 v_phi, S~ = rho h W^2 v^2 + 3 p
    (orthonormal components)."""
    r, th, ph = cell_centres(list(n), [0.0, 0.0, 0.0], [r_max, np.pi, 2 * np.pi])
    rr = r[None, None, :]
    tt = th[None, :, None]
    varpi = rr * np.sin(tt)
    z = rr * np.cos(tt)
    xi = np.sqrt((varpi / R) ** 2 + (z / (axis_ratio * R)) ** 2)
    rho = _lane_emden_n1(xi, rho_c)
    v = omega * varpi
    W2 = 1.0 / (1.0 - v * v)
    p = K_POLY * rho * rho
    h = 1.0 + 2.0 * K_POLY * rho
    shp = (n[2], n[1], n[0])
    U = np.broadcast_to(rho * h * W2 - p, shp)
    S = np.broadcast_to(rho * h * W2 * v * v + 3.0 * p, shp)
    Sphi = np.broadcast_to(rho * h * W2 * v, shp)
    zero = np.zeros(shp)
    return (np.ascontiguousarray(U), np.ascontiguousarray(S),
            [zero.copy(), zero.copy(), np.ascontiguousarray(Sphi)])


def rotating_polytrope_sph2d(n_r=64, n_theta=32, r_max=100.0, rho_c=1.28e-3, R=10.0,
                             axis_ratio=0.8, omega=0.02):
    """The rotating star of :func:`rotating_polytrope_sph3d` on a 2D
    axisymmetric (r, theta) grid."""
    U, S, Si = rotating_polytrope_sph3d((n_r, n_theta, 2), r_max, rho_c, R, axis_ratio, omega)
    return (np.ascontiguousarray(U[0]), np.ascontiguousarray(S[0]),
            [np.ascontiguousarray(a[0]) for a in Si])


def rotating_polytrope_cyl(n, extent=100.0, rho_c=1.28e-3, R=10.0, axis_ratio=0.8, omega=0.02):
    """Rotating star on a cylindrical grid R in [0, extent], z in
    [-extent, extent] (and phi in [0, 2 pi) in 3D); components (R, z, phi)."""
    three = len(n) == 3
    lo = [0.0, -extent] + ([0.0] if three else [])
    hi = [extent, extent] + ([2 * np.pi] if three else [])
    c = cell_centres(list(n), lo, hi)
    if three:
        Rr = c[0][None, None, :]
        zz = c[1][None, :, None]
        shp = (n[2], n[1], n[0])
    else:
        Rr = c[0][None, :]
        zz = c[1][:, None]
        shp = (n[1], n[0])
    xi = np.sqrt((Rr / R) ** 2 + (zz / (axis_ratio * R)) ** 2)
    rho = _lane_emden_n1(xi, rho_c)
    v = omega * Rr
    W2 = 1.0 / (1.0 - v * v)
    p = K_POLY * rho * rho
    h = 1.0 + 2.0 * K_POLY * rho
    U = np.broadcast_to(rho * h * W2 - p, shp)
    S = np.broadcast_to(rho * h * W2 * v * v + 3.0 * p, shp)
    Sphi = np.broadcast_to(rho * h * W2 * v, shp)
    zero = np.zeros(shp)
    return (np.ascontiguousarray(U), np.ascontiguousarray(S),
            [zero.copy(), zero.copy(), np.ascontiguousarray(Sphi)])


def rotating_polytrope_cart3d(n=(32, 32, 32), extent=30.0, rho_c=1.28e-3, R=10.0, axis_ratio=0.8, omega=0.02):
    """The rotating star of :func:`rotating_polytrope_sph3d` on a 3D
    Cartesian grid [-extent, extent]^3, shaped (n_z, n_y, n_x); velocity
    omega (-y, x, 0), momentum components (x, y, z)."""
    x, y, z = cell_centres(list(n), [-extent] * 3, [extent] * 3)
    xx = x[None, None, :]
    yy = y[None, :, None]
    zz = z[:, None, None]
    varpi = np.sqrt(xx * xx + yy * yy)
    xi = np.sqrt((varpi / R) ** 2 + (zz / (axis_ratio * R)) ** 2)
    rho = _lane_emden_n1(xi, rho_c)
    v = omega * varpi
    W2 = 1.0 / (1.0 - v * v)
    p = K_POLY * rho * rho
    h = 1.0 + 2.0 * K_POLY * rho
    shp = (n[2], n[1], n[0])
    a = rho * h * W2
    U = np.broadcast_to(a - p, shp)
    S = np.broadcast_to(a * v * v + 3.0 * p, shp)
    Sx = np.broadcast_to(-a * omega * yy, shp)
    Sy = np.broadcast_to(a * omega * xx, shp)
    return (np.ascontiguousarray(U), np.ascontiguousarray(S),
            [np.ascontiguousarray(Sx), np.ascontiguousarray(Sy), np.zeros(shp)])


def divb_field(n=256, n_modes=32, k_max=8, noise=1e-3, seed_modes=0, seed_noise=1):
    """Magnetic field on the Cartesian cube [-1, 1]^3 (n^3 cells).

    A = sum_m a_m sin(pi k_m . x + phi_m), k_m integer with 0 < |k_m| <= k_max
    (uniform over that set), a_m ~ N(0, I_3), phi_m ~ U[0, 2 pi) (seed_modes);
    B = central-difference curl of A sampled on the cells and one layer
    beyond; then B += eta, eta ~ N(0, (noise * B_rms)^2) per component and
    cell (seed_noise).  Returns [Bx, By, Bz], each of shape (n, n, n)."""
    rng = np.random.default_rng(seed_modes)
    ks = np.array([(a, b, c) for a in range(-k_max, k_max + 1) for b in range(-k_max, k_max + 1)
                   for c in range(-k_max, k_max + 1) if 0 < a * a + b * b + c * c <= k_max * k_max])
    pick = ks[rng.integers(0, len(ks), size=n_modes)]
    amp = rng.standard_normal((n_modes, 3))
    phase = rng.uniform(0.0, 2 * np.pi, size=n_modes)
    hx = 2.0 / n
    x = -1.0 + (np.arange(-1, n + 1) + 0.5) * hx          # cells plus one layer
    A = np.zeros((3, n + 2, n + 2, n + 2))
    for m in range(n_modes):
        ex = np.exp(1j * np.pi * pick[m, 0] * x)
        ey = np.exp(1j * np.pi * pick[m, 1] * x)
        ez = np.exp(1j * (np.pi * pick[m, 2] * x + phase[m]))
        mode = np.imag(ez[:, None, None] * ey[None, :, None] * ex[None, None, :])
        for c in range(3):
            A[c] += amp[m, c] * mode
    inv2h = 1.0 / (2.0 * hx)
    # central differences; array axes are (z, y, x)
    def dx(F):
        return (F[1:-1, 1:-1, 2:] - F[1:-1, 1:-1, :-2]) * inv2h
    def dy(F):
        return (F[1:-1, 2:, 1:-1] - F[1:-1, :-2, 1:-1]) * inv2h
    def dz(F):
        return (F[2:, 1:-1, 1:-1] - F[:-2, 1:-1, 1:-1]) * inv2h
    B = [dy(A[2]) - dz(A[1]), dz(A[0]) - dx(A[2]), dx(A[1]) - dy(A[0])]
    brms = np.sqrt(np.mean(B[0] ** 2 + B[1] ** 2 + B[2] ** 2) / 3.0)
    rng2 = np.random.default_rng(seed_noise)
    return [np.ascontiguousarray(b + rng2.standard_normal(b.shape) * noise * brms) for b in B]


def random_field(shape, seed, scale=1.0):
    """I.i.d. uniform [-scale, scale) values (operator-level parity tests)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=shape)


def batch_static_stars_2d(count=512, seed=2, axis_ratio=1.0, omega=0.0):
    """Uneven batch of 2D axisymmetric stars, static by default (Omega = 0,
    spherical n = 1 polytropes): half on spherical grids N_r in {32..256} x
    N_theta in {16..128} (r <= 100), half on cylindrical grids N_R in
    {32..256} x N_z in {64..512} (R <= 100, |z| <= 100); rho_c ~ U[5e-4,
    2e-3], R ~ U[8, 14].  With omega != 0 the same grids and draws carry
    uniformly rotating stars of the given axis ratio (momentum sources S_i).
    Returns (geom, n, lo, hi, U, S, Si) tuples."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        rho_c, R = rng.uniform(5e-4, 2e-3), rng.uniform(8.0, 14.0)
        if q % 2 == 0:
            n = [int(rng.choice([32, 64, 128, 256])), int(rng.choice([16, 32, 64, 128]))]
            U, S, Si = rotating_polytrope_sph2d(n[0], n[1], 100.0, rho_c, R, axis_ratio=axis_ratio, omega=omega)
            out.append(("sph", n, [0.0, 0.0], [100.0, np.pi], U, S, Si))
        else:
            n = [int(rng.choice([32, 64, 128, 256])), int(rng.choice([64, 128, 256, 512]))]
            U, S, Si = rotating_polytrope_cyl(n, 100.0, rho_c, R, axis_ratio=axis_ratio, omega=omega)
            out.append(("cyl", n, [0.0, -100.0], [100.0, 100.0], U, S, Si))
    return out
