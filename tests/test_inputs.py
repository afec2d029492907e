"""The seeded synthetic inputs follow the stated recipe (CPU).

The sources stand in for the paper's XNS stars and the benchmark's magnetic
field; both the oracle and the CUDA path receive exactly these arrays, so
their structure is checked here: support and shape of the stars, rotation,
axisymmetry, determinism of the seeds and the noise level of the field."""
import numpy as np

from paper_2012_07322_gb300 import inputs

PI = np.pi


def test_static_star_profile():
    n_r, n_t, r_max = 64, 32, 100.0
    U = inputs.static_polytrope_sph2d(n_r, n_t, r_max)
    assert U.shape == (n_t, n_r)
    r = (np.arange(n_r) + 0.5) * r_max / n_r
    # spherical, positive inside R = 10, zero outside
    assert np.all(U == U[0:1, :])
    assert np.all(U[:, r < 10.0] > 0) and np.all(U[:, r >= 10.0] == 0)
    # U = rho + K rho^2 with rho = rho_c sinc(pi r / R): the first cell
    rho0 = 1.28e-3 * np.sin(PI * r[0] / 10.0) / (PI * r[0] / 10.0)
    assert abs(U[0, 0] - (rho0 + 100.0 * rho0 ** 2)) <= 1e-15 * U[0, 0]
    assert np.all(np.diff(U[0, r < 10.0]) < 0)  # monotone density


def test_rotating_star_structure():
    n, r_max = (64, 32, 16), 100.0
    U, S, Si = inputs.rotating_polytrope_sph3d(n, r_max)
    assert U.shape == S.shape == (n[2], n[1], n[0])
    # axisymmetric, only the phi component of the momentum, prograde
    for a in (U, S, Si[2]):
        assert np.all(a == a[0:1])
    assert np.all(Si[0] == 0) and np.all(Si[1] == 0) and np.all(Si[2] >= 0)
    assert np.all(U >= 0) and np.all(S >= 0)
    # oblate support: xi = sqrt((varpi / 10)^2 + (z / 8)^2) < 1
    r = (np.arange(n[0]) + 0.5) * r_max / n[0]
    th = (np.arange(n[1]) + 0.5) * PI / n[1]
    varpi = r[None, :] * np.sin(th)[:, None]
    z = r[None, :] * np.cos(th)[:, None]
    inside = (varpi / 10.0) ** 2 + (z / 8.0) ** 2 < 1.0
    assert np.all(U[0][inside] > 0) and np.all(U[0][~inside] == 0)
    assert np.all(Si[2][0][inside] > 0) and np.all(Si[2][0][~inside] == 0)
    # the 2D star is a meridional plane of the 3D one
    U2, S2, Si2 = inputs.rotating_polytrope_sph2d(n[0], n[1], r_max)
    assert np.array_equal(U2, U[0]) and np.array_equal(Si2[2], Si[2][0])


def test_magnetic_field_seeds_and_noise():
    n = 32
    B1 = inputs.divb_field(n=n)
    B1b = inputs.divb_field(n=n)
    assert all(np.array_equal(a, b) for a, b in zip(B1, B1b))
    assert all(b.shape == (n, n, n) for b in B1)
    # another noise seed changes the field by the stated 1e-3 B_rms per
    # component and cell (the difference of two draws has rms sqrt(2) of it)
    B2 = inputs.divb_field(n=n, seed_noise=2)
    brms = np.sqrt(np.mean(sum(b * b for b in B1)) / 3.0)
    drms = np.sqrt(np.mean(sum((a - b) ** 2 for a, b in zip(B1, B2))) / 3.0)
    assert 0.9 * np.sqrt(2) * 1e-3 < drms / brms < 1.1 * np.sqrt(2) * 1e-3
    # another mode seed gives another field
    B3 = inputs.divb_field(n=n, seed_modes=5)
    assert np.abs(B3[0] - B1[0]).max() > 0.1 * np.abs(B1[0]).max()


def test_cartesian_rotating_star_symmetries():
    """The Cartesian rotating star: U and S even in x, y and z, the momentum
    omega (-y, x, 0) a rigid rotation about z (S_x odd in y and even in x,
    S_y the reverse, S_z = 0), and the same U as the spherical generator at
    the centre."""
    U, S, Si = inputs.rotating_polytrope_cart3d((16, 16, 16), 30.0)
    for A in (U, S):
        for ax in range(3):
            assert np.allclose(A, np.flip(A, axis=ax))
    assert np.allclose(Si[0], -np.flip(Si[0], axis=1)) and np.allclose(Si[0], np.flip(Si[0], axis=2))
    assert np.allclose(Si[1], -np.flip(Si[1], axis=2)) and np.allclose(Si[1], np.flip(Si[1], axis=1))
    assert (Si[2] == 0).all() and np.abs(Si[0]).max() > 0
    Us, _, _ = inputs.rotating_polytrope_sph3d((64, 32, 4), 100.0)
    assert U.max() <= Us.max() * (1 + 1e-12)
