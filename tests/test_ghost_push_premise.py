"""The premise of the vector smoother's ghost push, checked on the oracle's
own ghost rules (CPU).

A colour pass of vector component c may write the ghosts of the cells it
updates at its end, instead of a ghost fill after it, only if (1) every
ghost of c under the Dirichlet-0 rule is plus or minus one interior cell, and
(2) no cell of the same pass reads such a ghost before it is written unless
the cell shares a block with the ghost's source.  A component's own stencil
reads only face neighbours, and these have the other colour except across
the poles (and the cylinder axis), where the ghost copies the cell n_phi / 2
planes away; the pass pairs planes k and k + n_phi / 2 in one block.  Here
both facts are checked for every ghost, on grids of every geometry, with the
oracle's fill rules (which share nothing with the CUDA library).  With
n_phi / 2 odd (n_phi = 2) the origin ghosts copy same-colour cells mirrored
in theta, which no pairing of planes covers: the host then keeps the fill
launch unless the whole level is one block, and the last check below shows
that case."""
import numpy as np
import pytest

import oracle.oracle as o

PI = np.pi


@pytest.mark.parametrize("geom,n,lo,hi", [
    ("sph", [8, 8, 8], [0, 0, 0], [30.0, PI, 2 * PI]),
    ("sph", [16, 8, 4], [0, 0, 0], [30.0, PI, 2 * PI]),
    ("sph", [16, 8], [0, 0], [30.0, PI]),
    ("cyl", [8, 8, 8], [0, -30, 0], [30.0, 30.0, 2 * PI]),
    ("cyl", [8, 16], [0, -30], [30.0, 30.0]),
    ("cart", [8, 4, 8], [-1, -1, -1], [1, 1, 1]),
    ("cart", [8, 8], [-1, -1], [1, 1]),
])
def test_vector_ghosts_are_signed_copies_read_safely(geom, n, lo, hi):
    d = o.desc(geom, n, lo, hi)
    nd = len(n)
    shp = o.shape(d)                      # interior shape, slowest dimension first
    gshp = o.shape(d, True)
    nk = n[2] if nd == 3 else 1
    cells = int(np.prod(shp))
    for comp in range(3):
        g = np.zeros(gshp)
        inner = (slice(1, -1),) * nd
        g[inner] = (np.arange(cells) + 1.0).reshape(shp)
        o.fill_ghosts(d, "dirichlet", comp, g)
        val = g
        # coordinates (i, j, k) of every ghosted slot, dimension 0 = i fastest
        if nd == 3:
            K, J, I = np.meshgrid(np.arange(-1, nk + 1), np.arange(-1, n[1] + 1), np.arange(-1, n[0] + 1),
                                  indexing="ij")
        else:
            J, I = np.meshgrid(np.arange(-1, n[1] + 1), np.arange(-1, n[0] + 1), indexing="ij")
            K = np.zeros_like(I)
        interior = (I >= 0) & (I < n[0]) & (J >= 0) & (J < n[1]) & (K >= 0) & (K < nk)
        ghost = ~interior
        if nd == 3:
            ghost &= ~(((I < 0) | (I >= n[0])) & ((J < 0) | (J >= n[1])) & ((K < 0) | (K >= nk)))  # corners unused
        # (1) every ghost is +- one interior cell
        v = val[ghost]
        src = np.abs(v).astype(np.int64) - 1
        assert np.all(np.abs(v) == np.round(np.abs(v))) and np.all(src >= 0) and np.all(src < cells), comp
        si, sj, sk = src % n[0], (src // n[0]) % n[1], src // (n[0] * n[1])
        gi, gj, gk = I[ghost], J[ghost], K[ghost]
        scol = (si + sj + sk) & 1
        # (2) face readers of the same colour are the source itself or its pole partner
        dims = 3 if nd == 3 else 2
        for dd in range(dims):
            for s in (-1, 1):
                ri, rj, rk = gi + (dd == 0) * s, gj + (dd == 1) * s, gk + (dd == 2) * s
                rin = (ri >= 0) & (ri < n[0]) & (rj >= 0) & (rj < n[1]) & (rk >= 0) & (rk < nk)
                same = rin & (((ri + rj + rk) & 1) == scol) & ~((ri == si) & (rj == sj) & (rk == sk))
                if not same.any():
                    continue
                assert nd == 3 and geom != "cart", (comp, dd, s)
                ok = (ri == si) & (rj == sj) & (np.abs(rk - sk) == nk // 2)
                assert np.all(ok[same]), (comp, dd, s)


def test_two_phi_planes_break_the_pairing():
    """n_phi = 2: the origin ghost (-1, j, k) copies (0, n_theta - 1 - j,
    k + 1), a cell of the reader's colour in another row."""
    n = [8, 4, 2]
    d = o.desc("sph", n, [0, 0, 0], [30.0, PI, 2 * PI])
    g = np.zeros(o.shape(d, True))
    g[1:-1, 1:-1, 1:-1] = (np.arange(64) + 1.0).reshape(o.shape(d))
    o.fill_ghosts(d, "dirichlet", 0, g)
    for j in range(n[1]):
        for k in range(n[2]):
            src = int(abs(g[k + 1, j + 1, 0])) - 1
            si, sj, sk = src % n[0], (src // n[0]) % n[1], src // (n[0] * n[1])
            assert (si, sj, sk) == (0, n[1] - 1 - j, (k + 1) % 2)
            assert (si + sj + sk) % 2 == (0 + j + k) % 2 and sj != j
