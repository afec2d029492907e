"""Manufactured fields for the oracle pins: smooth Cartesian scalar and
vector fields, sampled on a (ghosted) curvilinear grid, with their exact
continuous derivatives computed symbolically (sympy) in Cartesian
coordinates and projected on the grid's orthonormal basis."""
import numpy as np
import sympy as sp

X, Y, Z = sp.symbols("x y z", real=True)


def scalar_expr(axisym):
    if axisym:
        R2 = X ** 2 + Y ** 2
        return sp.exp(-(R2 + (Z - 0.3) ** 2) / 0.8) * (1 + 0.3 * Z + 0.1 * R2)
    return sp.exp(-((X - 0.2) ** 2 + (Y + 0.1) ** 2 + (Z - 0.3) ** 2) / 0.6) * (1 + 0.2 * X * Y + 0.1 * Z)


def vector_expr(axisym):
    if axisym:
        R2 = X ** 2 + Y ** 2
        g = sp.exp(-(R2 + (Z - 0.2) ** 2) / 0.7) * (1 + 0.2 * Z)
        h = sp.exp(-(R2 + (Z + 0.1) ** 2) / 0.9) * (0.5 + 0.3 * R2)
        k = sp.exp(-(R2 + Z ** 2) / 0.6) * (1 - 0.4 * Z)
        return [X * g - Y * h, Y * g + X * h, k]
    e = sp.exp(-((X - 0.2) ** 2 + (Y + 0.15) ** 2 + (Z - 0.1) ** 2) / 0.7)
    return [e * (1 + 0.3 * Y), e * (0.5 - 0.2 * X * Z), e * (0.8 + 0.25 * X)]


def planar(expr):
    """Drop z (2D Cartesian fields are z-independent)."""
    return expr.subs(Z, 0)


def lap(e):
    return sp.diff(e, X, 2) + sp.diff(e, Y, 2) + sp.diff(e, Z, 2)


def vec_op(F):
    div = sp.diff(F[0], X) + sp.diff(F[1], Y) + sp.diff(F[2], Z)
    grad = [sp.diff(div, v) for v in (X, Y, Z)]
    return [lap(F[c]) + sp.Rational(1, 3) * grad[c] for c in range(3)]


def sym_grad(F):
    """A~_ij = d_i F_j + d_j F_i - 2/3 delta_ij div F (Cartesian)."""
    v = (X, Y, Z)
    div = sum(sp.diff(F[c], v[c]) for c in range(3))
    return [[sp.diff(F[j], v[i]) + sp.diff(F[i], v[j]) - (sp.Rational(2, 3) * div if i == j else 0)
             for j in range(3)] for i in range(3)]


def fn(e):
    return sp.lambdify((X, Y, Z), e, "numpy")


def coords(geom, n, lo, hi, ghosted=True):
    """Coordinate arrays q0, q1, q2 broadcast to the (ghosted) array shape."""
    nd = len(n)
    g = 1 if ghosted else 0
    axes = []
    for d in range(nd):
        h = (hi[d] - lo[d]) / n[d]
        axes.append(lo[d] + (np.arange(-g, n[d] + g) + 0.5) * h)
    if nd == 2:
        q1, q0 = np.meshgrid(axes[1], axes[0], indexing="ij")
        q2 = np.zeros_like(q0)
    else:
        q2, q1, q0 = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return q0, q1, q2


def cart_and_basis(geom, q0, q1, q2):
    """Cartesian position and the orthonormal basis vectors (as Cartesian
    triples) of the grid's components at each point."""
    if geom == "cart":
        one, zero = np.ones_like(q0), np.zeros_like(q0)
        return (q0, q1, q2), [(one, zero, zero), (zero, one, zero), (zero, zero, one)]
    if geom == "cyl":
        R, z, ph = q0, q1, q2
        c, s = np.cos(ph), np.sin(ph)
        zero, one = np.zeros_like(R), np.ones_like(R)
        return (R * c, R * s, z), [(c, s, zero), (zero, zero, one), (-s, c, zero)]
    r, th, ph = q0, q1, q2
    st, ct, sp_, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    pos = (r * st * cp, r * st * sp_, r * ct)
    return pos, [(st * cp, st * sp_, ct), (ct * cp, ct * sp_, -st), (-sp_, cp, np.zeros_like(r))]


def eval_scalar(e, geom, q0, q1, q2):
    (x, y, z), _ = cart_and_basis(geom, q0, q1, q2)
    return np.ascontiguousarray(np.broadcast_to(fn(e)(x, y, z), q0.shape), dtype=np.float64)


def eval_vector(F, geom, q0, q1, q2):
    """Physical components of a Cartesian vector field."""
    (x, y, z), basis = cart_and_basis(geom, q0, q1, q2)
    comps = [np.broadcast_to(fn(F[c])(x, y, z), q0.shape) for c in range(3)]
    return [np.ascontiguousarray(sum(basis[a][c] * comps[c] for c in range(3))) for a in range(3)]


def eval_tensor(T, geom, q0, q1, q2):
    (x, y, z), basis = cart_and_basis(geom, q0, q1, q2)
    comps = [[np.broadcast_to(fn(T[i][j])(x, y, z), q0.shape) for j in range(3)] for i in range(3)]
    out = {}
    for a in range(3):
        for b in range(3):
            out[(a, b)] = sum(basis[a][i] * basis[b][j] * comps[i][j] for i in range(3) for j in range(3))
    return out
