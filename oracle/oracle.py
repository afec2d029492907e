"""ctypes binding of the plain FP64 CPU oracle (``mg_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this module; the CUDA library never does.
The oracle follows the paper's multigrid (Sec. 2.7) and xCFC / divergence
cleaning equations (Secs. 2.6, 2.2) step by step; see the C file's header for
the passages and readings.

Arrays crossing this boundary are float64, C-contiguous, dimension 0
fastest: numpy shape (n2, n1, n0) in 3D and (n1, n0) in 2D.  "Ghosted"
arrays carry one ghost layer per active dimension: shape (n2+2, n1+2, n0+2)
or (n1+2, n0+2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

GEOM = {"cart": 0, "cyl": 1, "sph": 2}
BC = {"robin": 0, "dirichlet": 1, "neumann": 2}
EQ = {"psi": 0, "lin": 1, "vec": 2}
MIXED = {"4pt": 0, "corner": 1}
STATUS = {0: "ok", 3: "noconv", 4: "stalled", 5: "nan"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP colour loops)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("geom", C.c_int), ("n", C.c_int * 3),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("nu1", C.c_int), ("nu2", C.c_int), ("max_cycles", C.c_int),
                ("tol", C.c_double), ("mixed", C.c_int), ("stall_window", C.c_int),
                ("accel_depth", C.c_int), ("cycle", C.c_int)]


class Report(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("rel", C.c_double),
                ("nhist", C.c_int), ("hist", C.c_double * 1024)]

    def as_dict(self):
        return {"status": STATUS.get(self.status, self.status), "cycles": self.cycles,
                "rel": self.rel, "hist": list(self.hist[: self.nhist])}


class CfcReport(C.Structure):
    _fields_ = [("psi_only", C.c_int), ("rep", Report * 4), ("seconds", C.c_double)]


class DivbReport(C.Structure):
    _fields_ = [("solve", Report), ("max_div_before", C.c_double), ("l2_div_before", C.c_double),
                ("max_div_after", C.c_double), ("l2_div_after", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            P = C.c_void_p
            D = C.POINTER(Desc)
            _lib.or_num_levels.argtypes = [D]
            _lib.or_solve_scalar.argtypes = [D, C.c_int, C.c_int, C.c_int, P, P, P, P, P,
                                             C.POINTER(Report)]
            _lib.or_solve_vector.argtypes = [D, C.c_int, P, P, C.POINTER(Report)]
            _lib.or_ghosted_size.argtypes = [D]
            _lib.or_ghosted_size.restype = C.c_long
            _lib.or_fill_ghosts.argtypes = [D, C.c_int, C.c_int, P]
            _lib.or_apply_raw.argtypes = [D, C.c_int, P, P, P, P, P]
            _lib.or_smooth.argtypes = [D, C.c_int, C.c_int, C.c_int, P, P, P, P, P]
            _lib.or_restrict.argtypes = [D, P, P]
            _lib.or_prolong_add.argtypes = [D, P, P]
            _lib.or_aij.argtypes = [D, P, P, P]
            _lib.or_solve_cfc.argtypes = [D, P, P, P, P, P, P, P, C.POINTER(CfcReport)]
            _lib.or_clean_divb.argtypes = [D, P, P, C.POINTER(DivbReport)]
            _lib.or_clean_divb_exact.argtypes = [D, P, P, C.POINTER(DivbReport)]
            I3 = C.c_int * 3
            _lib.or_solve_scalar_amr.argtypes = [D, I3, I3, C.c_int, C.c_int, P, P, P, P, P, P, P, P, P, P,
                                                 C.POINTER(Report)]
            _lib.or_apply_amr.argtypes = [D, I3, I3, C.c_int, C.c_int, P, P, P, P, P, P, P, P, P, P]
            _lib.or_div_c.argtypes = [D, P, P]
            _lib.or_beta_rhs.argtypes = [D, P, P, P, P, P]
        return _lib


def desc(geom, n, lo, hi, nu1=2, nu2=2, max_cycles=200, tol=1e-10, mixed="4pt", stall_window=10,
         accel_depth=0, cycle="v"):
    """Grid + solver descriptor.  n, lo, hi have one entry per dimension."""
    d = Desc()
    nd = len(n)
    d.ndim = nd
    d.geom = GEOM[geom]
    for k in range(3):
        d.n[k] = n[k] if k < nd else 1
        d.lo[k] = lo[k] if k < nd else 0.0
        d.hi[k] = hi[k] if k < nd else 1.0
    d.nu1, d.nu2, d.max_cycles, d.tol = nu1, nu2, min(max_cycles, 1000), tol
    d.mixed = MIXED[mixed]
    d.stall_window = stall_window
    d.accel_depth = accel_depth
    d.cycle = {"v": 0, "fmg": 1}[cycle]
    return d


def shape(d, ghosted=False):
    g = 2 if ghosted else 0
    s = [d.n[k] + g for k in range(d.ndim)]
    return tuple(reversed(s))


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def _parr(arrs):
    ptrs = (C.c_void_p * len(arrs))(*[_p(a) for a in arrs])
    return ptrs


def num_levels(d):
    return lib().or_num_levels(C.byref(d))


def solve_scalar(d, kind, bc, u, U=None, A2=None, c=None, f=None, zero_mean=False):
    """Solve L(u) = f for one scalar (kind 'psi' or 'lin'); u updated in place."""
    r = Report()
    lib().or_solve_scalar(C.byref(d), EQ[kind], BC[bc], int(zero_mean), _p(U), _p(A2), _p(c),
                          _p(f), _p(u), C.byref(r))
    return r.as_dict()


def solve_vector(d, bc, f, V):
    """Solve lap V + 1/3 grad div V = f; f and V are lists of 3 arrays."""
    r = Report()
    fp, vp = _parr(f), _parr(V)
    lib().or_solve_vector(C.byref(d), BC[bc], fp, vp, C.byref(r))
    return r.as_dict()


def fill_ghosts(d, bc, comp, u):
    """Fill the ghosts of a ghosted array in place (comp -1 scalar)."""
    lib().or_fill_ghosts(C.byref(d), BC[bc], comp, _p(u))


def apply_raw(d, kind, V, U=None, A2=None, c=None):
    """Apply L to ghosted field(s) without refilling ghosts; returns ghosted
    output(s) with the interior written."""
    ncomp = 3 if kind == "vec" else 1
    if ncomp == 1 and not isinstance(V, (list, tuple)):
        V = [V]
    Vs = list(V) + [V[0]] * (3 - len(V))
    out = [np.zeros(shape(d, True)) for _ in range(3)]
    lib().or_apply_raw(C.byref(d), EQ[kind], _parr(Vs), _p(U), _p(A2), _p(c), _parr(out))
    return out[:ncomp] if ncomp == 3 else out[0]


def smooth(d, kind, bc, nsweeps, u, f, U=None, A2=None, c=None):
    """nsweeps red-black NGS sweeps on ghosted arrays (in place)."""
    if not isinstance(u, (list, tuple)):
        u, f = [u], [f]
    us = list(u) + [u[0]] * (3 - len(u))
    fs = list(f) + [f[0]] * (3 - len(f))
    lib().or_smooth(C.byref(d), EQ[kind], BC[bc], nsweeps, _parr(us), _parr(fs), _p(U), _p(A2),
                    _p(c))


def coarse_desc(d):
    nd = d.ndim
    return desc({0: "cart", 1: "cyl", 2: "sph"}[d.geom], [d.n[k] // 2 for k in range(nd)],
                [d.lo[k] for k in range(nd)], [d.hi[k] for k in range(nd)])


def restrict(d, uf):
    uc = np.zeros(shape(coarse_desc(d), True))
    lib().or_restrict(C.byref(d), _p(uf), _p(uc))
    return uc


def prolong_add(d, uf, e):
    lib().or_prolong_add(C.byref(d), _p(uf), _p(e))


def aij(d, X, want_components=False):
    """A2 (and optionally the six A~ components rr, tt, pp, rt, rp, tp)."""
    A2 = np.zeros(shape(d))
    A6 = [np.zeros(shape(d)) for _ in range(6)] if want_components else None
    lib().or_aij(C.byref(d), _parr(X), _parr(A6) if A6 else None, _p(A2))
    return (A2, A6) if want_components else A2


def solve_cfc(d, U, S, Si, psi, alpha, beta, X, psi_only=False):
    """xCFC Steps 1-6 (Sec. 2.6); psi, alpha, beta[3], X[3] updated in place."""
    r = CfcReport()
    r.psi_only = int(psi_only)
    st = lib().or_solve_cfc(C.byref(d), _p(U), _p(S), _parr(Si), _p(psi), _p(alpha), _parr(beta),
                            _parr(X), C.byref(r))
    names = ["X", "psi", "alphapsi", "beta"]
    return {"status": STATUS.get(st, st), **{names[k]: r.rep[k].as_dict() for k in range(4)}}


def clean_divb(d, B, phi, exact=False):
    """Elliptic divergence cleaning (eqs. poisson, update_bfield); B in place.
    exact: the exact-projection variant (Cartesian; div_c grad_c Phi = b,
    split into its 2^d compact parity-class problems)."""
    r = DivbReport()
    Bs = list(B) + [B[0]] * (3 - len(B))
    fn = lib().or_clean_divb_exact if exact else lib().or_clean_divb
    st = fn(C.byref(d), _parr(Bs), _p(phi), C.byref(r))
    return {"status": STATUS.get(st, st), "solve": r.solve.as_dict(),
            "max_div_before": r.max_div_before, "l2_div_before": r.l2_div_before,
            "max_div_after": r.max_div_after, "l2_div_after": r.l2_div_after}


def div_c(d, B):
    out = np.zeros(shape(d))
    Bs = list(B) + [B[0]] * (3 - len(B))
    lib().or_div_c(C.byref(d), _parr(Bs), _p(out))
    return out


def beta_rhs(d, X, psi, alpha, Si):
    """Right-hand side of eq. (beta) from X, psi, alpha and S_i (Sec. 2.6 Step 6)."""
    f = [np.zeros(shape(d)) for _ in range(3)]
    lib().or_beta_rhs(C.byref(d), _parr(X), _p(psi), _p(alpha), _parr(Si), _parr(f))
    return f


def patch_shape(d, a, b):
    """numpy shape of the refined patch over base cells a <= I < b."""
    return tuple(reversed([2 * (b[k] - a[k]) for k in range(d.ndim)]))


def _box(v, nd):
    return (C.c_int * 3)(*([int(x) for x in v] + [0] * (3 - nd)))


def solve_scalar_amr(d, a, b, kind, bc, u, up, U=None, A2=None, c=None, f=None, Up=None, A2p=None, cp=None,
                     fp=None):
    """Two-level composite-grid solve (base grid of d, refined patch over
    base cells a <= I < b); u (base) and up (patch) updated in place."""
    r = Report()
    st = lib().or_solve_scalar_amr(C.byref(d), _box(a, d.ndim), _box(b, d.ndim), EQ[kind], BC[bc], _p(U), _p(A2),
                                   _p(c), _p(f), _p(Up), _p(A2p), _p(cp), _p(fp), _p(u), _p(up), C.byref(r))
    if st == 1 and r.cycles == 0 and r.nhist == 0:
        raise ValueError("patch box rejected")
    return r.as_dict()


def apply_amr(d, a, b, kind, bc, u, up, U=None, A2=None, c=None, Up=None, A2p=None, cp=None):
    """The composite operator on (u, up): (out on uncovered base cells, 0 on
    covered ones; out on the patch)."""
    out = np.zeros(shape(d))
    outp = np.zeros(patch_shape(d, a, b))
    st = lib().or_apply_amr(C.byref(d), _box(a, d.ndim), _box(b, d.ndim), EQ[kind], BC[bc], _p(U), _p(A2), _p(c),
                            _p(Up), _p(A2p), _p(cp), _p(u), _p(up), _p(out), _p(outp))
    if st:
        raise ValueError("patch box rejected")
    return out, outp
