"""ctypes binding of libgmunu_mg.so (the C ABI of include/mg.h).

Argument marshalling only: every step of the solve runs in the CUDA
library.  Arrays are torch tensors: float64, contiguous, shaped like the
grid with dimension 0 fastest, i.e. (n1, n0) in 2D and (n2, n1, n0) in 3D;
on the hierarchy's CUDA device, or on the host with ``host=True``
(MG_HOST_POINTERS, pinned memory recommended).  If the library cannot be
loaded this module raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

MG_OK, MG_ERR_INVALID, MG_ERR_OOM, MG_ERR_NOCONV, MG_ERR_STALLED, MG_ERR_NAN, MG_ERR_CUDA = range(7)
MG_ERR_BUSY, MG_ERR_NOTFOUND = 7, 8
MG_CART, MG_CYL, MG_SPH = 0, 1, 2
MG_FP64, MG_MIXED = 0, 1
MG_MIXED_4PT, MG_MIXED_CORNER = 0, 1
MG_BC_ROBIN, MG_BC_DIRICHLET, MG_BC_NEUMANN = 0, 1, 2
MG_EQ_PSI, MG_EQ_LIN, MG_EQ_VEC = 0, 1, 2
MG_CFC_PSI_ONLY, MG_HOST_POINTERS = 1, 2
MG_DIVB_COMPACT, MG_DIVB_EXACT = 0, 1
MG_HIST = 1024

GEOM = {"cart": MG_CART, "cyl": MG_CYL, "sph": MG_SPH}
BC = {"robin": MG_BC_ROBIN, "dirichlet": MG_BC_DIRICHLET, "neumann": MG_BC_NEUMANN}
KIND = {"psi": MG_EQ_PSI, "lin": MG_EQ_LIN, "vec": MG_EQ_VEC}
STATUS = {0: "ok", 1: "invalid", 2: "oom", 3: "noconv", 4: "stalled", 5: "nan", 6: "cuda", 7: "busy",
          8: "notfound"}

# Every symbol include/mg.h declares.
EXPORTS = ["mg_strerror", "mg_last_error", "mg_hierarchy_bytes", "mg_create_hierarchy", "mg_destroy_hierarchy",
           "mg_num_levels", "mg_solve_cfc", "mg_clean_divB", "mg_solve_scalar", "mg_solve_vector",
           "mg_apply_operator", "mg_smooth", "mg_compute_a2", "mg_divergence", "mg_restrict", "mg_prolong_add",
           "mg_kernel_launches", "mg_profile_enable", "mg_profile_read", "mg_divb_norms_noalloc",
           "mg_server_create", "mg_server_destroy", "mg_submit", "mg_poll", "mg_solve_scalar_amr", "mg_apply_amr",
           "mg_solve_cfc_batch"]
MG_REQ_CFC, MG_REQ_DIVB, MG_REQ_AMR = 0, 1, 2
MG_NOALLOC_MAX_CELLS = 2097152
PROF_CLASSES = ["smooth64_scalar", "smooth64_vec", "smooth32_scalar", "smooth32_vec", "resid64_scalar",
                "resid64_vec", "sweep64_fused", "sweep32_fused", "smooth32_coarse", "aa_update", "aa_combine",
                "block_cycle32", "resid64_psi"]


class mg_grid_desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("geom", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("precision", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("max_cycles", C.c_int), ("tol", C.c_double), ("mixed_deriv", C.c_int),
                ("stall_window", C.c_int), ("accel_depth", C.c_int), ("cycle", C.c_int),
                ("divb_variant", C.c_int)]


class mg_solve_report(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("rel", C.c_double), ("nhist", C.c_int),
                ("hist", C.c_double * MG_HIST), ("ms", C.c_double), ("cell_updates", C.c_int64)]

    def as_dict(self):
        return {"status": STATUS.get(self.status, self.status), "cycles": self.cycles, "rel": self.rel,
                "hist": list(self.hist[: self.nhist]), "ms": self.ms, "cell_updates": self.cell_updates}


class mg_cfc_sources(C.Structure):
    _fields_ = [("U", C.c_void_p), ("S", C.c_void_p), ("Si", C.c_void_p * 3)]


class mg_cfc_fields(C.Structure):
    _fields_ = [("psi", C.c_void_p), ("alpha", C.c_void_p), ("beta", C.c_void_p * 3), ("X", C.c_void_p * 3)]


class mg_cfc_report(C.Structure):
    _fields_ = [("eq", mg_solve_report * 4), ("ms", C.c_double)]


class mg_batch_opts(C.Structure):
    _fields_ = [("team", C.c_int), ("team_cells", C.c_int64)]


class mg_batch_report(C.Structure):
    _fields_ = [("kernel_ms", C.c_double), ("blocks", C.c_int), ("team", C.c_int), ("persistent", C.c_int),
                ("general", C.c_int)]


class mg_divb_report(C.Structure):
    _fields_ = [("solve", mg_solve_report), ("max_div_before", C.c_double), ("l2_div_before", C.c_double),
                ("max_div_after", C.c_double), ("l2_div_after", C.c_double)]


class mg_amr_arrays(C.Structure):
    _fields_ = [("box_lo", C.c_int * 3), ("box_hi", C.c_int * 3), ("A2", C.c_void_p), ("Up", C.c_void_p),
                ("A2p", C.c_void_p), ("u", C.c_void_p), ("up", C.c_void_p)]


class mg_request(C.Structure):
    _fields_ = [("desc", mg_grid_desc), ("kind", C.c_int), ("flags", C.c_int), ("stream_id", C.c_uint64),
                ("src", mg_cfc_sources), ("io", mg_cfc_fields), ("B", C.c_void_p * 3), ("phi", C.c_void_p),
                ("wait_stream", C.c_void_p), ("amr", mg_amr_arrays)]


class mg_result(C.Structure):
    _fields_ = [("status", C.c_int), ("cfc", mg_cfc_report), ("divb", mg_divb_report), ("latency_ms", C.c_double),
                ("queue_ms", C.c_double), ("warm_started", C.c_int)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load (building first if needed) libgmunu_mg.so."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB if os.path.exists(_build.LIB) and not _build._stale() else _build.build()
        L = C.CDLL(path)
        P, I, D = C.c_void_p, C.c_int, C.POINTER(mg_grid_desc)
        L.mg_strerror.restype = C.c_char_p
        L.mg_strerror.argtypes = [I]
        L.mg_last_error.restype = C.c_char_p
        L.mg_last_error.argtypes = []
        L.mg_hierarchy_bytes.argtypes = [D, C.POINTER(C.c_size_t)]
        L.mg_create_hierarchy.argtypes = [D, P, C.POINTER(P)]
        L.mg_destroy_hierarchy.argtypes = [P]
        L.mg_num_levels.argtypes = [P, C.POINTER(I)]
        L.mg_solve_cfc.argtypes = [P, C.POINTER(mg_cfc_sources), C.POINTER(mg_cfc_fields), I,
                                   C.POINTER(mg_cfc_report)]
        L.mg_solve_cfc_batch.argtypes = [C.POINTER(P), I, C.POINTER(mg_cfc_sources), C.POINTER(mg_cfc_fields), I,
                                         C.POINTER(mg_batch_opts), C.POINTER(mg_cfc_report),
                                         C.POINTER(mg_batch_report)]
        L.mg_clean_divB.argtypes = [P, C.POINTER(P), P, I, C.POINTER(mg_divb_report)]
        L.mg_solve_scalar.argtypes = [P, I, I, I, P, P, P, P, P, C.POINTER(mg_solve_report)]
        L.mg_solve_vector.argtypes = [P, I, C.POINTER(P), C.POINTER(P), C.POINTER(mg_solve_report)]
        L.mg_apply_operator.argtypes = [P, I, I, C.POINTER(P), P, P, P, C.POINTER(P)]
        L.mg_smooth.argtypes = [P, I, I, I, C.POINTER(P), C.POINTER(P), P, P, P]
        L.mg_compute_a2.argtypes = [P, C.POINTER(P), P]
        L.mg_divergence.argtypes = [P, C.POINTER(P), P]
        L.mg_restrict.argtypes = [P, P, P]
        L.mg_prolong_add.argtypes = [P, I, P, P]
        L.mg_kernel_launches.restype = C.c_uint64
        L.mg_kernel_launches.argtypes = []
        L.mg_profile_enable.argtypes = [P, I]
        L.mg_profile_read.argtypes = [P, I, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.mg_server_create.argtypes = [C.c_size_t, I, I, C.POINTER(P)]
        L.mg_server_destroy.argtypes = [P]
        L.mg_submit.argtypes = [P, C.POINTER(mg_request), C.POINTER(C.c_uint64)]
        L.mg_poll.argtypes = [P, C.c_uint64, C.POINTER(I), C.POINTER(mg_result)]
        I3 = C.c_int * 3
        L.mg_solve_scalar_amr.argtypes = [P, C.POINTER(I3), C.POINTER(I3), I, I, P, P, P, P, P, P, P, P, P, P,
                                          C.POINTER(mg_solve_report)]
        L.mg_apply_amr.argtypes = [P, C.POINTER(I3), C.POINTER(I3), I, I, P, P, P, P, P, P, P, P, P, P]
        L.mg_divb_norms_noalloc.argtypes = [I, C.POINTER(C.c_int * 3), C.POINTER(C.c_double * 3),
                                            C.POINTER(C.c_double * 3), C.POINTER(P), P,
                                            C.POINTER(C.c_double), C.POINTER(C.c_double)]
        _lib = L
        return L


class MgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        detail = lib().mg_last_error().decode()
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), detail))


def _check(status, where, allow=(MG_OK,)):
    if status not in allow:
        raise MgError(status, where)
    return status


def grid_desc(geom, n, lo=None, hi=None, precision="fp64", nu1=2, nu2=2, max_cycles=1000, tol=1e-10,
              mixed="4pt", stall_window=10, accel_depth=0, cycle="v", divb="compact"):
    """Build an mg_grid_desc; lo / hi default to the natural domain of the
    geometry where it is fixed (spherical angles, cylindrical phi)."""
    d = mg_grid_desc()
    nd = len(n)
    d.ndim = nd
    d.geom = GEOM[geom]
    if lo is None:
        lo = [0.0] * nd
    for k in range(3):
        d.n[k] = n[k] if k < nd else 1
        d.lo[k] = lo[k] if k < nd else 0.0
        d.hi[k] = hi[k] if k < nd else 1.0
    d.precision = MG_MIXED if precision == "mixed" else MG_FP64
    d.nu1, d.nu2, d.max_cycles, d.tol = nu1, nu2, max_cycles, tol
    d.mixed_deriv = MG_MIXED_CORNER if mixed == "corner" else MG_MIXED_4PT
    d.stall_window = stall_window
    d.accel_depth = accel_depth
    d.cycle = {"v": 0, "fmg": 1}[cycle]
    d.divb_variant = {"compact": MG_DIVB_COMPACT, "exact": MG_DIVB_EXACT}[divb]
    return d


def mg_hierarchy_bytes(desc) -> int:
    out = C.c_size_t()
    _check(lib().mg_hierarchy_bytes(C.byref(desc), C.byref(out)), "mg_hierarchy_bytes")
    return out.value


class Hierarchy:
    """Owner of an mg_hierarchy* (freed on close / garbage collection)."""

    def __init__(self, desc, stream=None):
        import torch
        self.desc = desc
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.device = stream.device
        h = C.c_void_p()
        _check(lib().mg_create_hierarchy(C.byref(desc), C.c_void_p(stream.cuda_stream), C.byref(h)),
               "mg_create_hierarchy")
        self.handle = h
        nl = C.c_int()
        _check(lib().mg_num_levels(h, C.byref(nl)), "mg_num_levels")
        self.nlev = nl.value
        nd = desc.ndim
        self.shape = tuple(desc.n[k] for k in reversed(range(nd)))

    def close(self):
        if getattr(self, "handle", None):
            lib().mg_destroy_hierarchy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_shape(self, l):
        nd = self.desc.ndim
        return tuple(self.desc.n[k] >> l for k in reversed(range(nd)))


def mg_create_hierarchy(desc, stream=None) -> Hierarchy:
    return Hierarchy(desc, stream)


def mg_destroy_hierarchy(h: Hierarchy):
    h.close()


def _ptr(t, h, host=False, shape=None, name="array"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("%s must be contiguous float64" % name)
    if host:
        if t.is_cuda:
            raise ValueError("%s must be a host tensor with host=True" % name)
    elif not t.is_cuda or t.device != h.device:
        raise ValueError("%s must be on %s" % (name, h.device))
    want = shape if shape is not None else h.shape
    if tuple(t.shape) != tuple(want):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(want)))
    return C.c_void_p(t.data_ptr())


def _parr(ts, h, host=False, name="array"):
    arr = (C.c_void_p * 3)()
    for k, t in enumerate(ts):
        p = _ptr(t, h, host, name="%s[%d]" % (name, k))
        arr[k] = p.value if p is not None else None
    return arr


def mg_solve_cfc(h, U, S, Si, psi, alpha, beta, X, psi_only=False, host=False, allow=(MG_OK,)):
    """xCFC Steps 1-6 (Sec. 2.6).  Returns per-equation reports."""
    src = mg_cfc_sources()
    io = mg_cfc_fields()
    src.U = _ptr(U, h, host, name="U").value
    io.psi = _ptr(psi, h, host, name="psi").value
    if not psi_only:
        src.S = _ptr(S, h, host, name="S").value
        io.alpha = _ptr(alpha, h, host, name="alpha").value
        src.Si = _parr(Si, h, host, "Si")
        io.beta = _parr(beta, h, host, "beta")
        io.X = _parr(X, h, host, "X")
    rep = mg_cfc_report()
    flags = (MG_CFC_PSI_ONLY if psi_only else 0) | (MG_HOST_POINTERS if host else 0)
    st = lib().mg_solve_cfc(h.handle, C.byref(src), C.byref(io), flags, C.byref(rep))
    _check(st, "mg_solve_cfc", allow)
    names = ["X", "psi", "alphapsi", "beta"]
    return {"status": STATUS[st], "ms": rep.ms, **{names[k]: rep.eq[k].as_dict() for k in range(4)}}


def mg_solve_cfc_batch(problems, psi_only=False, reports=True, team=0, team_cells=0, allow=(MG_OK,)):
    """Independent xCFC solves in one persistent launch (mg_solve_cfc_batch).
    problems: sequence of (h, U, S, Si, psi, alpha, beta, X) as mg_solve_cfc
    takes them (device tensors, one hierarchy per problem); team, team_cells:
    the launch shape (0: the library's default).  Returns (per-problem
    reports or None, batch report dict)."""
    count = len(problems)
    hs = (C.c_void_p * count)()
    srcs = (mg_cfc_sources * count)()
    ios = (mg_cfc_fields * count)()
    for q, (h, U, S, Si, psi, alpha, beta, X) in enumerate(problems):
        hs[q] = h.handle
        srcs[q].U = _ptr(U, h, name="U").value
        ios[q].psi = _ptr(psi, h, name="psi").value
        if not psi_only:
            srcs[q].S = _ptr(S, h, name="S").value
            ios[q].alpha = _ptr(alpha, h, name="alpha").value
            srcs[q].Si = _parr(Si, h, name="Si")
            ios[q].beta = _parr(beta, h, name="beta")
            ios[q].X = _parr(X, h, name="X")
    reps = (mg_cfc_report * count)() if reports else None
    brep = mg_batch_report()
    opts = mg_batch_opts(team, team_cells)
    st = lib().mg_solve_cfc_batch(hs, count, srcs, ios, MG_CFC_PSI_ONLY if psi_only else 0, C.byref(opts), reps,
                                  C.byref(brep))
    _check(st, "mg_solve_cfc_batch", allow)
    names = ["X", "psi", "alphapsi", "beta"]
    out = None
    if reports:
        out = [{"ms": r.ms, **{names[k]: r.eq[k].as_dict() for k in range(4)}} for r in reps]
    return out, {"status": STATUS[st], "kernel_ms": brep.kernel_ms, "blocks": brep.blocks, "team": brep.team,
                 "persistent": brep.persistent, "general": brep.general}


def mg_clean_divB(h, B, phi=None, host=False, allow=(MG_OK,)):
    """Elliptic divergence cleaning (eqs. poisson, update_bfield); B in place."""
    arr = (C.c_void_p * 3)()
    for k, t in enumerate(B):
        arr[k] = _ptr(t, h, host, name="B[%d]" % k).value
    rep = mg_divb_report()
    st = lib().mg_clean_divB(h.handle, arr, _ptr(phi, h, host, name="phi"), MG_HOST_POINTERS if host else 0,
                             C.byref(rep))
    _check(st, "mg_clean_divB", allow)
    return {"status": STATUS[st], "solve": rep.solve.as_dict(), "max_div_before": rep.max_div_before,
            "l2_div_before": rep.l2_div_before, "max_div_after": rep.max_div_after,
            "l2_div_after": rep.l2_div_after}


def mg_solve_scalar(h, kind, bc, u, U=None, A2=None, c=None, f=None, zero_mean=False, allow=(MG_OK,)):
    rep = mg_solve_report()
    st = lib().mg_solve_scalar(h.handle, KIND[kind], BC[bc], int(zero_mean), _ptr(U, h, name="U"),
                               _ptr(A2, h, name="A2"), _ptr(c, h, name="c"), _ptr(f, h, name="f"),
                               _ptr(u, h, name="u"), C.byref(rep))
    _check(st, "mg_solve_scalar", allow)
    return rep.as_dict()


def patch_shape(h, box_lo, box_hi):
    """Shape (n2, n1, n0) / (n1, n0) of the refined patch over base cells
    box_lo <= I < box_hi."""
    nd = h.desc.ndim
    return tuple(2 * (box_hi[k] - box_lo[k]) for k in reversed(range(nd)))


def _box3(v):
    return (C.c_int * 3)(*(list(v) + [0] * (3 - len(v))))


def mg_solve_scalar_amr(h, box_lo, box_hi, kind, bc, u, up, U=None, A2=None, c=None, f=None, Up=None, A2p=None,
                        cp=None, fp=None, allow=(MG_OK,)):
    """Two-level composite-grid solve (base grid of h, refined patch over
    base cells box_lo <= I < box_hi); u and up updated in place."""
    ps = patch_shape(h, box_lo, box_hi)
    rep = mg_solve_report()
    st = lib().mg_solve_scalar_amr(h.handle, C.byref(_box3(box_lo)), C.byref(_box3(box_hi)), KIND[kind], BC[bc],
                                   _ptr(U, h, name="U"), _ptr(A2, h, name="A2"), _ptr(c, h, name="c"),
                                   _ptr(f, h, name="f"), _ptr(Up, h, shape=ps, name="Up"),
                                   _ptr(A2p, h, shape=ps, name="A2p"), _ptr(cp, h, shape=ps, name="cp"),
                                   _ptr(fp, h, shape=ps, name="fp"), _ptr(u, h, name="u"),
                                   _ptr(up, h, shape=ps, name="up"), C.byref(rep))
    _check(st, "mg_solve_scalar_amr", allow)
    return rep.as_dict()


def mg_apply_amr(h, box_lo, box_hi, kind, bc, u, up, out, outp, U=None, A2=None, c=None, Up=None, A2p=None,
                 cp=None):
    ps = patch_shape(h, box_lo, box_hi)
    st = lib().mg_apply_amr(h.handle, C.byref(_box3(box_lo)), C.byref(_box3(box_hi)), KIND[kind], BC[bc],
                            _ptr(U, h, name="U"), _ptr(A2, h, name="A2"), _ptr(c, h, name="c"),
                            _ptr(Up, h, shape=ps, name="Up"), _ptr(A2p, h, shape=ps, name="A2p"),
                            _ptr(cp, h, shape=ps, name="cp"), _ptr(u, h, name="u"), _ptr(up, h, shape=ps, name="up"),
                            _ptr(out, h, name="out"), _ptr(outp, h, shape=ps, name="outp"))
    _check(st, "mg_apply_amr")


def mg_solve_vector(h, bc, f, V, allow=(MG_OK,)):
    rep = mg_solve_report()
    st = lib().mg_solve_vector(h.handle, BC[bc], _parr(f, h, name="f"), _parr(V, h, name="V"), C.byref(rep))
    _check(st, "mg_solve_vector", allow)
    return rep.as_dict()


def mg_apply_operator(h, kind, bc, u, out, U=None, A2=None, c=None):
    us = list(u) if isinstance(u, (list, tuple)) else [u]
    os_ = list(out) if isinstance(out, (list, tuple)) else [out]
    _check(lib().mg_apply_operator(h.handle, KIND[kind], BC[bc], _parr(us, h, name="u"), _ptr(U, h, name="U"),
                                   _ptr(A2, h, name="A2"), _ptr(c, h, name="c"), _parr(os_, h, name="out")),
           "mg_apply_operator")


def mg_smooth(h, kind, bc, nsweeps, u, f=None, U=None, A2=None, c=None):
    us = list(u) if isinstance(u, (list, tuple)) else [u]
    fs = (list(f) if isinstance(f, (list, tuple)) else [f]) if f is not None else [None] * len(us)
    _check(lib().mg_smooth(h.handle, KIND[kind], BC[bc], nsweeps, _parr(us, h, name="u"), _parr(fs, h, name="f"),
                           _ptr(U, h, name="U"), _ptr(A2, h, name="A2"), _ptr(c, h, name="c")), "mg_smooth")


def mg_compute_a2(h, X, A2):
    _check(lib().mg_compute_a2(h.handle, _parr(X, h, name="X"), _ptr(A2, h, name="A2")), "mg_compute_a2")


def mg_divergence(h, B, div):
    arr = (C.c_void_p * 3)()
    for k, t in enumerate(B):
        arr[k] = _ptr(t, h, name="B[%d]" % k).value
    _check(lib().mg_divergence(h.handle, arr, _ptr(div, h, name="div")), "mg_divergence")


def mg_restrict(h, fine, coarse):
    _check(lib().mg_restrict(h.handle, _ptr(fine, h, name="fine"),
                             _ptr(coarse, h, shape=h.level_shape(1), name="coarse")), "mg_restrict")


def mg_prolong_add(h, bc, coarse_e, fine):
    _check(lib().mg_prolong_add(h.handle, BC[bc], _ptr(coarse_e, h, shape=h.level_shape(1), name="coarse_e"),
                                _ptr(fine, h, name="fine")), "mg_prolong_add")


def mg_kernel_launches() -> int:
    return int(lib().mg_kernel_launches())


def mg_profile_enable(h, enable=True):
    _check(lib().mg_profile_enable(h.handle, int(bool(enable))), "mg_profile_enable")


def mg_profile_read(h):
    """{class: (launches, device ms, cells)} since mg_profile_enable."""
    out = {}
    for k, name in enumerate(PROF_CLASSES):
        n, ms, cells = C.c_int64(), C.c_double(), C.c_int64()
        _check(lib().mg_profile_read(h.handle, k, C.byref(n), C.byref(ms), C.byref(cells)), "mg_profile_read")
        out[name] = (n.value, ms.value, cells.value)
    return out


def mg_divb_norms_noalloc(B, lo, hi, stream=None, allow=(MG_OK,)):
    """(max |div B|, |div B|_2) of a Cartesian field through the
    allocation-free entry point; B is a list of ndim CUDA float64 tensors
    shaped (n1, n0) or (n2, n1, n0).  Returns (status, max, l2)."""
    import torch
    nd = len(B)
    shp = tuple(B[0].shape)
    n = (C.c_int * 3)(*([shp[nd - 1 - d] for d in range(nd)] + [1] * (3 - nd)))
    lo3 = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - nd)))
    hi3 = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - nd)))
    arr = (C.c_void_p * 3)()
    for k, t in enumerate(B):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and tuple(t.shape) == shp):
            raise ValueError("B[%d] must be a contiguous CUDA float64 tensor of shape %s" % (k, shp))
        arr[k] = t.data_ptr()
    if stream is None:
        stream = torch.cuda.current_stream()
    mx, l2 = C.c_double(), C.c_double()
    st = lib().mg_divb_norms_noalloc(nd, C.byref(n), C.byref(lo3), C.byref(hi3), arr,
                                     C.c_void_p(stream.cuda_stream), C.byref(mx), C.byref(l2))
    _check(st, "mg_divb_norms_noalloc", allow)
    return st, mx.value, l2.value


class Server:
    """A request server (mg_server_create): submit() queues a CFC or div-B
    request and returns a ticket; poll() is non-blocking.  The tensors of a
    request are kept referenced until it has been collected."""

    def __init__(self, hbm_budget, max_slots=4, max_queue=256):
        h = C.c_void_p()
        _check(lib().mg_server_create(int(hbm_budget), max_slots, max_queue, C.byref(h)), "mg_server_create")
        self.handle = h
        self._keep = {}

    def close(self):
        if getattr(self, "handle", None):
            lib().mg_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _check_shapes(desc, named):
        """The request's arrays must have the grid's shape and dtype: the
        server reads and writes them through raw device pointers."""
        import torch
        want = tuple(desc.n[k] for k in reversed(range(desc.ndim)))
        for name, t in named:
            if t is None:
                continue
            if not isinstance(t, torch.Tensor) or not t.is_cuda:
                raise ValueError("%s must be a CUDA tensor" % name)
            if t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != want:
                raise ValueError("%s must be contiguous float64 of shape %s, got %s %s"
                                 % (name, want, t.dtype, tuple(t.shape)))

    def submit_cfc(self, desc, U, S, Si, psi, alpha, beta, X, psi_only=False, stream_id=0, allow=(MG_OK,)):
        named = [("U", U), ("psi", psi)]
        if not psi_only:
            named += [("S", S), ("alpha", alpha)] + [("Si[%d]" % k, Si[k]) for k in range(3)]
            named += [("beta[%d]" % k, beta[k]) for k in range(3)] + [("X[%d]" % k, X[k]) for k in range(3)]
        self._check_shapes(desc, named)
        r = mg_request()
        r.desc = desc
        r.kind = MG_REQ_CFC
        r.flags = MG_CFC_PSI_ONLY if psi_only else 0
        r.stream_id = stream_id
        r.src.U = U.data_ptr()
        r.io.psi = psi.data_ptr()
        if not psi_only:
            r.src.S = S.data_ptr()
            r.io.alpha = alpha.data_ptr()
            for k in range(3):
                r.src.Si[k] = Si[k].data_ptr()
                r.io.beta[k] = beta[k].data_ptr()
                r.io.X[k] = X[k].data_ptr()
        return self._submit(r, (U, S, Si, psi, alpha, beta, X), allow)

    def submit_amr(self, desc, box_lo, box_hi, U, A2, Up, A2p, u, up, allow=(MG_OK,)):
        """Eq. psi on the two-level composite grid (deviations u = psi - 1 on
        the base grid and up on the patch, updated in place)."""
        nd = desc.ndim
        pshape = tuple(2 * (box_hi[k] - box_lo[k]) for k in reversed(range(nd)))
        self._check_shapes(desc, [("U", U), ("A2", A2), ("u", u)])
        pd = mg_grid_desc()
        pd.ndim = nd
        for k in range(3):
            pd.n[k] = pshape[nd - 1 - k] if k < nd else 1
        self._check_shapes(pd, [("Up", Up), ("A2p", A2p), ("up", up)])
        r = mg_request()
        r.desc = desc
        r.kind = MG_REQ_AMR
        r.src.U = U.data_ptr()
        for k in range(3):
            r.amr.box_lo[k] = box_lo[k] if k < nd else 0
            r.amr.box_hi[k] = box_hi[k] if k < nd else 1
        r.amr.A2, r.amr.Up, r.amr.A2p = A2.data_ptr(), Up.data_ptr(), A2p.data_ptr()
        r.amr.u, r.amr.up = u.data_ptr(), up.data_ptr()
        return self._submit(r, (U, A2, Up, A2p, u, up), allow)

    def submit_divb(self, desc, B, phi=None, allow=(MG_OK,)):
        self._check_shapes(desc, [("B[%d]" % k, b) for k, b in enumerate(B)] + [("phi", phi)])
        r = mg_request()
        r.desc = desc
        r.kind = MG_REQ_DIVB
        for k, t in enumerate(B):
            r.B[k] = t.data_ptr()
        r.phi = phi.data_ptr() if phi is not None else None
        return self._submit(r, (B, phi), allow)

    def _submit(self, r, keep, allow):
        import torch
        r.wait_stream = torch.cuda.current_stream().cuda_stream
        t = C.c_uint64()
        st = lib().mg_submit(self.handle, C.byref(r), C.byref(t))
        _check(st, "mg_submit", allow)
        if st != MG_OK:
            return None
        self._keep[t.value] = keep
        return t.value

    def poll(self, ticket):
        """(done, result dict or None)."""
        done = C.c_int()
        res = mg_result()
        st = lib().mg_poll(self.handle, ticket, C.byref(done), C.byref(res))
        if st == MG_ERR_NOTFOUND:
            raise MgError(st, "mg_poll")
        if not done.value:
            return False, None
        self._keep.pop(ticket, None)
        names = ["X", "psi", "alphapsi", "beta"]
        out = {"status": STATUS.get(res.status, res.status), "latency_ms": res.latency_ms,
               "queue_ms": res.queue_ms, "warm_started": bool(res.warm_started),
               "cfc": {names[k]: res.cfc.eq[k].as_dict() for k in range(4)},
               "divb": {"solve": res.divb.solve.as_dict(), "max_div_before": res.divb.max_div_before,
                        "max_div_after": res.divb.max_div_after}}
        return True, out

    def wait(self, ticket, timeout_s=600.0):
        import time
        t0 = time.time()
        while True:
            done, res = self.poll(ticket)
            if done:
                return res
            if time.time() - t0 > timeout_s:
                raise TimeoutError("ticket %d not done after %.0f s" % (ticket, timeout_s))
            time.sleep(0.0005)


def mg_server_create(hbm_budget, max_slots=4, max_queue=256):
    return Server(hbm_budget, max_slots, max_queue)
