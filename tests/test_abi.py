"""The C ABI library loads and exports every entry point include/mg.h
declares (no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "mg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-zA-Z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("mg_create_hierarchy", "mg_destroy_hierarchy", "mg_solve_cfc", "mg_clean_divB",
                 "mg_hierarchy_bytes", "mg_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2012_07322_gb300 import build, mg
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(mg.EXPORTS) == _declared()


def test_host_only_entry_points():
    """Descriptor validation and the admission size need no device."""
    from paper_2012_07322_gb300 import mg
    import numpy as np
    d = mg.grid_desc("sph", [64, 32], hi=[100.0, np.pi])
    assert mg.mg_hierarchy_bytes(d) > 64 * 32 * 8 * 10
    bad = mg.grid_desc("sph", [64, 24], hi=[100.0, np.pi])          # 24 is not a power of two
    with pytest.raises(mg.MgError) as e:
        mg.mg_hierarchy_bytes(bad)
    assert e.value.status == mg.MG_ERR_INVALID
    bad = mg.grid_desc("sph", [64, 32], hi=[100.0, 3.0])             # theta must end at pi
    with pytest.raises(mg.MgError):
        mg.mg_hierarchy_bytes(bad)
    assert mg.mg_hierarchy_bytes(mg.grid_desc("sph", [64, 32], hi=[100.0, np.pi], cycle="fmg")) > 0
    # the exact projection adds the half-size hierarchy of its parity classes
    lo3, hi3 = [-1.0] * 3, [1.0] * 3
    plain = mg.mg_hierarchy_bytes(mg.grid_desc("cart", [32] * 3, lo3, hi3))
    exact = mg.mg_hierarchy_bytes(mg.grid_desc("cart", [32] * 3, lo3, hi3, divb="exact"))
    assert exact == plain + mg.mg_hierarchy_bytes(mg.grid_desc("cart", [16] * 3, lo3, hi3))
    bad = mg.grid_desc("sph", [64, 32], hi=[100.0, np.pi])
    bad.cycle = 7                                                     # neither V nor FMG
    with pytest.raises(mg.MgError):
        mg.mg_hierarchy_bytes(bad)
    assert mg.lib().mg_strerror(3) == b"not converged"


def _set(d, **kw):
    for k, v in kw.items():
        if isinstance(v, tuple):
            arr = getattr(d, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(d, k, v)
    return d


@pytest.mark.parametrize("what,geom,n,kw", [
    ("empty grid", "cart", [0, 8, 8], {}),
    ("one cell", "cart", [1, 8], {}),
    ("n not a power of two", "cart", [12, 8, 8], {}),
    ("negative n", "cart", [-8, 8], {}),
    ("ndim 1", "cart", [8, 8], {"ndim": 1}),
    ("ndim 4", "cart", [8, 8, 8], {"ndim": 4}),
    ("geometry", "cart", [8, 8], {"geom": 7}),
    ("lo == hi", "cart", [8, 8], {"hi": (-1.0, 1.0, 1.0)}),
    ("spherical r from 1", "sph", [8, 8], {"lo": (1.0, 0.0, 0.0)}),
    ("spherical phi short of 2 pi", "sph", [8, 8, 8], {"hi": (10.0, 3.141592653589793, 6.0)}),
    ("cylindrical R from 1", "cyl", [8, 8], {"lo": (1.0, -1.0, 0.0)}),
    ("cylindrical phi short of 2 pi", "cyl", [8, 8, 8], {"hi": (10.0, 1.0, 6.0)}),
    ("grid above 2^31 cells", "cart", [4096, 4096, 256], {}),
    ("precision", "cart", [8, 8], {"precision": 9}),
    ("no smoothing", "cart", [8, 8], {"nu1": 0, "nu2": 0}),
    ("negative nu1", "cart", [8, 8], {"nu1": -1}),
    ("nu2 above 64", "cart", [8, 8], {"nu2": 65}),
    ("negative max_cycles", "cart", [8, 8], {"max_cycles": -1}),
    ("max_cycles beyond the history", "cart", [8, 8], {"max_cycles": 1024}),
    ("negative tol", "cart", [8, 8], {"tol": -1e-10}),
    ("NaN tol", "cart", [8, 8], {"tol": float("nan")}),
    ("mixed-derivative form", "cart", [8, 8], {"mixed_deriv": 5}),
    ("negative stall window", "cart", [8, 8], {"stall_window": -1}),
    ("Anderson depth above 16", "cart", [8, 8], {"accel_depth": 17}),
    ("negative Anderson depth", "cart", [8, 8], {"accel_depth": -1}),
    ("div-B variant", "cart", [8, 8], {"divb_variant": 2}),
    ("exact projection on a spherical grid", "sph", [8, 8], {"divb_variant": 1}),
    ("exact projection with n = 2", "cart", [8, 2], {"divb_variant": 1}),
])
def test_descriptor_validation_rejects(what, geom, n, kw):
    """Every rule of the descriptor (grid, domain of the geometry, solver
    settings) answers MG_ERR_INVALID with a message, without a device."""
    from paper_2012_07322_gb300 import mg
    import numpy as np
    nd = len(n)
    lo = {"cart": [-1.0] * nd, "cyl": [0.0, -1.0, 0.0][:nd], "sph": [0.0] * nd}[geom]
    hi = {"cart": [1.0] * nd, "cyl": [10.0, 1.0, 2 * np.pi][:nd], "sph": [10.0, np.pi, 2 * np.pi][:nd]}[geom]
    d = _set(mg.grid_desc(geom, [max(x, 1) for x in n], lo=lo, hi=hi), **kw)
    for k in range(nd):
        d.n[k] = n[k]
    with pytest.raises(mg.MgError) as e:
        mg.mg_hierarchy_bytes(d)
    assert e.value.status == mg.MG_ERR_INVALID, what
    assert mg.lib().mg_last_error(), what


@pytest.mark.parametrize("geom,n", [
    ("cart", [2, 2]), ("cart", [2, 2, 2]), ("sph", [2, 2]), ("cyl", [2, 2, 2]),
    ("sph", [1024, 2]), ("cart", [4, 4096]),
])
def test_degenerate_but_valid_grids(geom, n):
    """The smallest grids (one level of two cells per direction) and the most
    anisotropic ones are accepted: the hierarchy then has one level, or
    stops halving where the short direction reaches two cells."""
    from paper_2012_07322_gb300 import mg
    import numpy as np
    nd = len(n)
    lo = {"cart": [-1.0] * nd, "cyl": [0.0, -1.0, 0.0][:nd], "sph": [0.0] * nd}[geom]
    hi = {"cart": [1.0] * nd, "cyl": [10.0, 1.0, 2 * np.pi][:nd], "sph": [10.0, np.pi, 2 * np.pi][:nd]}[geom]
    b = mg.mg_hierarchy_bytes(mg.grid_desc(geom, n, lo=lo, hi=hi))
    assert b >= int(np.prod(n)) * 8


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the CUDA library and without a toolkit to
    build it, the binding raises instead of computing anything."""
    from paper_2012_07322_gb300 import build, mg

    def no_nvcc():
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgmunu_mg.so")

    monkeypatch.setattr(mg, "_lib", None)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "libgmunu_mg.so"))
    monkeypatch.setattr(build, "nvcc", no_nvcc)
    with pytest.raises(RuntimeError, match="nvcc not found"):
        mg.lib()
    with pytest.raises(RuntimeError):
        mg.mg_hierarchy_bytes(mg.grid_desc("cart", [8, 8], [-1.0, -1.0], [1.0, 1.0]))


def test_null_arguments_are_rejected_without_a_device():
    """Every entry point checks its pointers before any device work: null
    handles and outputs answer MG_ERR_INVALID (destroying null is a no-op),
    and an invalid descriptor never reaches an allocation."""
    from paper_2012_07322_gb300 import mg
    L = mg.lib()
    INV = mg.MG_ERR_INVALID
    good = mg.grid_desc("sph", [64, 32], hi=[100.0, 3.141592653589793])
    bad = mg.grid_desc("sph", [64, 24], hi=[100.0, 3.141592653589793])
    out = ctypes.c_void_p()
    assert L.mg_create_hierarchy(None, None, ctypes.byref(out)) == INV
    assert L.mg_create_hierarchy(ctypes.byref(bad), None, ctypes.byref(out)) == INV and not out.value
    assert L.mg_create_hierarchy(ctypes.byref(good), None, None) == INV
    assert L.mg_hierarchy_bytes(ctypes.byref(good), None) == INV
    assert L.mg_hierarchy_bytes(None, ctypes.byref(ctypes.c_size_t())) == INV
    assert L.mg_destroy_hierarchy(None) == mg.MG_OK
    assert L.mg_num_levels(None, None) == INV
    assert L.mg_solve_cfc(None, None, None, 0, None) == INV
    assert L.mg_clean_divB(None, None, None, 0, None) == INV
    assert L.mg_solve_scalar(None, 0, 0, 0, None, None, None, None, None, None) == INV
    assert L.mg_solve_vector(None, 0, None, None, None) == INV
    assert L.mg_apply_operator(None, 0, 0, None, None, None, None, None) == INV
    assert L.mg_smooth(None, 0, 0, 1, None, None, None, None, None) == INV
    assert L.mg_compute_a2(None, None, None) == INV
    assert L.mg_divergence(None, None, None) == INV
    assert L.mg_restrict(None, None, None) == INV
    assert L.mg_prolong_add(None, 0, None, None) == INV
    assert L.mg_profile_enable(None, 1) == INV
    assert L.mg_profile_read(None, 0, None, None, None) == INV
    srv = ctypes.c_void_p()
    assert L.mg_server_create(0, 4, 8, ctypes.byref(srv)) == INV and not srv.value
    assert L.mg_server_create(1 << 30, 0, 8, ctypes.byref(srv)) == INV
    assert L.mg_server_create(1 << 30, 4, 8, None) == INV
    assert L.mg_server_destroy(None) == mg.MG_OK
    ticket = ctypes.c_uint64()
    assert L.mg_submit(None, None, ctypes.byref(ticket)) == INV
    done = ctypes.c_int()
    assert L.mg_poll(None, 0, ctypes.byref(done), None) == INV
    # batched solves: null arrays, an empty batch, host pointers, a cluster
    # of 3 blocks and a null hierarchy are refused before any device work
    hs = (ctypes.c_void_p * 1)(None)
    srcs, ios = (mg.mg_cfc_sources * 1)(), (mg.mg_cfc_fields * 1)()
    assert L.mg_solve_cfc_batch(None, 1, srcs, ios, 0, None, None, None) == INV
    assert L.mg_solve_cfc_batch(hs, 0, srcs, ios, 0, None, None, None) == INV
    assert L.mg_solve_cfc_batch(hs, 1, srcs, ios, mg.MG_HOST_POINTERS, None, None, None) == INV
    assert L.mg_solve_cfc_batch(hs, 1, srcs, ios, 0, ctypes.byref(mg.mg_batch_opts(3, 0)), None, None) == INV
    assert L.mg_solve_cfc_batch(hs, 1, srcs, ios, 0, None, None, None) == INV
    assert L.mg_last_error()
