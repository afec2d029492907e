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
    bad = mg.grid_desc("sph", [64, 32], hi=[100.0, np.pi])
    bad.cycle = 7                                                     # neither V nor FMG
    with pytest.raises(mg.MgError):
        mg.mg_hierarchy_bytes(bad)
    assert mg.lib().mg_strerror(3) == b"not converged"
