"""The allocation-free divergence diagnostic (mg_divb_norms_noalloc).

It serves callers that cannot allocate device memory (a host framework that
owns all device memory, or code that must not let cudaMalloc synchronise
the device): it keeps its scratch in a static device array instead of a
hierarchy.  Its max |div B| and |div B|_2 must equal the before-cleaning
numbers the allocating entry point mg_clean_divB reports for the same field,
on two calls in a row (the scratch keeps the previous call's contents), and
the norms of the oracle's central divergence.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle.oracle as o
from paper_2012_07322_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_07322_gb300 import mg as m
    m.lib()
    return m


def _reference_norms(mg, B, lo, hi):
    """Before-cleaning norms from the allocating entry point."""
    nd = len(B)
    n = [B[0].shape[nd - 1 - d] for d in range(nd)]
    h = mg.Hierarchy(mg.grid_desc("cart", n, lo, hi, tol=1e-8, max_cycles=200))
    rep = mg.mg_clean_divB(h, [b.clone() for b in B])
    h.close()
    return rep["max_div_before"], rep["l2_div_before"]


@pytest.mark.parametrize("case", ["cube32", "slab2d"])
def test_noalloc_norms_match_allocating_entry_point(mg, case):
    if case == "cube32":
        B = [torch.from_numpy(b).cuda() for b in inputs.divb_field(n=32, n_modes=16, k_max=6)]
        lo, hi = [-1.0] * 3, [1.0] * 3
    else:
        rng = np.random.default_rng(11)
        B = [torch.from_numpy(rng.standard_normal((32, 64))).cuda() for _ in range(2)]
        lo, hi = [-1.0, -0.5], [1.0, 0.75]
    want_max, want_l2 = _reference_norms(mg, B, lo, hi)
    nd = len(B)
    n = [B[0].shape[nd - 1 - d] for d in range(nd)]
    div = o.div_c(o.desc("cart", n, lo, hi), [np.ascontiguousarray(b.cpu().numpy()) for b in B])
    orc_max, orc_l2 = np.abs(div).max(), np.sqrt(np.mean(div ** 2))
    for call in range(2):
        st, mx, l2 = mg.mg_divb_norms_noalloc(B, lo, hi)
        assert st == mg.MG_OK
        assert abs(mx - want_max) <= 1e-12 * want_max, (call, mx, want_max)
        assert abs(l2 - want_l2) <= 1e-12 * want_l2, (call, l2, want_l2)
        assert abs(mx - orc_max) <= 1e-12 * orc_max, (call, mx, orc_max)
        assert abs(l2 - orc_l2) <= 1e-12 * orc_l2, (call, l2, orc_l2)


def test_noalloc_rejects_grids_beyond_its_scratch(mg):
    """More cells than MG_NOALLOC_MAX_CELLS: refused before any GPU work."""
    n = 1 << 7  # 128^3 = 2097152 cells is the limit; 256 x 128 x 128 is beyond it
    B = [torch.zeros((n, n, 2 * n), dtype=torch.float64, device="cuda") for _ in range(3)]
    st, _, _ = mg.mg_divb_norms_noalloc(B, [-1.0] * 3, [1.0] * 3, allow=(mg.MG_OK, mg.MG_ERR_INVALID))
    assert st == mg.MG_ERR_INVALID
    assert "MG_NOALLOC_MAX_CELLS" in mg.lib().mg_last_error().decode()
