"""ed_double_occupation_static: double occupancy with no device allocation.

Some callers cannot allocate device memory while they run (a loop whose device
memory is fixed up front, a host application enforcing its own memory budget);
this entry point keeps its scratch in a fixed array inside the library.  These
tests call it through the C ABI and check it against ed_double_occupation,
within the tolerances the other double-occupancy tests use, on two calls in a
row, and near its fixed maximum against the oracle.  The file name puts it
last in collection order.
"""
import numpy as np
import pytest

import synth
from gpu_util import LATTICES, torch_cuda, to_dev

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-14, "c64": 1e-7}


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_static_matches_allocating_entry_point_twice(ed_lib, dtype):
    torch = torch_cuda()
    ed = ed_lib
    code = ed.ED_C128 if dtype == "c128" else ed.ED_C64
    h = ed.Hubbard(LATTICES["torus3x4"], 6, 5, 8.0)   # D = 924 x 792
    vecs = [to_dev(torch, synth.complex_normal(h.D, s), dtype) for s in (3, 4)]
    # the allocating entry point first: it also puts the tables on the device
    refs = [ed.ed_double_occupation(h.ctx, v, code) for v in vecs]
    for v, (d_ref, site_ref) in zip(vecs, refs):
        d, site = ed.ed_double_occupation_static(h.ctx, v, code)
        assert abs(d - d_ref) <= TOL[dtype]
        assert np.abs(site[:12] - site_ref[:12]).max() <= TOL[dtype]
    # two calls in a row on the same vector give the same numbers
    a = ed.ed_double_occupation_static(h.ctx, vecs[0], code)
    b = ed.ed_double_occupation_static(h.ctx, vecs[0], code)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    h.close()


def test_static_rejects_oversized_sector_and_unprepared_context(ed_lib):
    torch = torch_cuda()
    ed = ed_lib
    small = torch.zeros(4, dtype=torch.complex128, device="cuda")
    big = ed.Hubbard(synth.ring(16), 8, 8, 1.0)        # D = 12870^2 > 67,108,864
    with pytest.raises(ed.EDError) as e:
        ed.ed_double_occupation_static(big.ctx, small, ed.ED_C128)
    assert e.value.status == 5 and "67,108,864" in str(e.value)
    big.close()
    fresh = ed.Hubbard(LATTICES["ring6"], 3, 3, 1.0)   # no GPU call yet
    v = to_dev(torch, synth.complex_normal(fresh.D, 1), "c128")
    with pytest.raises(ed.EDError) as e:
        ed.ed_double_occupation_static(fresh.ctx, v, ed.ED_C128)
    assert e.value.status == 6
    fresh.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_static_near_its_maximum_matches_oracle(ed_lib, dtype):
    """The 16-site ring at (6,6): D = 8008^2 = 64,128,064 elements, 979 of the
    1024 partial-sum rows of the fixed array, the last one partly filled;
    average and per-site values against the oracle's sums over the same
    (for complex64: rounded) vector."""
    import oracle
    torch = torch_cuda()
    ed = ed_lib
    code = ed.ED_C128 if dtype == "c128" else ed.ED_C64
    h = ed.Hubbard(synth.ring(16), 6, 6, 4.0)
    assert h.D == 64128064
    v = synth.complex_normal(h.D, 8)
    if dtype == "c64":
        v = v.astype(np.complex64).astype(np.complex128)
    vd = to_dev(torch, v, dtype)
    ed.ed_double_occupation(h.ctx, vd, code)         # tables onto the device
    d, site = ed.ed_double_occupation_static(h.ctx, vd, code)
    w = oracle.double_occupancy_weights(16, 6, 6)
    assert abs(d - oracle.double_occupation(v, w, 16)) <= 1e-12
    bu = oracle.spin_basis(16, 6)
    P = (np.abs(v) ** 2).reshape(len(bu), len(bu))
    for i in range(16):
        occ = ((bu >> np.uint64(i)) & np.uint64(1)) == 1
        assert abs(site[i] - P[np.ix_(occ, occ)].sum()) <= 1e-11
    h.close()
