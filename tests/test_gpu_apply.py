"""GPU parity of ed_apply_H against the oracle's H(A) v (element by element).

Tolerances: complex128 relative L2 <= 1e-13 (rounding of a sum of at most
~2 Ns + 1 terms); complex64 relative L2 <= 3e-6 (float32 rounding of the
same sums, ~sqrt(#terms) * 6e-8, with margin).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (LATTICES, torch_cuda, to_dev, from_dev, rel_l2, ed_dtype, max_el,
                      TOL_EL)
from oracle.krylov import make_H

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-13, "c64": 3e-6}

CASES = [
    ("ring8", 4, 4, 8.0), ("ring8", 3, 5, 8.0), ("triangle", 2, 1, 1.5),
    ("dimer", 1, 1, 4.0), ("chain6_eps", 3, 2, 2.0), ("complete7", 3, 4, 1.3),
    ("torus3x4", 6, 6, 8.0), ("torus3x4", 5, 6, 8.0), ("torus3x4", 7, 6, 8.0),
    ("ring6", 0, 3, 2.0), ("ring6", 6, 6, 2.0), ("ring6", 1, 0, 0.0),
]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("name,nu,nd,U", CASES,
                         ids=[f"{c[0]}-{c[1]}{c[2]}" for c in CASES])
def test_apply_matches_oracle(ed_lib, dtype, name, nu, nd, U):
    torch = torch_cuda()
    ed = ed_lib
    lat = LATTICES[name]
    A = np.array([0.37, -0.21, 0.0])
    h = ed.Hubbard(lat, nu, nd, U)
    ed.ed_set_field(h.ctx, A)
    v = synth.random_state(h.dim_up, h.dim_dn, seed=3, nvec=2).reshape(2, -1)
    H = make_H(lat, nu, nd, U, A)
    ref = np.stack([H @ v[0], H @ v[1]])
    vd = to_dev(torch, v, dtype)
    wd = torch.zeros_like(vd)
    ed.ed_apply_H(h.ctx, vd, wd, ed_dtype(ed, dtype), nvec=2)
    torch.cuda.synchronize()
    w = from_dev(wd)
    assert rel_l2(w, ref) <= TOL[dtype]
    assert max_el(w, ref) <= TOL_EL[dtype]
    h.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_apply_full_size_ladder(ed_lib, dtype, parity_log):
    """Ns = 14 ladder, (7,7), D = 11,778,624: the configuration the step bench
    runs, compared on every element."""
    torch = torch_cuda()
    ed = ed_lib
    lat = LATTICES["ladder2x7"]
    h = ed.Hubbard(lat, 7, 7, 8.0)
    A = np.array([0.25, 0.0, 0.0])
    ed.ed_set_field(h.ctx, A)
    v = synth.complex_normal(h.D, 0)
    ref = make_H(lat, 7, 7, 8.0, A, form="kron") @ v
    vd = to_dev(torch, v, dtype)
    wd = torch.zeros_like(vd)
    ed.ed_apply_H(h.ctx, vd, wd, ed_dtype(ed, dtype))
    torch.cuda.synchronize()
    w = from_dev(wd)
    assert rel_l2(w, ref) <= TOL[dtype]
    assert max_el(w, ref) <= TOL_EL[dtype]
    parity_log(f"apply_ladder_full_{dtype}", rel_l2=rel_l2(w, ref), max_el=max_el(w, ref))
    h.close()


def test_apply_long_rows_ns16(ed_lib):
    """Rows longer than one block chunk (dim_dn = 4368 for Ns=16, n_dn=5)."""
    torch = torch_cuda()
    ed = ed_lib
    lat = LATTICES["ring16"]
    h = ed.Hubbard(lat, 2, 5, 3.0)
    A = np.array([0.5, 0.0, 0.0])
    ed.ed_set_field(h.ctx, A)
    v = synth.complex_normal(h.D, 4)
    ref = make_H(lat, 2, 5, 3.0, A, form="kron") @ v
    for dtype in ("c128", "c64"):
        vd = to_dev(torch, v, dtype)
        wd = torch.zeros_like(vd)
        ed.ed_apply_H(h.ctx, vd, wd, ed_dtype(ed, dtype))
        torch.cuda.synchronize()
        assert rel_l2(from_dev(wd), ref) <= TOL[dtype]
        assert max_el(from_dev(wd), ref) <= TOL_EL[dtype]
    h.close()


def test_apply_rejects_host_pointer(ed_lib):
    ed = ed_lib
    torch_cuda()
    h = ed.Hubbard(LATTICES["ring6"], 3, 3, 1.0)
    v = np.zeros(h.D, dtype=np.complex128)
    w = np.zeros(h.D, dtype=np.complex128)
    with pytest.raises(ed.EDError):
        ed.ed_apply_H(h.ctx, v, w, ed.ED_C128)
    h.close()
