"""Degenerate inputs of the propagation path against the oracle: the zero
state, Krylov dimension 1, one-element sectors (all sites empty / full, one
spin species absent), and a batched apply whose row blocks leave a ragged
last block.  Tolerances as in the other parity tests."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (LATTICES, torch_cuda, to_dev, from_dev, rel_l2, ed_dtype, max_el,
                      TOL_EL)
from oracle.krylov import make_H

pytestmark = pytest.mark.gpu

PULSE = {"A0": 0.7, "omega": 4.0, "sigma": 1.0, "t0": 0.3, "dir": (1.0, 0.0, 0.0)}


def run(ed, torch, lat, nu, nd, U, psi0, n, m, dt=0.05, dtype="c128"):
    h = ed.Hubbard(lat, nu, nd, U)
    x = to_dev(torch, psi0, dtype)
    out = ed.ed_propagate(h.ctx, x, ed_dtype(ed, dtype), PULSE, 0.0, dt, n, m)
    torch.cuda.synchronize()
    psi = from_dev(x)
    h.close()
    return psi, out


def test_zero_state_stays_zero(ed_lib):
    torch = torch_cuda()
    lat = LATTICES["ring6"]
    D = oracle.sector_dims(6, 3, 2)[2]
    psi, out = run(ed_lib, torch, lat, 3, 2, 4.0, np.zeros(D, complex), 5, 8)
    assert np.abs(psi).max() == 0.0
    assert np.abs(out["norm2"]).max() == 0.0 and np.abs(out["docc"]).max() == 0.0


def test_krylov_dimension_one_is_a_phase(ed_lib):
    """m = 1: psi <- exp(-i tau <v|H|v>) psi each step (Algorithm 6 with one
    vector), against the oracle."""
    torch = torch_cuda()
    lat = LATTICES["ring6"]
    psi0 = synth.complex_normal(oracle.sector_dims(6, 3, 3)[2], 2)
    ref = oracle.propagate(lat, 3, 3, 4.0, psi0, PULSE, 0.05, 6, 1)
    psi, out = run(ed_lib, torch, lat, 3, 3, 4.0, psi0, 6, 1)
    assert rel_l2(psi, ref["psi"]) <= 1e-12
    assert list(out["m_eff"]) == [1] * 6
    assert np.abs(out["norm2"] - 1.0).max() <= 1e-12


@pytest.mark.parametrize("nu,nd", [(0, 0), (6, 6), (0, 3), (6, 2)])
def test_one_element_and_single_species_sectors(ed_lib, nu, nd):
    """(0,0) and (6,6) have one basis state (H is the diagonal U n_d);
    (0,3) and (6,2) have a single spin species hopping."""
    torch = torch_cuda()
    lat = LATTICES["ring6"]
    D = oracle.sector_dims(6, nu, nd)[2]
    psi0 = synth.complex_normal(D, 4)
    ref = oracle.propagate(lat, nu, nd, 3.0, psi0, PULSE, 0.05, 5, 6)
    psi, out = run(ed_lib, torch, lat, nu, nd, 3.0, psi0, 5, 6)
    assert rel_l2(psi, ref["psi"]) <= 1e-12
    assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-12
    if D == 1:
        # exact: a pure phase exp(-i U n_d t)
        nd_ = 6 if nu == 6 else 0
        exact = psi0 * np.exp(-1j * 3.0 * nd_ * 0.25)
        assert np.abs(psi - exact).max() <= 1e-13


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batched_apply_ragged_row_blocks(ed_lib, dtype):
    """Three vectors in one call on the 11-site ring: (3,4) has dim_up = 165
    (odd: the last block of 2 or 4 rows holds one row) and dim_dn = 330
    (2 mod 4 columns); (4,3) the transpose shapes."""
    torch = torch_cuda()
    ed = ed_lib
    lat = synth.ring(11)
    for nu, nd in ((3, 4), (4, 3)):
        h = ed.Hubbard(lat, nu, nd, 6.0)
        A = np.array([0.2, -0.4, 0.0])
        ed.ed_set_field(h.ctx, A)
        v = synth.random_state(h.dim_up, h.dim_dn, seed=9, nvec=3).reshape(3, -1)
        H = make_H(lat, nu, nd, 6.0, A)
        ref = np.stack([H @ v[b] for b in range(3)])
        vd = to_dev(torch, v, dtype)
        wd = torch.zeros_like(vd)
        ed.ed_apply_H(h.ctx, vd, wd, ed_dtype(ed, dtype), nvec=3)
        torch.cuda.synchronize()
        tol = 1e-13 if dtype == "c128" else 3e-6
        assert rel_l2(from_dev(wd), ref) <= tol
        assert max_el(from_dev(wd), ref) <= TOL_EL[dtype]
        h.close()
