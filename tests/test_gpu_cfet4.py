"""GPU parity of the fourth-order commutator-free integrator (CFET4,
ed_set_integrator) against the oracle's CFET4 steps: two Krylov steps per
time step on the combined Hamiltonians a2 H1 + a1 H2 and a1 H1 + a2 H2 at
the Gauss nodes.  Tolerances as for the midpoint rule: complex128 1e-10
(same arithmetic up to rounding), complex64 <d> 1e-5.
"""
import functools

import numpy as np
import pytest

import oracle
import synth
from gpu_util import LATTICES, torch_cuda, to_dev, from_dev, rel_l2, ed_dtype

pytestmark = pytest.mark.gpu


def run(ed, torch, lat, nu, nd, U, psi0, pulse, dt, n, m, dtype, energy=False, tol=0.0):
    h = ed.Hubbard(lat, nu, nd, U)
    ed.ed_set_integrator(h.ctx, ed.ED_CFET4)
    ed.ed_set_krylov_tol(h.ctx, tol)
    xd = to_dev(torch, psi0, dtype)
    out = ed.ed_propagate(h.ctx, xd, ed_dtype(ed, dtype), pulse, 0.0, dt, n, m, energy=energy)
    torch.cuda.synchronize()
    psi = from_dev(xd)
    h.close()
    return psi, out


def torus_case():
    lat = LATTICES["torus3x4"]
    pulse = dict(synth.workload("torus3x4")["pulse_params"], t0=0.2)
    psi0 = synth.complex_normal(924 * 792, 17)
    return lat, pulse, psi0


@functools.lru_cache(maxsize=1)
def torus_reference():
    lat, pulse, psi0 = torus_case()
    return oracle.propagate(lat, 6, 5, 8.0, psi0, pulse, 0.05, 8, 20, with_energy=True,
                            scheme="cfet4")


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_torus_cfet4_matches_oracle(ed_lib, dtype, parity_log):
    torch = torch_cuda()
    lat, pulse, psi0 = torus_case()
    ref = torus_reference()
    psi, out = run(ed_lib, torch, lat, 6, 5, 8.0, psi0, pulse, 0.05, 8, 20, dtype,
                   energy=True)
    assert len(out["docc"]) == 9 and len(out["m_eff"]) == 8
    parity_log(f"torus_cfet4_{dtype}", state_rel_l2=rel_l2(psi, ref["psi"]),
               docc_max_err=np.abs(out["docc"] - ref["docc"]).max(),
               energy_max_err=np.abs(out["energy"] - ref["energy"]).max())
    if dtype == "c128":
        assert rel_l2(psi, ref["psi"]) <= 1e-10
        assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-10
        assert np.abs(out["energy"] - ref["energy"]).max() <= 1e-10
        assert list(out["m_eff"]) == list(ref["m_eff"])
    else:
        assert rel_l2(psi, ref["psi"]) <= 1e-4
        assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-5
        assert np.abs(out["energy"] - ref["energy"]).max() <= 1e-4


def test_ring_cfet4_from_ground_state_c128(ed_lib):
    torch = torch_cuda()
    w = synth.workload("ring8")
    lat = LATTICES["ring8"]
    E0, psi0, gap = oracle.ground_state(lat, 4, 4, 8.0)
    ref = oracle.propagate(lat, 4, 4, 8.0, psi0, w["pulse_params"], 0.05, 200, 16,
                           scheme="cfet4")
    psi, out = run(ed_lib, torch, lat, 4, 4, 8.0, psi0, w["pulse_params"], 0.05, 200, 16,
                   "c128")
    assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-10
    assert rel_l2(psi, ref["psi"]) <= 1e-10
    assert np.ptp(ref["docc"]) > 1e-3


def test_cfet4_with_adaptive_exit_c128(ed_lib):
    torch = torch_cuda()
    lat, pulse, psi0 = torus_case()
    ref = oracle.propagate(lat, 6, 5, 8.0, psi0, pulse, 0.05, 6, 24, scheme="cfet4",
                           eps_tol=1e-9)
    psi, out = run(ed_lib, torch, lat, 6, 5, 8.0, psi0, pulse, 0.05, 6, 24, "c128", tol=1e-9)
    assert list(out["m_eff"]) == list(ref["m_eff"])
    assert max(ref["m_eff"]) < 24
    assert rel_l2(psi, ref["psi"]) <= 1e-10


def test_spectral_cfet4_matches_oracle(ed_lib):
    torch = torch_cuda()
    lat = LATTICES["ring6"]
    pulse = {"A0": 0.6, "omega": 5.0, "sigma": 1.0, "t0": 0.3, "dir": (1.0, 0.0, 0.0)}
    E0, psi0, gap = oracle.ground_state(lat, 3, 3, 4.0)
    ref = oracle.spectral_batch(lat, 3, 3, 4.0, psi0, pulse, 0.1, 6, 16, scheme="cfet4")
    h = ed_lib.Hubbard(lat, 3, 3, 4.0)
    ed_lib.ed_set_integrator(h.ctx, "cfet4")
    Gl, Gg = ed_lib.ed_spectral_propagate(h.ctx, to_dev(torch, psi0, "c128"), ed_lib.ED_C128,
                                          pulse, 0.1, 6, 16, 6)
    h.close()
    assert Gl.shape == (7, 6, 2)
    assert np.abs(Gl - ref["G_less"]).max() <= 1e-9
    assert np.abs(Gg - ref["G_greater"]).max() <= 1e-9
