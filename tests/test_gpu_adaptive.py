"""GPU parity of the adaptive Krylov dimension (the a-posteriori exit of
Algorithm 6, ed_set_krylov_tol) against the oracle's adaptive steps.

complex128: the same float64 decisions on both sides, so the dimension used
in every step is identical and the trajectories agree to rounding (1e-10).
complex64: Lanczos scalars carry float32 rounding of the vectors, so a step
whose epsilon lands within rounding of the tolerance may exit one step
earlier or later; <d> within 1e-5 and the dimensions within one.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import LATTICES, torch_cuda, to_dev, from_dev, rel_l2, ed_dtype

pytestmark = pytest.mark.gpu


def run(ed, torch, lat, nu, nd, U, psi0, pulse, dt, n, m, dtype, tol, energy=False):
    h = ed.Hubbard(lat, nu, nd, U)
    ed.ed_set_krylov_tol(h.ctx, tol)
    xd = to_dev(torch, psi0, dtype)
    out = ed.ed_propagate(h.ctx, xd, ed_dtype(ed, dtype), pulse, 0.0, dt, n, m,
                          energy=energy)
    torch.cuda.synchronize()
    psi = from_dev(xd)
    h.close()
    return psi, out


def torus_case():
    lat = LATTICES["torus3x4"]
    pulse = dict(synth.workload("torus3x4")["pulse_params"], t0=0.1)
    psi0 = synth.complex_normal(924 * 792, 13)
    return lat, pulse, psi0


def test_torus_adaptive_c128_matches_oracle(ed_lib, parity_log):
    torch = torch_cuda()
    lat, pulse, psi0 = torus_case()
    ref = oracle.propagate(lat, 6, 5, 8.0, psi0, pulse, 0.02, 10, 24, eps_tol=1e-8,
                           with_energy=True)
    psi, out = run(ed_lib, torch, lat, 6, 5, 8.0, psi0, pulse, 0.02, 10, 24, "c128", 1e-8,
                   energy=True)
    parity_log("torus_adaptive_c128", state_rel_l2=rel_l2(psi, ref["psi"]),
               docc_max_err=np.abs(out["docc"] - ref["docc"]).max())
    assert list(out["m_eff"]) == list(ref["m_eff"])
    assert max(ref["m_eff"]) < 24          # the exit is really taken
    assert rel_l2(psi, ref["psi"]) <= 1e-10
    assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-10
    assert np.abs(out["energy"] - ref["energy"]).max() <= 1e-10


def test_torus_adaptive_c64_close_to_oracle(ed_lib, parity_log):
    torch = torch_cuda()
    lat, pulse, psi0 = torus_case()
    ref = oracle.propagate(lat, 6, 5, 8.0, psi0, pulse, 0.02, 10, 24, eps_tol=1e-6)
    psi, out = run(ed_lib, torch, lat, 6, 5, 8.0, psi0, pulse, 0.02, 10, 24, "c64", 1e-6)
    parity_log("torus_adaptive_c64", state_rel_l2=rel_l2(psi, ref["psi"]),
               docc_max_err=np.abs(out["docc"] - ref["docc"]).max(),
               norm_drift=np.abs(out["norm2"] - out["norm2"][0]).max())
    assert np.abs(np.array(out["m_eff"]) - np.array(ref["m_eff"])).max() <= 1
    assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-5
    assert np.abs(out["norm2"] - out["norm2"][0]).max() <= 1e-6
    assert rel_l2(psi, ref["psi"]) <= 1e-4


def test_ring_adaptive_long_trajectory_c128(ed_lib):
    """Ns=8 ring, (4,4), from the ground state through the pulse, 300 steps,
    maximum 16, tolerance 1e-10."""
    torch = torch_cuda()
    w = synth.workload("ring8")
    lat = LATTICES["ring8"]
    E0, psi0, gap = oracle.ground_state(lat, 4, 4, 8.0)
    ref = oracle.propagate(lat, 4, 4, 8.0, psi0, w["pulse_params"], 0.02, 300, 16,
                           eps_tol=1e-10)
    psi, out = run(ed_lib, torch, lat, 4, 4, 8.0, psi0, w["pulse_params"], 0.02, 300, 16,
                   "c128", 1e-10)
    assert list(out["m_eff"]) == list(ref["m_eff"])
    assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-10
    assert rel_l2(psi, ref["psi"]) <= 1e-10


def test_spectral_adaptive_matches_oracle(ed_lib):
    """Ring of 6 sites, (3,3): the batch of c/c+ vectors and psi, each vector
    with its own exit step, against the oracle's adaptive spectral batch."""
    torch = torch_cuda()
    lat = LATTICES["ring6"]
    pulse = {"A0": 0.6, "omega": 5.0, "sigma": 1.0, "t0": 0.3, "dir": (1.0, 0.0, 0.0)}
    E0, psi0, gap = oracle.ground_state(lat, 3, 3, 4.0)
    ref = oracle.spectral_batch(lat, 3, 3, 4.0, psi0, pulse, 0.05, 8, 16, eps_tol=1e-9)
    h = ed_lib.Hubbard(lat, 3, 3, 4.0)
    ed_lib.ed_set_krylov_tol(h.ctx, 1e-9)
    Gl, Gg = ed_lib.ed_spectral_propagate(h.ctx, to_dev(torch, psi0, "c128"), ed_lib.ED_C128,
                                          pulse, 0.05, 8, 16, 6)
    h.close()
    assert np.abs(Gl - ref["G_less"]).max() <= 1e-9
    assert np.abs(Gg - ref["G_greater"]).max() <= 1e-9


def test_spectral_adaptive_multi_vector_configs(ed_lib):
    """The adaptive ring-6 batch with each complex128 multi-vector
    configuration pinned: vectors that share thread blocks exit at their own
    Lanczos step, and the traces match the oracle's adaptive batch."""
    torch = torch_cuda()
    lat = LATTICES["ring6"]
    pulse = {"A0": 0.6, "omega": 5.0, "sigma": 1.0, "t0": 0.3, "dir": (1.0, 0.0, 0.0)}
    E0, psi0, gap = oracle.ground_state(lat, 3, 3, 4.0)
    ref = oracle.spectral_batch(lat, 3, 3, 4.0, psi0, pulse, 0.05, 8, 16, eps_tol=1e-9)
    mv = [c for c in range(ed_lib.ed_apply_config_count())
          if ed_lib.ed_apply_config_info(c)["mv"] and ed_lib.ed_apply_config_info(c)["fp64"]]
    assert mv
    try:
        for cfg in mv:
            ed_lib.ed_set_apply_config(cfg)
            h = ed_lib.Hubbard(lat, 3, 3, 4.0)
            ed_lib.ed_set_krylov_tol(h.ctx, 1e-9)
            Gl, Gg = ed_lib.ed_spectral_propagate(h.ctx, to_dev(torch, psi0, "c128"),
                                                  ed_lib.ED_C128, pulse, 0.05, 8, 16, 6)
            h.close()
            assert np.abs(Gl - ref["G_less"]).max() <= 1e-9, cfg
            assert np.abs(Gg - ref["G_greater"]).max() <= 1e-9, cfg
    finally:
        ed_lib.ed_set_apply_config(-1)
