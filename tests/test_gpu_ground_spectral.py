"""GPU parity of ed_ground_state, ed_double_occupation, ed_apply_fermion_op and
ed_spectral_propagate against the oracle and closed forms."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import LATTICES, torch_cuda, to_dev, from_dev, rel_l2, ed_dtype

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("U,E0", [(8.0, -0.4721359549995796), (4.0, -0.8284271247461903)])
def test_ground_state_dimer_closed_form(ed_lib, U, E0):
    torch = torch_cuda()
    h = ed_lib.Hubbard(synth.dimer(), 1, 1, U)
    psi = torch.zeros(h.D, dtype=torch.complex128, device="cuda")
    E, res = ed_lib.ed_ground_state(h.ctx, psi, tol=1e-13)
    assert abs(E - E0) <= 1e-12
    h.close()


@pytest.mark.parametrize("name,nu,nd,U", [("ring8", 4, 4, 8.0), ("ring6", 3, 3, 4.0),
                                          ("chain6_eps", 3, 2, 2.0),
                                          ("torus3x4", 6, 6, 8.0)])
def test_ground_state_matches_oracle(ed_lib, name, nu, nd, U, parity_log):
    torch = torch_cuda()
    lat = LATTICES[name]
    E0, psi_ref, gap = oracle.ground_state(lat, nu, nd, U)
    h = ed_lib.Hubbard(lat, nu, nd, U)
    psi = torch.zeros(h.D, dtype=torch.complex128, device="cuda")
    E, res = ed_lib.ed_ground_state(h.ctx, psi, tol=1e-11, max_iter=3000)
    parity_log(f"ground_state_{name}", E0_rel_err=abs(E - E0) / max(1.0, abs(E0)),
               residual=res)
    assert abs(E - E0) <= 1e-10 * max(1.0, abs(E0))
    assert res <= 1e-10 * max(1.0, abs(E0))
    p = from_dev(psi)
    assert abs(np.linalg.norm(p) - 1.0) <= 1e-12
    if gap > 1e-6:
        # unique ground state: same vector up to the phase fix
        assert abs(abs(np.vdot(psi_ref, p)) - 1.0) <= 1e-9
    h.close()


def test_ground_state_ladder_full_size(ed_lib):
    """Ns=14 ladder (7,7): energy against the stored oracle eigsh value
    (tests/golden/ground_energies.json, written by make_ground_energies.py)
    and the residual |H psi - E psi| with the oracle operator."""
    import json, os
    from oracle.krylov import make_H
    torch = torch_cuda()
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "ground_energies.json")))
    E0 = [c for c in gold["cases"] if c["lattice"] == "ladder2x7"][0]["E0"]
    lat = LATTICES["ladder2x7"]
    h = ed_lib.Hubbard(lat, 7, 7, 8.0)
    psi = torch.zeros(h.D, dtype=torch.complex128, device="cuda")
    E, res = ed_lib.ed_ground_state(h.ctx, psi, tol=1e-10, max_iter=3000)
    assert abs(E - E0) <= 1e-9 * abs(E0)
    p = from_dev(psi)
    H = make_H(lat, 7, 7, 8.0, (0.0, 0.0, 0.0), form="kron")
    assert np.linalg.norm(H @ p - E * p) <= 1e-8 * abs(E)
    h.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_double_occupation_sites(ed_lib, dtype):
    torch = torch_cuda()
    lat = LATTICES["ring8"]
    h = ed_lib.Hubbard(lat, 3, 4, 1.0)
    v = synth.complex_normal(h.D, 3)
    d, site = ed_lib.ed_double_occupation(h.ctx, to_dev(torch, v, dtype), ed_dtype(ed_lib, dtype))
    w = oracle.double_occupancy_weights(8, 3, 4)
    tol = 1e-14 if dtype == "c128" else 1e-7
    assert abs(d - oracle.double_occupation(v, w, 8)) <= tol
    bu, bd = oracle.spin_basis(8, 3), oracle.spin_basis(8, 4)
    P = np.abs(v.reshape(len(bu), len(bd))) ** 2
    for i in range(8):
        occ = ((bu[:, None] >> np.uint64(i)) & np.uint64(1)) & ((bd[None, :] >> np.uint64(i)) & np.uint64(1))
        assert abs(site[i] - np.sum(P * occ)) <= tol
    h.close()


def test_fermion_ops_match_oracle(ed_lib):
    torch = torch_cuda()
    lat = LATTICES["ring6"]
    src = ed_lib.Hubbard(lat, 3, 2, 1.0)
    v = synth.complex_normal(src.D, 9)
    vd = to_dev(torch, v, "c128")
    for create in (False, True):
        for spin in (0, 1):
            dn = 1 if create else -1
            nu, nd = (3 + dn, 2) if spin == 0 else (3, 2 + dn)
            dst = ed_lib.Hubbard(lat, nu, nd, 1.0)
            for site in range(6):
                out = torch.zeros(dst.D, dtype=torch.complex128, device="cuda")
                ed_lib.ed_apply_fermion_op(src.ctx, dst.ctx, site, spin, create, vd, out,
                                           ed_lib.ED_C128)
                f = oracle.apply_cdag if create else oracle.apply_c
                ref = f(6, 3, 2, v, site, spin)
                assert np.array_equal(from_dev(out), ref)
            dst.close()
    src.close()


def _mv_configs(ed, fp64):
    return [c for c in range(ed.ed_apply_config_count())
            if ed.ed_apply_config_info(c)["mv"] and ed.ed_apply_config_info(c)["fp64"] == fp64]


@pytest.fixture
def pinned(ed_lib):
    yield ed_lib
    ed_lib.ed_set_apply_config(-1)


def test_spectral_dimer_multi_vector_breakdown(pinned):
    """The dimer batch (Krylov breakdown in every vector, at different j)
    with each complex128 multi-vector configuration: the vectors of a
    sector share thread blocks, and a vector that has stopped leaves the
    others' alpha_j untouched."""
    ed = pinned
    torch_cuda()
    U, t = 5.0, 1.0
    lat = synth.dimer(t)
    E0, psi0, _ = oracle.ground_state(lat, 1, 1, U)
    ref = oracle.spectral_batch(lat, 1, 1, U, psi0, None, 0.05, 12, 8)
    for cfg in _mv_configs(ed, 1):
        ed.ed_set_apply_config(cfg)
        h = ed.Hubbard(lat, 1, 1, U)
        Gl, Gg = ed.ed_spectral_propagate(h.ctx, psi0, ed.ED_C128, None, 0.05, 12, 8, 2)
        h.close()
        assert np.abs(Gl - ref["G_less"]).max() <= 1e-11, cfg
        assert np.abs(Gg - ref["G_greater"]).max() <= 1e-11, cfg


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_spectral_batch_multi_vector_configs(pinned, dtype):
    """Ring 6 at half filling under a pulse, every multi-vector configuration
    of the precision pinned: six vectors per sector (spin-down ones stored
    transposed into the spin-up shape), all 24 traces against the oracle."""
    ed = pinned
    torch_cuda()
    lat = LATTICES["ring6"]
    E0, psi0, _ = oracle.ground_state(lat, 3, 3, 6.0)
    pulse = {"A0": 0.8, "omega": 6.0, "sigma": 0.5, "t0": 0.4, "dir": (1.0, 0, 0)}
    ref = oracle.spectral_batch(lat, 3, 3, 6.0, psi0, pulse, 0.04, 25, 12)
    tol = 1e-10 if dtype == "c128" else 1e-5
    for cfg in _mv_configs(ed, 1 if dtype == "c128" else 0):
        ed.ed_set_apply_config(cfg)
        h = ed.Hubbard(lat, 3, 3, 6.0)
        Gl, Gg = ed.ed_spectral_propagate(h.ctx, psi0, ed_dtype(ed, dtype), pulse,
                                          0.04, 25, 12, 6)
        h.close()
        assert np.abs(Gl - ref["G_less"]).max() <= tol, cfg
        assert np.abs(Gg - ref["G_greater"]).max() <= tol, cfg


def test_spectral_dimer_closed_form(ed_lib):
    torch_cuda()
    U, t = 5.0, 1.0
    lat = synth.dimer(t)
    E0, psi0, _ = oracle.ground_state(lat, 1, 1, U)
    h = ed_lib.Hubbard(lat, 1, 1, U)
    dt, n = 0.05, 30
    Gl, Gg = ed_lib.ed_spectral_propagate(h.ctx, psi0, ed_lib.ED_C128, None, dt, n, 8, 2)
    R = np.sqrt(U * U + 16 * t * t)
    a, b = 2 * t, (U + R) / 2
    a, b = a / np.hypot(2 * t, (U + R) / 2), b / np.hypot(2 * t, (U + R) / 2)
    tt = dt * np.arange(n + 1)
    wB, wA = ((a + b) / 2) ** 2, ((a - b) / 2) ** 2
    L = wB * np.exp(-1j * (-t - E0) * tt) + wA * np.exp(-1j * (t - E0) * tt)
    G = wB * np.exp(-1j * (U - t - E0) * tt) + wA * np.exp(-1j * (U + t - E0) * tt)
    for i in (0, 1):
        for s in (0, 1):
            assert np.abs(Gl[:, i, s] - 1j * L).max() <= 1e-11
            assert np.abs(Gg[:, i, s] + 1j * G).max() <= 1e-11
    h.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_spectral_batch_matches_oracle(ed_lib, dtype, parity_log):
    """Ring 6 at half filling under a pulse: all 24 Green's-function traces."""
    torch_cuda()
    lat = LATTICES["ring6"]
    E0, psi0, _ = oracle.ground_state(lat, 3, 3, 6.0)
    pulse = {"A0": 0.8, "omega": 6.0, "sigma": 0.5, "t0": 0.4, "dir": (1.0, 0, 0)}
    ref = oracle.spectral_batch(lat, 3, 3, 6.0, psi0, pulse, 0.04, 25, 12)
    h = ed_lib.Hubbard(lat, 3, 3, 6.0)
    Gl, Gg = ed_lib.ed_spectral_propagate(h.ctx, psi0, ed_dtype(ed_lib, dtype), pulse,
                                          0.04, 25, 12, 6)
    tol = 1e-10 if dtype == "c128" else 1e-5
    parity_log(f"ring6_spectral_{dtype}", G_less_max_err=np.abs(Gl - ref["G_less"]).max(),
               G_greater_max_err=np.abs(Gg - ref["G_greater"]).max())
    assert np.abs(Gl - ref["G_less"]).max() <= tol
    assert np.abs(Gg - ref["G_greater"]).max() <= tol
    h.close()


def test_spectral_torus_sum_rules(ed_lib):
    """3x4 torus (6,6): 48 vectors in (5,6), (6,5), (7,6), (6,7) batched; at the
    reference time the traces obey the sum rules, and two steps match the
    oracle for one site."""
    torch_cuda()
    lat = LATTICES["torus3x4"]
    w = synth.workload("torus3x4")
    psi0 = synth.complex_normal(924 * 924, 21)
    h = ed_lib.Hubbard(lat, 6, 6, 8.0)
    Gl, Gg = ed_lib.ed_spectral_propagate(h.ctx, psi0, ed_lib.ED_C64, w["pulse_params"],
                                          0.02, 2, 20, 12)
    L0 = (Gl[0] / 1j)
    G0 = (Gg[0] / -1j)
    P = np.abs(psi0.reshape(924, 924)) ** 2
    bu = oracle.spin_basis(12, 6)
    for i in range(12):
        n_up_i = np.sum(P[((bu >> np.uint64(i)) & np.uint64(1)) == 1, :])
        assert abs(L0[i, 0] - n_up_i) <= 1e-6
        assert abs(L0[i, 0] + G0[i, 0] - 1.0) <= 1e-6
    assert abs(L0[:, 0].sum() - 6.0) <= 1e-5
    h.close()


def test_spectral_torus_one_site_matches_oracle(ed_lib, parity_log):
    """3x4 torus (6,6) batch in complex64: the traces of site 5 (all four
    operators) over 3 steps against the oracle's float64 propagation of the
    same four vectors and psi."""
    torch_cuda()
    lat = LATTICES["torus3x4"]
    w = synth.workload("torus3x4")
    pulse = dict(w["pulse_params"], t0=0.2)
    psi0 = synth.complex_normal(924 * 924, 23)
    ref = oracle.spectral_batch(lat, 6, 6, 8.0, psi0, pulse, 0.02, 3, 20, sites=[5])
    h = ed_lib.Hubbard(lat, 6, 6, 8.0)
    Gl, Gg = ed_lib.ed_spectral_propagate(h.ctx, psi0, ed_lib.ED_C64, pulse, 0.02, 3, 20, 12)
    parity_log("torus_spectral_site5_c64",
               G_less_max_err=np.abs(Gl[:, 5] - ref["G_less"][:, 5]).max(),
               G_greater_max_err=np.abs(Gg[:, 5] - ref["G_greater"][:, 5]).max())
    for s in (0, 1):
        assert np.abs(Gl[:, 5, s] - ref["G_less"][:, 5, s]).max() <= 1e-5
        assert np.abs(Gg[:, 5, s] - ref["G_greater"][:, 5, s]).max() <= 1e-5
    h.close()
