"""Pins of the oracle's Krylov step, midpoint stepping and observables (CPU).

* Dense scipy.linalg.expm on the full sector matrix at Ns <= 6.
* U = 0: the exact midpoint propagator factorises into Slater-determinant
  matrices, entries = n x n minors of the one-electron propagator
  (Cauchy-Binet), independent of the many-body code.
* Atomic limit t = 0: psi_k(t) = exp(-i U w_d[k] t) psi_k(0) exactly, and the
  Lanczos recursion stops at the number of distinct diagonal values.
* A = 0 from the ground state: psi(t) = exp(-i E0 t) psi0; <d> and E
  stationary (the stationarity test of Sec. 3.9).
* Unitarity (norm conservation); <d>(t) invariant under A -> -A on an
  inversion-symmetric lattice; second-order convergence of the exponential
  midpoint rule (Eq. (32)).
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synth
from oracle.krylov import make_H


def rand_vec(D, seed):
    return synth.complex_normal(D, seed)


@pytest.mark.parametrize("lat,sec,tau,m", [
    (synth.ring(6), (3, 3), 0.02, 12),
    (synth.ring(6), (2, 3), 0.1, 20),
    (synth.chain(5, eps=[0.1, 0.0, -0.3, 0.2, 0.0]), (2, 2), 0.05, 16),
    (synth.complete_graph(5, seed=2), (2, 3), 0.02, 20),
])
def test_lanczos_step_equals_dense_expm(lat, sec, tau, m):
    A = (0.3, -0.1, 0.2)
    H = oracle.build_H(lat, *sec, 6.0, A)
    v = rand_vec(H.shape[0], 5) * 1.7
    ref = sla.expm(-1j * tau * H.toarray()) @ v
    out, info = oracle.lanczos_expm(H, v, tau, m)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-12
    assert info["m_eff"] == m


def test_small_expm_e1_equals_dense():
    rng = np.random.default_rng(3)
    a = rng.standard_normal(9) * 3
    b = np.abs(rng.standard_normal(8)) + 0.1
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    y = oracle.small_expm_e1(a, b, 0.37)
    assert np.abs(y - sla.expm(-0.37j * T)[:, 0]).max() < 1e-13


def minors_matrix(u, Ns, n):
    """Many-body propagator on the n-electron spin basis: det of minors of u."""
    basis = oracle.spin_basis(Ns, n)
    occ = [[i for i in range(Ns) if (int(w) >> i) & 1] for w in basis]
    M = np.zeros((len(basis), len(basis)), dtype=complex)
    for a, ra in enumerate(occ):
        for b, cb in enumerate(occ):
            M[a, b] = np.linalg.det(u[np.ix_(ra, cb)]) if n else 1.0
    return M


@pytest.mark.parametrize("lat,sec", [(synth.ring(6), (3, 2)),
                                     (synth.ladder(3), (3, 3)),
                                     (synth.triangle(), (2, 1))])
def test_free_fermion_midpoint_propagation_is_slater(lat, sec):
    pulse = {"A0": 0.9, "omega": 5.0, "sigma": 0.6, "t0": 0.5,
             "dir": (1.0, 0.7, 0.0)}
    dt, n_steps, m = 0.05, 30, 20
    Ns = lat["Ns"]
    D = oracle.sector_dims(Ns, *sec)[2]
    psi0 = rand_vec(D, 9)
    res = oracle.propagate(lat, *sec, 0.0, psi0, pulse, dt, n_steps, m,
                           form="csr")
    u = np.eye(Ns, dtype=complex)
    for n in range(n_steps):
        h = oracle.single_particle_matrix(lat, oracle.pulse_A((n + 0.5) * dt, pulse))
        u = sla.expm(-1j * dt * h) @ u
    Mu, Md = minors_matrix(u, Ns, sec[0]), minors_matrix(u, Ns, sec[1])
    P = psi0.reshape(Mu.shape[0], Md.shape[0])
    ref = (Mu @ P @ Md.T).reshape(-1)
    assert np.linalg.norm(res["psi"] - ref) < 1e-11


def test_atomic_limit_exact_phases_and_breakdown():
    lat = synth.ring(6, t=0.0)
    U, dt, n_steps = 8.0, 0.02, 25
    D = oracle.sector_dims(6, 3, 3)[2]
    psi0 = rand_vec(D, 2)
    res = oracle.propagate(lat, 3, 3, U, psi0, synth.PULSES["ring8"], dt,
                           n_steps, 12, form="csr")
    w = oracle.double_occupancy_weights(6, 3, 3)
    ref = np.exp(-1j * U * w * dt * n_steps) * psi0
    assert np.abs(res["psi"] - ref).max() < 1e-12
    # distinct diagonal values: #doubles in 0..3 -> Krylov space of dim 4
    assert max(res["m_eff"]) <= 4


def test_stationarity_from_ground_state():
    lat = synth.ring(6)
    U = 4.0
    E0, psi0, gap = oracle.ground_state(lat, 3, 3, U)
    assert gap > 1e-6
    dt, n_steps = 0.05, 40
    res = oracle.propagate(lat, 3, 3, U, psi0, None, dt, n_steps, 12,
                           with_energy=True, form="csr")
    ref = np.exp(-1j * E0 * dt * n_steps) * psi0
    assert np.abs(res["psi"] - ref).max() < 1e-12
    assert np.ptp(res["docc"]) < 1e-13
    assert np.abs(res["energy"] - E0 / 6).max() < 1e-13


def test_norm_conservation_under_pulse():
    lat = synth.torus(3, 3)
    D = oracle.sector_dims(9, 2, 2)[2]
    psi0 = rand_vec(D, 4)
    pulse = {"A0": 1.0, "omega": 4.0, "sigma": 1.0, "t0": 0.6,
             "dir": (1.0, 1.0, 0.0)}
    res = oracle.propagate(lat, 2, 2, 6.0, psi0, pulse, 0.04, 30, 16)
    assert np.abs(res["norm2"] - 1.0).max() < 1e-12


def test_docc_invariant_under_field_reversal():
    lat = synth.ring(6)
    E0, psi0, gap = oracle.ground_state(lat, 3, 3, 8.0)
    p = {"A0": 0.8, "omega": 6.0, "sigma": 0.7, "t0": 1.0, "dir": (1.0, 0, 0)}
    pm = dict(p, dir=(-1.0, 0, 0))
    r1 = oracle.propagate(lat, 3, 3, 8.0, psi0, p, 0.05, 40, 14, form="csr")
    r2 = oracle.propagate(lat, 3, 3, 8.0, psi0, pm, 0.05, 40, 14, form="csr")
    assert np.ptp(r1["docc"]) > 1e-4          # the pulse does something
    assert np.abs(r1["docc"] - r2["docc"]).max() < 1e-12


def test_midpoint_rule_second_order():
    lat = synth.ring(6)
    E0, psi0, _ = oracle.ground_state(lat, 3, 3, 4.0)
    p = {"A0": 1.2, "omega": 5.0, "sigma": 0.5, "t0": 0.8, "dir": (1.0, 0, 0)}
    T = 1.6

    def run(dt):
        return oracle.propagate(lat, 3, 3, 4.0, psi0, p, dt,
                                int(round(T / dt)), 20, form="csr")["psi"]
    ref = run(0.1 / 16)
    e1 = np.linalg.norm(run(0.1) - ref)
    e2 = np.linalg.norm(run(0.05) - ref)
    order = np.log2(e1 / e2)
    assert order >= 1.9, order


def test_observables_definitions():
    # <d> of a single basis state = #doubles / Ns; E of an eigenvector = eig/Ns
    lat = synth.ring(4)
    H = oracle.build_H(lat, 2, 2, 3.0)
    w = oracle.double_occupancy_weights(4, 2, 2)
    for k in range(len(w)):
        e = np.zeros(len(w), dtype=complex)
        e[k] = 1.0
        assert oracle.double_occupation(e, w, 4) == w[k] / 4
    lam, vec = np.linalg.eigh(H.toarray())
    assert abs(oracle.energy_per_site(H, vec[:, 3], 4) - lam[3] / 4) < 1e-14


# ---------------------------------------------------------------- adaptive m
# The a-posteriori exit of Algorithm 6: delta = |y^(j) - y^(j-1)| / |y^(j)|,
# epsilon = min(1 + |y|, delta / (1 - delta) |y|) (delta < 1).

def test_adaptive_estimate_two_level_closed_form():
    """H = [[a, b], [b, a]], v = e_1: the Krylov space has dimension 2 and
    exp(-i tau T_2) e_1 = exp(-i tau a) (cos tau|b|, -i sin tau|b|), so
    delta = 2 |sin(tau |b| / 2)| exactly; y^(1) against y^(0) = 0 gives
    delta = 1, epsilon = 1 + |y^(1)| = 2."""
    a, b, tau = 0.7, -1.3, 0.4
    H = np.array([[a, b], [b, a]], dtype=np.complex128)
    v = np.array([1.0, 0.0], dtype=np.complex128)
    out, info = oracle.lanczos_expm(H, v, tau, 3, eps_tol=1e-9)
    assert info["m_eff"] == 2
    assert info["eps_history"] == [2.0]
    d = 2 * abs(np.sin(tau * abs(b) / 2))
    assert abs(info["delta"] - d) < 1e-14
    assert abs(info["eps"] - min(2.0, d / (1 - d))) < 1e-13
    ref = sla.expm(-1j * tau * H) @ v
    assert np.abs(out - ref).max() < 1e-14


def test_adaptive_exit_is_first_converged_step_and_equals_truncation():
    """The exit happens at the first j with epsilon_j < tol, and the result is
    then exactly the fixed-m step with m = j (same arithmetic, truncated)."""
    lat = synth.ring(6)
    H = oracle.build_H(lat, 3, 2, 4.0, (0.4, 0.0, 0.0))
    v = rand_vec(H.shape[0], 9)
    for tau, tol in ((0.05, 1e-6), (0.05, 1e-10), (0.3, 1e-8)):
        out, info = oracle.lanczos_expm(H, v, tau, 30, eps_tol=tol)
        eh = info["eps_history"]
        k = info["m_eff"]
        assert k < 30 and len(eh) == k
        assert eh[-1] < tol and all(e >= tol for e in eh[:-1])
        ref, rinfo = oracle.lanczos_expm(H, v, tau, k)
        assert rinfo["m_eff"] == k
        assert np.abs(out - ref).max() == 0.0


def test_adaptive_accuracy_against_dense_expm():
    """The error of the adaptive step stays within a small multiple of the
    tolerance (the estimate is within about an order of magnitude of the
    error, Fig. of Sec. 3.4), and a tighter tolerance never uses fewer
    vectors."""
    lat = synth.ring(6)
    H = oracle.build_H(lat, 3, 3, 6.0, (0.25, 0.0, 0.0))
    Hd = H.toarray()
    v = rand_vec(H.shape[0], 4)
    for tau in (0.02, 0.1, 0.4):
        ref = sla.expm(-1j * tau * Hd) @ v
        prev_m = 0
        for tol in (1e-4, 1e-7, 1e-10, 1e-13):
            out, info = oracle.lanczos_expm(H, v, tau, 40, eps_tol=tol)
            err = np.linalg.norm(out - ref)
            assert err <= 100 * tol + 1e-14, (tau, tol, err, info["m_eff"])
            assert info["m_eff"] >= prev_m
            prev_m = info["m_eff"]


def test_adaptive_with_tiny_tolerance_is_fixed_m():
    lat = synth.ring(6)
    H = oracle.build_H(lat, 3, 3, 6.0, (0.25, 0.0, 0.0))
    v = rand_vec(H.shape[0], 2)
    a, ia = oracle.lanczos_expm(H, v, 0.05, 14, eps_tol=1e-300)
    b, ib = oracle.lanczos_expm(H, v, 0.05, 14)
    assert ia["m_eff"] == ib["m_eff"] == 14
    assert np.array_equal(a, b)


def test_adaptive_trajectory_close_to_fixed_m():
    """A pulsed ring trajectory with the adaptive exit stays within the
    tolerance scale of the fixed-m trajectory and uses fewer vectors."""
    lat = synth.ring(8)
    psi0 = rand_vec(56 * 56, 3)
    p = synth.PULSES["ring8"]
    fixed = oracle.propagate(lat, 3, 3, 8.0, psi0, p, 0.02, 40, 20, t_start=4.0)
    adap = oracle.propagate(lat, 3, 3, 8.0, psi0, p, 0.02, 40, 20, t_start=4.0,
                            eps_tol=1e-10)
    assert max(adap["m_eff"]) < 20
    assert np.abs(adap["docc"] - fixed["docc"]).max() < 1e-8
    assert np.linalg.norm(adap["psi"] - fixed["psi"]) < 1e-8


# -------------------------------------------------------------------- CFET4
# exp(-i tau (a1 H1 + a2 H2)) exp(-i tau (a2 H1 + a1 H2)), H_k = H(t + c_k tau)

def test_cfet4_coefficients():
    """Gauss-Legendre nodes of [0, 1] and weights summing to 1/2 per factor
    with a1 - a2 = -sqrt(3)/3 (the conditions of fourth order)."""
    c1, c2 = oracle.CFET4_C
    a1, a2 = oracle.CFET4_A
    x, w = np.polynomial.legendre.leggauss(2)
    assert np.allclose(sorted([c1, c2]), (x + 1) / 2, atol=1e-15)
    assert abs(a1 + a2 - 0.5) < 1e-15
    assert abs((a1 - a2) + np.sqrt(3) / 3) < 1e-15


def test_cfet4_time_independent_is_exact_exponential():
    lat = synth.ring(6)
    psi0 = rand_vec(400, 8)
    H = oracle.build_H(lat, 3, 3, 5.0, (0.0, 0.0, 0.0)).toarray()
    res = oracle.propagate(lat, 3, 3, 5.0, psi0, None, 0.1, 6, 24, form="csr",
                           scheme="cfet4")
    ref = sla.expm(-0.6j * H) @ psi0
    assert np.linalg.norm(res["psi"] - ref) < 1e-11


@pytest.mark.parametrize("lat,sec", [(synth.ring(6), (3, 2)), (synth.triangle(), (2, 1))])
def test_cfet4_free_fermions_are_slater_of_one_electron_cfet4(lat, sec):
    """U = 0: the many-body CFET4 step is the determinant-minor lift of the
    one-electron CFET4 step (each factor is a quadratic Hamiltonian)."""
    pulse = {"A0": 0.9, "omega": 5.0, "sigma": 0.6, "t0": 0.5, "dir": (1.0, 0.7, 0.0)}
    dt, n_steps = 0.1, 12
    Ns = lat["Ns"]
    D = oracle.sector_dims(Ns, *sec)[2]
    psi0 = rand_vec(D, 4)
    res = oracle.propagate(lat, *sec, 0.0, psi0, pulse, dt, n_steps, 24, form="csr",
                           scheme="cfet4")
    (c1, c2), (a1, a2) = oracle.CFET4_C, oracle.CFET4_A
    u = np.eye(Ns, dtype=complex)
    for n in range(n_steps):
        h1 = oracle.single_particle_matrix(lat, oracle.pulse_A((n + c1) * dt, pulse))
        h2 = oracle.single_particle_matrix(lat, oracle.pulse_A((n + c2) * dt, pulse))
        u = sla.expm(-1j * dt * (a1 * h1 + a2 * h2)) @ sla.expm(-1j * dt * (a2 * h1 + a1 * h2)) @ u
    Mu = minors_matrix(u, Ns, sec[0])
    Md = minors_matrix(u, Ns, sec[1])
    ref = (Mu @ psi0.reshape(Mu.shape[0], -1) @ Md.T).reshape(-1)
    assert np.linalg.norm(res["psi"] - ref) < 1e-11


def test_cfet4_is_fourth_order():
    """Error at T = 1.2 against a dt/16 reference, for dt and dt/2: the
    observed order is >= 3.8 (midpoint: about 2)."""
    lat = synth.ring(6)
    psi0 = rand_vec(400, 6)
    p = {"A0": 0.8, "omega": 4.0, "sigma": 0.5, "t0": 0.6, "dir": (1.0, 0.0, 0.0)}

    def run(dt, scheme):
        n = int(round(1.2 / dt))
        return oracle.propagate(lat, 3, 3, 4.0, psi0, p, dt, n, 30, form="csr",
                                scheme=scheme)["psi"]
    ref = run(0.1 / 16, "cfet4")
    e1 = np.linalg.norm(run(0.1, "cfet4") - ref)
    e2 = np.linalg.norm(run(0.05, "cfet4") - ref)
    order = np.log2(e1 / e2)
    assert order >= 3.8, order
    em = np.linalg.norm(run(0.05, "midpoint") - ref)
    assert e2 < em / 10
