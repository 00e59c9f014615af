"""Pins of the oracle's Hamiltonian (CPU only).

* Full Fock-space construction from the operator algebra (Jordan-Wigner
  matrices of Eqs. (7)-(8)) at Ns <= 4, restricted to a sector, equals the
  oracle's sector matrix exactly (block mode order), and equals it up to a
  diagonal +-1 gauge in the paper's site-interleaved mode order (Eq. (6)).
* Closed forms: Hubbard dimer ground energy (U - sqrt(U^2+16 t^2))/2 (Sec. 3.9
  benchmarks against analytic eigenvalues), single-electron ring spectrum
  -2t cos(2 pi k/Ns + A) with flux, the 3-cycle spectrum {-2t, t, t}, U=0
  double occupancy 1/4 on a translation-invariant half-filled ring.
* Structure: upper-triangle non-zero count of Eq. (22) on the complete graph.
* Gauge: a static uniform A on an open chain leaves the spectrum unchanged.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from oracle.krylov import KronHamiltonian


# ---------------------------------------------------------------- Fock space
def fock_annihilators(n_modes):
    """Dense c_m on the 2^n_modes Fock space, sign (-1)^(#occupied modes < m)."""
    D = 1 << n_modes
    ops = []
    for m in range(n_modes):
        c = np.zeros((D, D))
        for f in range(D):
            if (f >> m) & 1:
                sgn = (-1) ** bin(f & ((1 << m) - 1)).count("1")
                c[f ^ (1 << m), f] = sgn
        ops.append(c)
    return ops


def fock_hamiltonian(lat, U, A, mode_of):
    """H of Eq. (1) with Peierls phases of Eq. (3), built from c/c^+ matrices."""
    Ns = lat["Ns"]
    c = fock_annihilators(2 * Ns)
    cd = [x.T for x in c]
    D = 1 << (2 * Ns)
    H = np.zeros((D, D), dtype=complex)
    phi = lat["d"] @ np.asarray(A)
    for b in range(len(lat["p"])):
        p, q, tb = int(lat["p"][b]), int(lat["q"][b]), lat["t"][b]
        for s in (0, 1):
            mp, mq = mode_of(p, s), mode_of(q, s)
            # hop p -> q: -v_qp(t) c^+_q c_p, v_qp(t) = t exp(-i A.(R_q - R_p))
            H += -tb * np.exp(-1j * phi[b]) * (cd[mq] @ c[mp])
            H += -tb * np.exp(+1j * phi[b]) * (cd[mp] @ c[mq])
    for i in range(Ns):
        nu = cd[mode_of(i, 0)] @ c[mode_of(i, 0)]
        nd = cd[mode_of(i, 1)] @ c[mode_of(i, 1)]
        H += U * (nu @ nd)
        if lat.get("eps") is not None:
            H += lat["eps"][i] * (nu + nd)
    return H


def sector_fock_indices(Ns, n_up, n_dn, mode_of):
    bu, bd = oracle.spin_basis(Ns, n_up), oracle.spin_basis(Ns, n_dn)
    idx = []
    for u in bu:
        for d in bd:
            f = 0
            for i in range(Ns):
                if (int(u) >> i) & 1:
                    f |= 1 << mode_of(i, 0)
                if (int(d) >> i) & 1:
                    f |= 1 << mode_of(i, 1)
            idx.append(f)
    return np.array(idx)


def block_mode(Ns):
    return lambda i, s: i + s * Ns


def interleaved_mode(Ns):
    return lambda i, s: 2 * i + s


LATS = [
    ("triangle", synth.triangle(), (1, 1)),
    ("triangle21", synth.triangle(), (2, 1)),
    ("chain4_eps", synth.chain(4, eps=[0.3, -0.2, 0.1, 0.7]), (2, 2)),
    ("ring4", synth.ring(4), (2, 1)),
    ("complete4", synth.complete_graph(4, seed=3), (2, 2)),
    ("complete4_13", synth.complete_graph(4, seed=5), (1, 3)),
]


@pytest.mark.parametrize("name,lat,sector", LATS, ids=[x[0] for x in LATS])
def test_sector_matrix_equals_fock_construction(name, lat, sector):
    rng = np.random.default_rng(7)
    A = rng.standard_normal(3) * 0.7
    U = 3.3
    Ns = lat["Ns"]
    Hf = fock_hamiltonian(lat, U, A, block_mode(Ns))
    idx = sector_fock_indices(Ns, *sector, block_mode(Ns))
    Hs = Hf[np.ix_(idx, idx)]
    H = oracle.build_H(lat, *sector, U, A).toarray()
    assert np.abs(H - Hs).max() < 1e-13


@pytest.mark.parametrize("name,lat,sector", LATS, ids=[x[0] for x in LATS])
def test_interleaved_mode_order_is_a_diagonal_gauge(name, lat, sector):
    rng = np.random.default_rng(11)
    A = rng.standard_normal(3) * 0.4
    U = 2.1
    Ns = lat["Ns"]
    Hf = fock_hamiltonian(lat, U, A, interleaved_mode(Ns))
    idx = sector_fock_indices(Ns, *sector, interleaved_mode(Ns))
    Hi = Hf[np.ix_(idx, idx)]
    H = oracle.build_H(lat, *sector, U, A).toarray()
    # g(u,d) = (-1)^(sum_j n_j,up * #{i < j : n_i,dn = 1})
    bu, bd = oracle.spin_basis(Ns, sector[0]), oracle.spin_basis(Ns, sector[1])
    g = []
    for u in bu:
        for d in bd:
            e = 0
            for j in range(Ns):
                if (int(u) >> j) & 1:
                    e += bin(int(d) & ((1 << j) - 1)).count("1")
            g.append((-1) ** e)
    G = np.diag(g)
    assert np.abs(Hi - G @ H @ G).max() < 1e-13
    assert np.allclose(np.linalg.eigvalsh(Hi), np.linalg.eigvalsh(H), atol=1e-12)


# --------------------------------------------------------------- closed forms
@pytest.mark.parametrize("U,E0", [(8.0, -0.4721359549995796),
                                  (4.0, -0.8284271247461903)])
def test_dimer_ground_energy(U, E0):
    # (U - sqrt(U^2 + 16 t^2)) / 2, t = 1
    assert abs(E0 - (U - np.sqrt(U * U + 16)) / 2) < 1e-15
    E, psi, gap = oracle.ground_state(synth.dimer(), 1, 1, U)
    assert abs(E - E0) < 1e-13
    lam = np.linalg.eigvalsh(oracle.build_H(synth.dimer(), 1, 1, U).toarray())
    assert np.allclose(sorted(lam), sorted([(U - np.sqrt(U * U + 16)) / 2, 0.0, U,
                                            (U + np.sqrt(U * U + 16)) / 2]),
                       atol=1e-13)


@pytest.mark.parametrize("Ns", [3, 5, 8])
@pytest.mark.parametrize("A", [0.0, 0.37, -1.1])
def test_single_electron_ring_with_flux(Ns, A):
    lat = synth.ring(Ns)
    H = oracle.build_H(lat, 1, 0, 5.0, (A, 0, 0)).toarray()
    ev = np.sort(np.linalg.eigvalsh(H))
    k = 2 * np.pi * np.arange(Ns) / Ns
    assert np.allclose(ev, np.sort(-2 * np.cos(k + A)), atol=1e-13)
    # the down-spin sector (0,1) is the same problem
    H2 = oracle.build_H(lat, 0, 1, 5.0, (A, 0, 0)).toarray()
    assert np.allclose(np.sort(np.linalg.eigvalsh(H2)), ev, atol=1e-13)


def test_three_cycle_sign_sensitive_spectrum():
    ev = np.sort(np.linalg.eigvalsh(
        oracle.build_H(synth.triangle(), 1, 0, 0.0).toarray()))
    assert np.allclose(ev, [-2.0, 1.0, 1.0], atol=1e-14)


def test_single_particle_matrix_matches_one_electron_sector():
    lat = synth.torus(4, 3)
    A = (0.3, -0.8, 0.0)
    H = oracle.build_H(lat, 1, 0, 1.0, A).toarray()
    h = oracle.single_particle_matrix(lat, A)
    # basis of (1,0): words 1<<i ascending, i.e. site order
    assert np.abs(H - h).max() < 1e-14


def test_atomic_limit_is_diagonal():
    lat = synth.ring(6, t=0.0)
    H = oracle.build_H(lat, 3, 3, 2.5).toarray()
    assert np.abs(H - np.diag(np.diag(H))).max() == 0.0
    w = oracle.double_occupancy_weights(6, 3, 3)
    assert np.array_equal(np.diag(H).real, 2.5 * w)


def test_free_fermion_double_occupancy_quarter():
    # U = 0, half-filled 6-ring (unique ground state): <d> = <n_up><n_dn> = 1/4
    lat = synth.ring(6)
    E0, psi, gap = oracle.ground_state(lat, 3, 3, 0.0)
    assert gap > 1e-6
    w = oracle.double_occupancy_weights(6, 3, 3)
    assert abs(oracle.double_occupation(psi, w, 6) - 0.25) < 1e-13
    # E0 = 2 * (sum of the three lowest one-electron levels -2, -1, -1)
    assert abs(E0 - 2 * (-2 - 1 - 1)) < 1e-12


# ------------------------------------------------------------------ structure
@pytest.mark.parametrize("Ns,nu,nd", [(4, 2, 2), (5, 2, 3), (6, 3, 3),
                                      (7, 3, 4), (8, 4, 4)])
def test_nnz_upper_triangle_complete_graph(Ns, nu, nd):
    lat = synth.complete_graph(Ns, seed=Ns)
    H = oracle.build_H(lat, nu, nd, 1.7, (0.2, 0.1, -0.3))
    N = H.shape[0]
    upper_off = sp.triu(H, k=1).count_nonzero()
    nnz_eq22 = N * (1 + 0.5 * nu * (Ns - nu) + 0.5 * nd * (Ns - nd))
    assert N + upper_off == nnz_eq22


def test_kron_operator_equals_csr():
    lat = synth.torus(4, 3)
    rng = np.random.default_rng(1)
    A = (0.2, -0.5, 0.0)
    for sec in [(2, 3), (3, 3)]:
        H = oracle.build_H(lat, *sec, 8.0, A)
        K = KronHamiltonian(lat, *sec, 8.0, A)
        v = rng.standard_normal(H.shape[0]) + 1j * rng.standard_normal(H.shape[0])
        assert np.abs(H @ v - K @ v).max() < 1e-12


def test_static_field_on_open_chain_is_a_gauge():
    lat = synth.chain(6)
    e0 = np.linalg.eigvalsh(oracle.build_H(lat, 3, 2, 4.0).toarray())
    e1 = np.linalg.eigvalsh(oracle.build_H(lat, 3, 2, 4.0, (0.9, 0, 0)).toarray())
    assert np.allclose(e0, e1, atol=1e-12)


def test_ring_flux_periodicity():
    Ns = 5
    lat = synth.ring(Ns)
    A = 0.23
    e0 = np.linalg.eigvalsh(oracle.build_H(lat, 2, 2, 3.0, (A, 0, 0)).toarray())
    e1 = np.linalg.eigvalsh(oracle.build_H(
        lat, 2, 2, 3.0, (A + 2 * np.pi / Ns, 0, 0)).toarray())
    assert np.allclose(e0, e1, atol=1e-12)
    e2 = np.linalg.eigvalsh(oracle.build_H(lat, 2, 2, 3.0, (A + 0.5, 0, 0)).toarray())
    assert not np.allclose(e0, e2, atol=1e-6)


def test_pulse_values():
    pulse = {"A0": 0.5, "omega": 8.0, "sigma": 2.0, "t0": 5.0,
             "dir": (1.0, 1.0, 0.0)}
    # A(0) = 0.5 exp(-25/8) sin(-40)
    a0 = 0.5 * np.exp(-25.0 / 8.0) * np.sin(-40.0)
    assert np.allclose(oracle.pulse_A(0.0, pulse), [a0, a0, 0.0], rtol=1e-15)
    assert abs(a0 - (-0.016369)) < 5e-6
    assert np.allclose(oracle.pulse_A(5.0, pulse), 0.0)
