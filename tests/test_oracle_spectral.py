"""Pins of the oracle's c / c^+ maps and G^< / G^> overlaps (CPU).

* Canonical anticommutation relations of Eqs. (7)-(8) on random vectors.
* Sum rules at the reference time: L_is(0) = <n_is>, G_is(0) = 1 - <n_is>,
  sum_i L_is(0) = n_s.
* A = 0: the propagated overlaps equal the Lehmann sums of Eq. (17) from a
  dense eigendecomposition.
* Hubbard dimer closed form (Sec. 3.9 benchmarks the Green's function against
  an analytic two-site computation): with R = sqrt(U^2 + 16 t^2) the (1,1)
  ground state is (a (D0 + D1) + b (S01 + S10)) / sqrt 2 with
  (a, b) proportional to (2t, (U + R)/2), and
      L(t) = ((a+b)/2)^2 e^{-i(-t - E0)t} + ((a-b)/2)^2 e^{-i(t - E0)t},
      G(t) = ((a+b)/2)^2 e^{-i(U - t - E0)t} + ((a-b)/2)^2 e^{-i(U + t - E0)t}.
"""
import numpy as np
import pytest

import oracle
import synth


def test_anticommutators():
    Ns, nu, nd = 4, 2, 2
    D = oracle.sector_dims(Ns, nu, nd)[2]
    psi = synth.complex_normal(D, 1)
    for i in range(Ns):
        for s in (0, 1):
            nu_c, nd_c = oracle.sector_shift(nu, nd, "c", s)
            nu_d, nd_d = oracle.sector_shift(nu, nd, "cdag", s)
            a = oracle.apply_cdag(Ns, nu_c, nd_c,
                                  oracle.apply_c(Ns, nu, nd, psi, i, s), i, s)
            b = oracle.apply_c(Ns, nu_d, nd_d,
                               oracle.apply_cdag(Ns, nu, nd, psi, i, s), i, s)
            assert np.abs(a + b - psi).max() < 1e-15
            for j in range(Ns):
                for s2 in (0, 1):
                    if (i, s) == (j, s2):
                        continue
                    # {c_is, c_js2} = 0
                    x = oracle.apply_c(Ns, *oracle.sector_shift(nu, nd, "c", s2),
                                       oracle.apply_c(Ns, nu, nd, psi, j, s2), i, s)
                    y = oracle.apply_c(Ns, *oracle.sector_shift(nu, nd, "c", s),
                                       oracle.apply_c(Ns, nu, nd, psi, i, s), j, s2)
                    assert np.abs(x + y).max() < 1e-15
                    # {c_is, c^+_js2} = 0
                    x = oracle.apply_c(Ns, *oracle.sector_shift(nu, nd, "cdag", s2),
                                       oracle.apply_cdag(Ns, nu, nd, psi, j, s2), i, s)
                    y = oracle.apply_cdag(Ns, *oracle.sector_shift(nu, nd, "c", s),
                                          oracle.apply_c(Ns, nu, nd, psi, i, s), j, s2)
                    assert np.abs(x + y).max() < 1e-15


def test_sum_rules_at_reference_time():
    lat = synth.torus(3, 3)
    E0, psi0, _ = oracle.ground_state(lat, 4, 4, 6.0)
    r = oracle.spectral_batch(lat, 4, 4, 6.0, psi0, None, 0.02, 0, 12)
    L0, G0 = r["L"][0], r["G"][0]
    for s, n in ((0, 4), (1, 4)):
        assert abs(L0[:, s].sum() - n) < 1e-12
        assert np.abs(L0[:, s] + G0[:, s] - 1.0).max() < 1e-12
    # <n_i> on a translation-invariant lattice = n/Ns
    assert np.abs(L0.real - 4 / 9).max() < 1e-12


def test_overlaps_match_lehmann_at_zero_field():
    lat = synth.ring(6)
    U = 5.0
    E0, psi0, _ = oracle.ground_state(lat, 3, 3, U)
    dt, n = 0.05, 20
    r = oracle.spectral_batch(lat, 3, 3, U, psi0, None, dt, n, 16, sites=[0, 2])
    times = dt * np.arange(n + 1)
    for i in (0, 2):
        for s in (0, 1):
            Lr, Gr = oracle.lehmann_overlaps(lat, 3, 3, U, psi0, E0, times, i, s)
            assert np.abs(r["L"][:, i, s] - Lr).max() < 1e-11
            assert np.abs(r["G"][:, i, s] - Gr).max() < 1e-11


@pytest.mark.parametrize("U", [0.0, 2.0, 8.0])
def test_dimer_green_function_closed_form(U):
    t = 1.0
    lat = synth.dimer(t)
    E0, psi0, _ = oracle.ground_state(lat, 1, 1, U)
    R = np.sqrt(U * U + 16 * t * t)
    assert abs(E0 - (U - R) / 2) < 1e-13
    a, b = 2 * t, (U + R) / 2
    nrm = np.hypot(a, b)
    a, b = a / nrm, b / nrm
    dt, n = 0.05, 30
    r = oracle.spectral_batch(lat, 1, 1, U, psi0, None, dt, n, 8)
    tt = dt * np.arange(n + 1)
    wB, wA = ((a + b) / 2) ** 2, ((a - b) / 2) ** 2
    L = wB * np.exp(-1j * (-t - E0) * tt) + wA * np.exp(-1j * (t - E0) * tt)
    G = wB * np.exp(-1j * (U - t - E0) * tt) + wA * np.exp(-1j * (U + t - E0) * tt)
    for i in (0, 1):
        for s in (0, 1):
            assert np.abs(r["L"][:, i, s] - L).max() < 1e-12
            assert np.abs(r["G"][:, i, s] - G).max() < 1e-12


# ------------------------------------------- reference time, Eq. (4) pulse, A(nu,t)

def test_cos_phase_pulse_is_the_papers_hopping_factor():
    """Eq. (4): with dir = (1,1,0) on the 3x4 torus every +x and +y hop
    p -> q carries f(t) = exp(i a [cos(omega (t - t_p)) - b]
    e^{-(t-t_p)^2/(2 sigma^2)}) (one-electron sector, h[q, p] = -t f(t));
    b = cos(omega t_p) makes f(0) = 1."""
    lat = synth.torus(4, 3)
    a, om, sg, tp = 0.7, 3.0, 1.2, 2.0
    b = np.cos(om * tp)
    pulse = {"A0": a, "omega": om, "sigma": sg, "t0": tp, "dir": (1.0, 1.0, 0.0),
             "shape": "cos_phase", "b": b}
    for t in (0.0, 1.3, 2.0, 4.1):
        f = np.exp(1j * a * (np.cos(om * (t - tp)) - b) * np.exp(-(t - tp) ** 2 / (2 * sg ** 2)))
        h = oracle.single_particle_matrix(lat, oracle.pulse_A(t, pulse))
        for p, q in zip(lat["p"], lat["q"]):
            assert abs(h[q, p] + f) < 1e-14
    assert np.abs(oracle.pulse_A(0.0, pulse)).max() < 1e-15


def test_broadened_transform_of_an_exponential():
    """(1/pi) Im int_0^T e^{(-eps + i nu) t} c e^{-i w t} dt
    = (1/pi) Im[c (e^{zT} - 1) / z], z = -eps + i (nu - w); the trapezoid
    error is O(dt^2)."""
    dt, n, eps = 1e-3, 20000, 0.3
    T = n * dt
    om, c = 1.7, 0.4 - 0.2j
    t = dt * np.arange(n + 1)
    G = c * np.exp(-1j * om * t)
    nu = np.array([-2.0, 0.5, 1.7, 3.0])
    got = oracle.broadened_transform(G, dt, eps, nu)
    z = -eps + 1j * (nu - om)
    exact = (c * (np.exp(z * T) - 1) / z).imag / np.pi
    assert np.abs(got - exact).max() < 1e-6
    # second order: halving dt divides the error by about 4
    e1 = np.abs(oracle.broadened_transform(G[::20], 20 * dt, eps, nu) - exact).max()
    e2 = np.abs(oracle.broadened_transform(G[::10], 10 * dt, eps, nu) - exact).max()
    assert 3.5 < e1 / e2 < 4.5


def test_equilibrium_spectral_function_equals_transformed_lehmann_sums():
    """At A = 0 the broadened transform of G^< + G^> from the propagated
    batch equals that of the Lehmann sums over the same window."""
    lat = synth.ring(6)
    U = 4.0
    E0, psi0, _ = oracle.ground_state(lat, 3, 3, U)
    dt, n, eps = 0.05, 160, 0.25
    r = oracle.spectral_batch(lat, 3, 3, U, psi0, None, dt, n, 16, sites=[0])
    times = dt * np.arange(n + 1)
    Lr, Gr = oracle.lehmann_overlaps(lat, 3, 3, U, psi0, E0, times, 0, 0)
    nu = np.linspace(-8, 8, 33)
    A = oracle.broadened_transform(r["G_less"][:, 0, 0] + r["G_greater"][:, 0, 0], dt, eps, nu)
    Ar = oracle.broadened_transform(1j * Lr - 1j * Gr, dt, eps, nu)
    assert np.abs(A - Ar).max() < 1e-9


def test_reference_time_batch_starts_from_the_propagated_state():
    """Sum rules at the reference time t_ref: L_is(t_ref, t_ref) =
    <psi(t_ref)| n_is |psi(t_ref)> and L + G = 1, with psi(t_ref) taken
    from the pulsed propagation."""
    lat = synth.ring(6)
    pulse = {"A0": 0.6, "omega": 5.0, "sigma": 1.0, "t0": 0.5, "dir": (1.0, 0.0, 0.0)}
    E0, psi0, _ = oracle.ground_state(lat, 3, 3, 4.0)
    pr = oracle.propagate(lat, 3, 3, 4.0, psi0, pulse, 0.05, 8, 16)["psi"]
    r = oracle.spectral_batch(lat, 3, 3, 4.0, pr, pulse, 0.05, 2, 16, t_start=0.4)
    assert np.abs(r["L"][0] + r["G"][0] - 1.0).max() < 1e-12
    assert abs(r["L"][0, :, 0].real.sum() - 3.0) < 1e-12
