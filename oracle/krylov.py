"""Krylov exponential, midpoint time stepping, observables, ground state.

Oracle (test infrastructure only).  Follows Sec. 3.4 of the paper:

* Eq. (32), exponential midpoint rule:
      v^{n+1} = exp(-i tau H(t_n + tau/2)) v^n,   t_n = t_start + n tau.
* Algorithm 6, Lanczos construction of the Krylov basis V and the tridiagonal
  projection h, then  exp(-i tau H) v ~= beta V exp(-i tau h) e_1.
  Readings: by default the Krylov dimension m is fixed (the adaptive exit of
  the algorithm is replaced by a fixed count); h_jj = Re(V_j^H w) because H is
  Hermitian; the breakdown exit |h_{j+1,j}| < alpha * tol of the algorithm is
  taken with alpha = max(1, max|h_kk|, max h_{k+1,k}) over the steps so far and
  tol = 1e-13 (the float64 rule the CUDA path uses too); the a-posteriori
  estimate delta / epsilon of the algorithm is computed and returned as a
  diagnostic.
  With an error tolerance ``eps_tol`` the adaptive exit is taken as printed:
  after every step j, y^(j) = exp(-i tau h_j) e_1 is compared with y^(j-1)
  (zero-padded; y^(0) = 0), delta = |y^(j) - y^(j-1)| / |y^(j)|, epsilon =
  min(1 + |y^(j)|, delta / (1 - delta) |y^(j)|) for delta < 1 and 1 + |y^(j)|
  otherwise, and the step returns beta V y^(j) once epsilon < eps_tol or
  |h_{j+1,j}| < alpha * eps_tol (alpha as above); m is then the largest
  dimension N_max.
* Commutator-free exponential time propagator of fourth order (CFET4; the
  family the paper names in Sec. 3.4 as the higher-order extension of
  Eq. (32)), in the two-exponential form of Alvermann and Fehske (J. Comput.
  Phys. 230, 5930 (2011)) and Blanes and Moan (Appl. Numer. Math. 56, 1519
  (2006)):  v^{n+1} = exp(-i tau (a1 H1 + a2 H2)) exp(-i tau (a2 H1 + a1 H2))
  v^n with H_k = H(t_n + c_k tau), Gauss nodes c_{1,2} = 1/2 -+ sqrt(3)/6 and
  weights a_{1,2} = (3 -+ 2 sqrt(3)) / 12.  Each factor is one Krylov step of
  Algorithm 6 on the combined (Hermitian) matrix.
* The m x m exponential (Expokit in the paper) is computed here from the
  eigendecomposition of the real symmetric tridiagonal h (numpy.linalg.eigh):
  exp(-i tau h) e_1 = Q diag(exp(-i tau lambda)) Q^T e_1.
* Observables (Sec. 3.5; Eqs. (13)-(14)): <d> = (1/Ns) v^H (w_d . v) without
  division by |v|^2; E = (1/Ns) v^H H(t_n) v.
* Ground state (Sec. 3.4): lowest eigenpair of H(A=0).  The paper uses a
  shifted power iteration (Algorithms 4-5); the oracle uses the textbook
  routines numpy.linalg.eigh (small) or scipy.sparse.linalg.eigsh (large),
  which reach the same eigenpair.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import spin_basis
from .hamiltonian import (build_H, spin_hopping_matrix, diag_U, pulse_A,
                          double_occupancy_weights)

BREAKDOWN_TOL = 1e-13


class KronHamiltonian:
    """H(A) applied as T_up Psi + Psi T_dn^T + diag . Psi.

    The same operator as ``build_H`` (kron(T_up,1) + kron(1,T_dn) + diag in the
    row-major index); a test checks the two agree.  Used where the full CSR
    matrix would be too large.
    """

    def __init__(self, lattice, n_up, n_dn, U, A=(0.0, 0.0, 0.0)):
        self.Tu = spin_hopping_matrix(lattice, n_up, A)
        self.TdT = spin_hopping_matrix(lattice, n_dn, A).T.tocsr()
        self.du, self.dd = self.Tu.shape[0], self.TdT.shape[0]
        self.dg = diag_U(lattice, n_up, n_dn, U).reshape(self.du, self.dd)
        self.shape = (self.du * self.dd, self.du * self.dd)

    def __matmul__(self, v):
        P = np.asarray(v).reshape(self.du, self.dd)
        W = self.Tu @ P + (self.TdT.T @ P.T).T + self.dg * P
        return W.reshape(-1)

    dot = __matmul__


def make_H(lattice, n_up, n_dn, U, A, form="auto"):
    du = len(spin_basis(lattice["Ns"], n_up))
    dd = len(spin_basis(lattice["Ns"], n_dn))
    if form == "csr" or (form == "auto" and du * dd <= 20000):
        return build_H(lattice, n_up, n_dn, U, A)
    return KronHamiltonian(lattice, n_up, n_dn, U, A)


def small_expm_e1(alpha, beta, tau):
    """exp(-i tau T) e_1 for the real symmetric tridiagonal T(alpha, beta)."""
    k = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    if k > 1:
        b = np.asarray(beta[:k - 1], dtype=np.float64)
        T += np.diag(b, 1) + np.diag(b, -1)
    lam, Q = np.linalg.eigh(T)
    return Q @ (np.exp(-1j * tau * lam) * Q[0, :])


def epsilon_estimate(y, y_prev):
    """(delta, epsilon) of the a-posteriori error estimate of Algorithm 6
    for consecutive approximations y = y^(j) and y_prev = y^(j-1) (shorter by
    one; zero-padded)."""
    yp = np.zeros(len(y), dtype=np.complex128)
    yp[:len(y_prev)] = y_prev
    ny = np.linalg.norm(y)
    delta = np.linalg.norm(y - yp) / ny
    eps = min(1 + ny, delta / (1 - delta) * ny) if delta < 1 else 1 + ny
    return float(delta), float(eps)


def lanczos_expm(H, v, tau, m, tol=BREAKDOWN_TOL, eps_tol=None):
    """One step of Algorithm 6 with Krylov dimension m (fixed), or at most m
    with the adaptive exit when eps_tol is given.

    Returns (beta0 * V y, info) with info = dict(alpha, beta, m_eff, delta,
    eps); with eps_tol also eps_history (epsilon after every step).
    """
    v = np.asarray(v, dtype=np.complex128)
    beta0 = np.sqrt(np.vdot(v, v).real)
    if beta0 == 0.0:
        return v.copy(), {"alpha": [], "beta": [], "m_eff": 0,
                          "delta": 0.0, "eps": 0.0, "eps_history": []}
    V = [v / beta0]
    alpha, beta = [], []
    scale = 1.0
    m_eff = m
    y_prev = np.zeros(0, dtype=np.complex128)
    eps_hist = []
    for j in range(m):
        w = H @ V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        a = np.vdot(V[j], w).real
        alpha.append(a)
        w = w - a * V[j]
        b = np.sqrt(np.vdot(w, w).real)
        scale = max(scale, abs(a))
        beta.append(b)
        if j == m - 1:
            break
        if b <= tol * scale:
            m_eff = j + 1
            break
        if eps_tol is not None:
            # a-posteriori exit of Algorithm 6 after step j + 1
            y = small_expm_e1(alpha, beta[:j], tau)
            _, e = epsilon_estimate(y, y_prev)
            eps_hist.append(e)
            y_prev = y
            if e < eps_tol or b < eps_tol * scale:
                m_eff = j + 1
                break
        scale = max(scale, b)
        V.append(w / b)
    y = small_expm_e1(alpha[:m_eff], beta[:m_eff - 1], tau)
    if m_eff > 1:
        yp = small_expm_e1(alpha[:m_eff - 1], beta[:m_eff - 2], tau)
        delta, eps = epsilon_estimate(y, yp)
    else:
        delta = eps = 0.0
    out = np.zeros_like(v)
    for j in range(m_eff):
        out += y[j] * V[j]
    out *= beta0
    return out, {"alpha": alpha, "beta": beta, "m_eff": m_eff,
                 "delta": delta, "eps": eps, "eps_history": eps_hist}


def double_occupation(psi, w_d, Ns):
    """<d> = (1/Ns) sum_k w_d[k] |psi_k|^2 (Eq. (13) via Sec. 3.5)."""
    psi = np.asarray(psi).reshape(-1)
    return float(np.sum(w_d * (psi.real ** 2 + psi.imag ** 2)) / Ns)


def energy_per_site(H, psi, Ns):
    """E = (1/Ns) <psi|H|psi> (Eq. (14))."""
    psi = np.asarray(psi).reshape(-1)
    return float(np.vdot(psi, H @ psi).real / Ns)


CFET4_C = (0.5 - np.sqrt(3.0) / 6.0, 0.5 + np.sqrt(3.0) / 6.0)
CFET4_A = ((3.0 - 2.0 * np.sqrt(3.0)) / 12.0, (3.0 + 2.0 * np.sqrt(3.0)) / 12.0)


def cfet4_factors(lattice, n_up, n_dn, U, pulse, t, dt, form="auto"):
    """The two matrices of one CFET4 step from t to t + dt, in the order
    they act: (a2 H1 + a1 H2, then a1 H1 + a2 H2)."""
    H1 = make_H(lattice, n_up, n_dn, U, pulse_A(t + CFET4_C[0] * dt, pulse), form)
    H2 = make_H(lattice, n_up, n_dn, U, pulse_A(t + CFET4_C[1] * dt, pulse), form)
    a1, a2 = CFET4_A
    return _lincomb(a2, H1, a1, H2), _lincomb(a1, H1, a2, H2)


def _lincomb(a, X, b, Y):
    if sp.issparse(X):
        return (a * X + b * Y).tocsr()
    return _KronLinComb(a, X, b, Y)


class _KronLinComb:
    """a X + b Y for two KronHamiltonian operators (applied, not formed)."""

    def __init__(self, a, X, b, Y):
        self.a, self.X, self.b, self.Y = a, X, b, Y
        self.shape = X.shape

    def __matmul__(self, v):
        return self.a * (self.X @ v) + self.b * (self.Y @ v)

    dot = __matmul__


def propagate(lattice, n_up, n_dn, U, psi0, pulse, dt, n_steps, m,
              t_start=0.0, with_energy=False, form="auto", record_states=False,
              eps_tol=None, scheme="midpoint"):
    """Trajectory by the exponential midpoint rule (Eq. (32); scheme
    "midpoint") or by CFET4 (scheme "cfet4", two Krylov steps per time
    step), with fixed-m Lanczos steps (or at most m with the adaptive exit,
    eps_tol given).  For CFET4, m_eff and delta are the larger of the two
    factors' values.

    Observables are recorded at t_0 = t_start and after every step at
    t_{n+1}.  Returns dict(psi, docc, norm2, energy, m_eff, delta, states).
    """
    Ns = lattice["Ns"]
    w_d = double_occupancy_weights(Ns, n_up, n_dn)
    psi = np.asarray(psi0, dtype=np.complex128).reshape(-1).copy()
    docc = [double_occupation(psi, w_d, Ns)]
    norm2 = [float(np.vdot(psi, psi).real)]
    energy = []
    if with_energy:
        energy.append(energy_per_site(
            make_H(lattice, n_up, n_dn, U, pulse_A(t_start, pulse), form),
            psi, Ns))
    m_eff, deltas, states = [], [], []
    if record_states:
        states.append(psi.copy())
    for n in range(n_steps):
        if scheme == "midpoint":
            t_mid = t_start + (n + 0.5) * dt
            H = make_H(lattice, n_up, n_dn, U, pulse_A(t_mid, pulse), form)
            psi, info = lanczos_expm(H, psi, dt, m, eps_tol=eps_tol)
            m_eff.append(info["m_eff"])
            deltas.append(info["delta"])
        elif scheme == "cfet4":
            Ha, Hb = cfet4_factors(lattice, n_up, n_dn, U, pulse, t_start + n * dt, dt, form)
            psi, ia = lanczos_expm(Ha, psi, dt, m, eps_tol=eps_tol)
            psi, ib = lanczos_expm(Hb, psi, dt, m, eps_tol=eps_tol)
            m_eff.append(max(ia["m_eff"], ib["m_eff"]))
            deltas.append(max(ia["delta"], ib["delta"]))
        else:
            raise ValueError(f"unknown scheme {scheme}")
        docc.append(double_occupation(psi, w_d, Ns))
        norm2.append(float(np.vdot(psi, psi).real))
        if with_energy:
            t_n1 = t_start + (n + 1) * dt
            energy.append(energy_per_site(
                make_H(lattice, n_up, n_dn, U, pulse_A(t_n1, pulse), form),
                psi, Ns))
        if record_states:
            states.append(psi.copy())
    return {"psi": psi, "docc": np.array(docc), "norm2": np.array(norm2),
            "energy": np.array(energy), "m_eff": m_eff, "delta": deltas,
            "states": states}


def phase_fix(psi):
    """Multiply by a unit phase so the largest-|.| component is real > 0."""
    k = int(np.argmax(np.abs(psi)))
    return psi * (np.conj(psi[k]) / abs(psi[k]))


def ground_state(lattice, n_up, n_dn, U, k=4, tol=1e-14):
    """(E0, psi0, gap) of H(A=0); psi0 unit norm, phase-fixed."""
    H = make_H(lattice, n_up, n_dn, U, (0.0, 0.0, 0.0), form="auto")
    D = H.shape[0]
    if D <= 4000:
        lam, vec = np.linalg.eigh(H.toarray())
        E = lam[:2]
        psi = vec[:, 0]
    else:
        kk = min(k, D - 1)
        op = H if sp.issparse(H) else spla.LinearOperator(
            H.shape, matvec=H.dot, dtype=np.complex128)
        lam, vec = spla.eigsh(op, k=kk, which="SA", tol=tol)
        order = np.argsort(lam)
        lam, vec = lam[order], vec[:, order]
        E = lam[:2]
        psi = vec[:, 0]
    psi = phase_fix(psi / np.linalg.norm(psi))
    gap = float(E[1] - E[0]) if len(E) > 1 else float("inf")
    return float(E[0]), psi, gap
