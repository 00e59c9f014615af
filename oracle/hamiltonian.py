"""Sparse Hubbard Hamiltonian in one (n_up, n_dn) sector (oracle; test infra).

Model (Sec. 2.1, Eq. (1)):  H = - sum_{i,j,sigma} v_ji c^+_{i sigma} c_{j sigma}
                                + U sum_i n_{i up} n_{i dn}.
v_ji is the amplitude of a hop from site j to site i.  A bond b = (p, q, t_b,
d_b) of the lattice contributes v_qp = v_pq = t_b; diagonal entries become an
on-site energy eps_i = -v_ii, added as eps_i (n_{i up} + n_{i dn}).

Peierls substitution (Sec. 2.2, Eq. (3)) with a spatially uniform vector
potential A(t) (e = 1):  v_ij(t) = v_ij exp(-i A(t).(R_j - R_i)).  The term
that moves an electron from p to q is -v_qp(t) c^+_q c_p with
v_qp(t) = t_b exp(-i A.(R_q - R_p)) = t_b exp(-i A.d_b), so its matrix element
is  -t_b exp(-i A.d_b) * sign,  and the reverse hop q -> p carries the complex
conjugate.  (Reading: the paper's sign convention; the phase of the q->p hop is
the conjugate, so H is Hermitian.)

Fermion sign (Sec. 2.3, Eqs. (7)-(8); Sec. 3.3, Eq. (26)): modes are ordered
all spin-up sites 0..Ns-1 first, then all spin-down sites.  Moving a spin-sigma
electron from p to q gives (-1)^(number of occupied sigma-modes strictly between
p and q); the other spin's modes lie entirely before or after both and cancel.
(Reading: the paper orders modes site-interleaved, Eq. (6); that order differs
from this one by a diagonal +-1 gauge, pinned by a test, and leaves spectra and
every observable used here unchanged.)

Pulse (workload definition): A(t) = A0 exp(-(t-t0)^2/(2 sigma^2))
sin(Omega (t-t0)) * dir, the vector potential whose time derivative is the
field of Eq. (2) up to the envelope derivative.
"""
import numpy as np
import scipy.sparse as sp

from .basis import spin_basis, rank_of, popcount


def pulse_A(t, pulse):
    """Vector potential A(t) (3-vector) of a pulse.

    shape "sin" (default): A0 exp(-s^2/(2 sigma^2)) sin(omega s) dir, s = t - t0.
    shape "cos_phase": the paper's phase function of Eq. (4) written as a
    vector potential, A(t) = -A0 [cos(omega s) - b] exp(-s^2/(2 sigma^2)) dir,
    so a hop along dir (d_b . dir = 1) carries f(t) = exp(i a [cos(omega
    (t - t_p)) - b] e^{-(t-t_p)^2/(2 sigma^2)}) with a = A0, t_p = t0.
    """
    if pulse is None:
        return np.zeros(3)
    s = t - pulse["t0"]
    env = np.exp(-s * s / (2.0 * pulse["sigma"] ** 2))
    if pulse.get("shape", "sin") == "cos_phase":
        amp = -pulse["A0"] * (np.cos(pulse["omega"] * s) - pulse.get("b", 0.0)) * env
    else:
        amp = pulse["A0"] * env * np.sin(pulse["omega"] * s)
    return amp * np.asarray(pulse["dir"], dtype=np.float64)


def bond_phases(lattice, A):
    """phi_b = A . d_b for every bond."""
    return np.asarray(lattice["d"], dtype=np.float64) @ np.asarray(A, dtype=np.float64)


def spin_hopping_matrix(lattice, n, A):
    """T_sigma for one spin species with n electrons (dim x dim, complex CSR).

    Entry [rank(x'), rank(x)] for the hop p -> q of bond b on configuration x
    (bit p set, bit q clear; x' = x ^ 2^p ^ 2^q) is
        -t_b exp(-i phi_b) (-1)^{popcount(x & between(p, q))},
    and the hop q -> p on configurations with bit q set and bit p clear has
    -t_b exp(+i phi_b) times its own sign.
    """
    Ns = lattice["Ns"]
    basis = spin_basis(Ns, n)
    dim = len(basis)
    phi = bond_phases(lattice, A)
    rows, cols, vals = [], [], []
    for b in range(len(lattice["p"])):
        p, q = int(lattice["p"][b]), int(lattice["q"][b])
        tb = float(lattice["t"][b])
        lo, hi = min(p, q), max(p, q)
        between = np.uint64(((1 << hi) - 1) & ~((1 << (lo + 1)) - 1))
        for (src, dst, coef) in ((p, q, -tb * np.exp(-1j * phi[b])),
                                 (q, p, -tb * np.exp(+1j * phi[b]))):
            bs, bd = np.uint64(1 << src), np.uint64(1 << dst)
            active = ((basis & bs) != 0) & ((basis & bd) == 0)
            x = basis[active]
            xn = x ^ bs ^ bd
            sign = np.where(popcount(x & between) % 2 == 1, -1.0, 1.0)
            rows.append(rank_of(basis, xn))
            cols.append(np.nonzero(active)[0])
            vals.append(coef * sign)
    if rows:
        r = np.concatenate(rows)
        c = np.concatenate(cols)
        v = np.concatenate(vals)
    else:
        r = c = np.zeros(0, dtype=np.int64)
        v = np.zeros(0, dtype=np.complex128)
    assert (r >= 0).all()
    return sp.csr_matrix((v, (r, c)), shape=(dim, dim), dtype=np.complex128)


def double_occupancy_weights(Ns, n_up, n_dn):
    """(w_d)_k = number of doubly occupied sites of sector state k (Sec. 3.5)."""
    bu, bd = spin_basis(Ns, n_up), spin_basis(Ns, n_dn)
    return popcount(bu[:, None] & bd[None, :]).astype(np.float64).ravel()


def diag_U(lattice, n_up, n_dn, U):
    """Diagonal of H: U * #doubles + sum_i eps_i (n_i_up + n_i_dn)."""
    Ns = lattice["Ns"]
    dg = U * double_occupancy_weights(Ns, n_up, n_dn)
    eps = lattice.get("eps")
    if eps is not None:
        bu, bd = spin_basis(Ns, n_up), spin_basis(Ns, n_dn)
        eu = np.array([sum(eps[i] for i in range(Ns) if (int(x) >> i) & 1)
                       for x in bu])
        ed = np.array([sum(eps[i] for i in range(Ns) if (int(x) >> i) & 1)
                       for x in bd])
        dg = dg + (eu[:, None] + ed[None, :]).ravel()
    return dg


def build_H(lattice, n_up, n_dn, U, A=(0.0, 0.0, 0.0)):
    """Full sector Hamiltonian H(A) as complex CSR (dim_up*dim_dn square).

    H = kron(T_up, 1) + kron(1, T_dn) + diag, matching the row-major
    index k = rank_up * dim_dn + rank_dn.
    """
    Tu = spin_hopping_matrix(lattice, n_up, A)
    Td = spin_hopping_matrix(lattice, n_dn, A)
    du, dd = Tu.shape[0], Td.shape[0]
    H = sp.kron(Tu, sp.identity(dd, format="csr")) + \
        sp.kron(sp.identity(du, format="csr"), Td) + \
        sp.diags(diag_U(lattice, n_up, n_dn, U))
    H = H.tocsr()
    H.sum_duplicates()
    herm = abs(H - H.getH())
    assert herm.nnz == 0 or herm.max() < 1e-14, "H not Hermitian"
    return H


def single_particle_matrix(lattice, A=(0.0, 0.0, 0.0)):
    """Ns x Ns one-electron Hamiltonian h[q, p] = -t_b exp(-i A.d_b) (p -> q)."""
    Ns = lattice["Ns"]
    phi = bond_phases(lattice, A)
    h = np.zeros((Ns, Ns), dtype=np.complex128)
    for b in range(len(lattice["p"])):
        p, q, tb = int(lattice["p"][b]), int(lattice["q"][b]), lattice["t"][b]
        h[q, p] += -tb * np.exp(-1j * phi[b])
        h[p, q] += -tb * np.exp(+1j * phi[b])
    eps = lattice.get("eps")
    if eps is not None:
        h += np.diag(eps)
    return h
