"""Creation / annihilation between sectors and the G^< / G^> overlaps.

Oracle (test infrastructure only).

* Eqs. (7)-(8): c^+_{i s} and c_{i s} act on a Fock state with sign
  (-1)^{c_{i s}}, c_{i s} = number of occupied modes before mode (i, s).  With
  the block mode order of ``hamiltonian`` (all up modes, then all down modes)
  c_{i up} counts up electrons on sites < i, and c_{i dn} counts all n_up up
  electrons plus down electrons on sites < i.
* Sec. 3.7: after applying the operator, the index of the new state in the
  sector with one electron more / less is looked up (here by binary search in
  the sorted spin basis).
* Eq. (15) with reference time t = t_start:
      G^<_{ii s}(t, t') = i <psi(t')| c^+_{is} U(t', t) c_{is} |psi(t)>,
      G^>_{ii s}(t', t) = -i <psi(t')| c_{is} U(t', t) c^+_{is} |psi(t)>,
  so with phi = U(t_n, t) c psi(t) and phi' = U(t_n, t) c^+ psi(t), both
  propagated by the same midpoint scheme as psi:
      L_{is}(n) = <c_{is} psi(t_n) | phi_{is}(t_n)>,    G^< = i L,
      G_{is}(n) = <c^+_{is} psi(t_n) | phi'_{is}(t_n)>, G^> = -i G.
* Lehmann sums (Eq. (17) without the delta functions): at A = 0,
      L_{is}(t) = sum_phi |<phi|c_{is}|psi0>|^2 exp(-i (E_phi - E0) t),
  and the same with c^+ for G.
"""
import numpy as np

from .basis import spin_basis, rank_of, popcount
from .krylov import make_H, lanczos_expm, cfet4_factors
from .hamiltonian import pulse_A


def sector_shift(n_up, n_dn, op, spin):
    """Target sector of op in {'c', 'cdag'} acting on spin in {0 (up), 1 (dn)}."""
    dn = -1 if op == "c" else +1
    return (n_up + dn, n_dn) if spin == 0 else (n_up, n_dn + dn)


def _apply(Ns, n_up, n_dn, psi, site, spin, create):
    bu, bd = spin_basis(Ns, n_up), spin_basis(Ns, n_dn)
    du, dd = len(bu), len(bd)
    P = np.asarray(psi, dtype=np.complex128).reshape(du, dd)
    nu2, nd2 = sector_shift(n_up, n_dn, "cdag" if create else "c", spin)
    if not (0 <= nu2 <= Ns and 0 <= nd2 <= Ns):
        raise ValueError("target sector does not exist")
    bu2, bd2 = spin_basis(Ns, nu2), spin_basis(Ns, nd2)
    out = np.zeros((len(bu2), len(bd2)), dtype=np.complex128)
    bit = np.uint64(1 << site)
    below = np.uint64((1 << site) - 1)
    if spin == 0:
        occ = (bu & bit) != 0
        src = np.nonzero(~occ if create else occ)[0]
        x = bu[src]
        sgn = np.where(popcount(x & below) % 2 == 1, -1.0, 1.0)
        dst = rank_of(bu2, x ^ bit)
        out[dst, :] = sgn[:, None] * P[src, :]
    else:
        occ = (bd & bit) != 0
        src = np.nonzero(~occ if create else occ)[0]
        x = bd[src]
        sgn = np.where(popcount(x & below) % 2 == 1, -1.0, 1.0)
        sgn = sgn * (-1.0) ** n_up
        dst = rank_of(bd2, x ^ bit)
        out[:, dst] = P[:, src] * sgn[None, :]
    return out.reshape(-1)


def apply_c(Ns, n_up, n_dn, psi, site, spin):
    """c_{site,spin} psi, as a vector of the sector with one electron fewer."""
    return _apply(Ns, n_up, n_dn, psi, site, spin, create=False)


def apply_cdag(Ns, n_up, n_dn, psi, site, spin):
    """c^+_{site,spin} psi, as a vector of the sector with one electron more."""
    return _apply(Ns, n_up, n_dn, psi, site, spin, create=True)


def spectral_batch(lattice, n_up, n_dn, U, psi0, pulse, dt, n_steps, m,
                   t_start=0.0, sites=None, form="auto", eps_tol=None,
                   scheme="midpoint"):
    """L_{is}(n) and G_{is}(n) for n = 0..n_steps (arrays [n+1, Ns, 2]).

    psi is propagated in (n_up, n_dn); phi_{is} = c_{is} psi0 and
    phi'_{is} = c^+_{is} psi0 in their sectors, all with the same pulse, dt
    and Krylov dimension m (fixed, or at most m with the adaptive exit of
    Algorithm 6 when eps_tol is given, each vector on its own), by the
    midpoint rule or by CFET4 (scheme).  Sectors that
    do not exist (n = 0 or n = Ns) give zeros.
    """
    Ns = lattice["Ns"]
    sites = list(range(Ns)) if sites is None else list(sites)
    L = np.zeros((n_steps + 1, Ns, 2), dtype=np.complex128)
    G = np.zeros((n_steps + 1, Ns, 2), dtype=np.complex128)
    psi = np.asarray(psi0, dtype=np.complex128).reshape(-1).copy()
    phis, phids = {}, {}
    for i in sites:
        for s in (0, 1):
            tgt_c = sector_shift(n_up, n_dn, "c", s)
            tgt_d = sector_shift(n_up, n_dn, "cdag", s)
            if min(tgt_c) >= 0:
                phis[(i, s)] = apply_c(Ns, n_up, n_dn, psi, i, s)
            if max(tgt_d) <= Ns:
                phids[(i, s)] = apply_cdag(Ns, n_up, n_dn, psi, i, s)

    def record(n):
        for (i, s), ph in phis.items():
            L[n, i, s] = np.vdot(apply_c(Ns, n_up, n_dn, psi, i, s), ph)
        for (i, s), ph in phids.items():
            G[n, i, s] = np.vdot(apply_cdag(Ns, n_up, n_dn, psi, i, s), ph)

    record(0)

    def step(vec, nu2, nd2, n):
        if scheme == "cfet4":
            Ha, Hb = cfet4_factors(lattice, nu2, nd2, U, pulse, t_start + n * dt, dt, form)
            vec, _ = lanczos_expm(Ha, vec, dt, m, eps_tol=eps_tol)
            vec, _ = lanczos_expm(Hb, vec, dt, m, eps_tol=eps_tol)
            return vec
        A = pulse_A(t_start + (n + 0.5) * dt, pulse)
        vec, _ = lanczos_expm(make_H(lattice, nu2, nd2, U, A, form), vec, dt, m,
                              eps_tol=eps_tol)
        return vec

    for n in range(n_steps):
        psi = step(psi, n_up, n_dn, n)
        for (i, s) in list(phis):
            phis[(i, s)] = step(phis[(i, s)], *sector_shift(n_up, n_dn, "c", s), n)
        for (i, s) in list(phids):
            phids[(i, s)] = step(phids[(i, s)], *sector_shift(n_up, n_dn, "cdag", s), n)
        record(n + 1)
    return {"L": L, "G": G, "G_less": 1j * L, "G_greater": -1j * G,
            "psi": psi}


def lehmann_overlaps(lattice, n_up, n_dn, U, psi0, E0, times, site, spin):
    """Lehmann sums for L_{is}(t), G_{is}(t) at A = 0 by dense eigh."""
    Ns = lattice["Ns"]
    out = {}
    for op in ("c", "cdag"):
        nu2, nd2 = sector_shift(n_up, n_dn, op, spin)
        if not (0 <= nu2 <= Ns and 0 <= nd2 <= Ns):
            out[op] = np.zeros(len(times), dtype=np.complex128)
            continue
        H2 = make_H(lattice, nu2, nd2, U, (0.0, 0.0, 0.0), "csr").toarray()
        lam, vec = np.linalg.eigh(H2)
        x = (apply_c if op == "c" else apply_cdag)(Ns, n_up, n_dn, psi0,
                                                   site, spin)
        wts = np.abs(vec.conj().T @ x) ** 2
        out[op] = np.array([np.sum(wts * np.exp(-1j * (lam - E0) * t))
                            for t in times])
    return out["c"], out["cdag"]


def broadened_transform(G, dt, eps, nu):
    """Eq. (37), Sec. 3.7: A(nu) = (1/pi) Im int_0^T e^{-eps t}
    e^{i nu t} G(t) dt with T = (len(G) - 1) dt, the integral by the
    trapezoid rule over the samples G[k] = G(k dt).  G: [n+1, ...]."""
    G = np.asarray(G, dtype=np.complex128)
    t = np.arange(G.shape[0]) * dt
    out = []
    for v in np.atleast_1d(nu):
        f = (np.exp((-eps + 1j * v) * t)).reshape((-1,) + (1,) * (G.ndim - 1)) * G
        integral = dt * (f.sum(axis=0) - 0.5 * (f[0] + f[-1]))
        out.append(integral.imag / np.pi)
    return np.array(out)
