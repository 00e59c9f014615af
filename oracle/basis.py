"""Spin bases of a fixed-particle-number sector (oracle; test infrastructure).

Sec. 3.1 of the paper: H^{n_up}_{n_dn}(Ns) is identified with
H^{n_up}_0 (x) H^0_{n_dn} (Eq. (18)), so a sector state is a pair of spin
configurations, each an Ns-bit word with bit i = occupation of site i.

Ordering (reading of Sec. 3.1 and Eq. (36)): the spin basis is the set of all
Ns-bit words with n set bits in ascending integer order.  The fermionic hash
of Eq. (36) "directly corresponds to the ordering" of states; with 0-based
sorted positions p_1 < ... < p_n it is the combinatorial number system, which
enumerates popcount-n words in ascending integer order.  The oracle finds a
rank by binary search in the sorted array (``rank_of``), never by the hash
formula, so the tests can check the hash reading against it.

Sector index of the pair (u, d) is rank_up(u) * dim_dn + rank_dn(d): Psi is a
dim_up x dim_dn matrix stored row-major.
"""
import math
import numpy as np


def binom(n, k):
    if k < 0 or k > n:
        return 0
    return math.comb(n, k)


def spin_basis(Ns, n):
    """All Ns-bit words with exactly n ones, ascending (uint64 array)."""
    if not (0 <= n <= Ns):
        raise ValueError("need 0 <= n <= Ns")
    words = np.arange(1 << Ns, dtype=np.uint64)
    # popcount by bit loop: plain and obviously correct
    pc = np.zeros(words.shape, dtype=np.int64)
    for b in range(Ns):
        pc += ((words >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return words[pc == n]


def rank_of(basis, words):
    """Position of each word in the sorted basis; -1 where absent."""
    words = np.asarray(words, dtype=np.uint64)
    idx = np.searchsorted(basis, words)
    idx_c = np.minimum(idx, len(basis) - 1)
    ok = (idx < len(basis)) & (basis[idx_c] == words)
    return np.where(ok, idx, -1).astype(np.int64)


def sector_dims(Ns, n_up, n_dn):
    """(dim_up, dim_dn, N_states) with N_states = C(Ns,n_up) C(Ns,n_dn), Eq. (18)."""
    du, dd = binom(Ns, n_up), binom(Ns, n_dn)
    return du, dd, du * dd


def popcount(words):
    words = np.asarray(words, dtype=np.uint64)
    pc = np.zeros(words.shape, dtype=np.int64)
    w = words.copy()
    for _ in range(64):
        pc += (w & np.uint64(1)).astype(np.int64)
        w = w >> np.uint64(1)
        if not w.any():
            break
    return pc
