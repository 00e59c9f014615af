"""Pins of the oracle's basis and ranks (CPU only).

Checked against: the count C(Ns,n) of Eq. (18), the printed Table 1, the
fermionic hash of Eq. (36) (read with 0-based sorted positions), and brute
force enumeration.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle.basis import popcount

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("Ns", range(1, 17))
def test_spin_basis_is_all_popcount_n_words_ascending(Ns):
    for n in range(Ns + 1):
        b = oracle.spin_basis(Ns, n)
        assert len(b) == math.comb(Ns, n)
        assert (np.diff(b.astype(np.int64)) > 0).all()
        assert (popcount(b) == n).all()


def test_spin_basis_matches_brute_force_small():
    for Ns in range(1, 9):
        for n in range(Ns + 1):
            brute = sorted(sum(1 << i for i in c)
                           for c in itertools.combinations(range(Ns), n))
            assert list(oracle.spin_basis(Ns, n).astype(int)) == brute


def hash_eq36(word, n):
    """Eq. (36): I = sum_k C(p_k, k), p_1 < ... < p_n the 0-based occupied sites."""
    pos = [i for i in range(64) if (word >> i) & 1]
    assert len(pos) == n
    return sum(math.comb(p, k + 1) for k, p in enumerate(pos))


@pytest.mark.parametrize("Ns", [4, 7, 10, 12])
def test_fermionic_hash_equals_ascending_rank(Ns):
    # Reading of Sec. 3.7 / Eq. (36): the hash enumerates the basis in the
    # same order as the oracle's sorted basis, and is a bijection onto
    # 0..C(Ns,n)-1.
    for n in range(Ns + 1):
        b = oracle.spin_basis(Ns, n)
        ranks = oracle.rank_of(b, b)
        hashes = np.array([hash_eq36(int(w), n) for w in b])
        assert (ranks == np.arange(len(b))).all()
        assert (hashes == ranks).all()


def test_lexicographic_multi_index_order_differs():
    # Eq. (21) orders multi-indices lexicographically on the sorted positions;
    # that order is NOT the ascending-word order the hash of Eq. (36) produces
    # (they first differ at Ns=4, n=2).  The build follows the hash.
    Ns, n = 4, 2
    lex = [sum(1 << i for i in c) for c in itertools.combinations(range(Ns), n)]
    asc = list(oracle.spin_basis(Ns, n).astype(int))
    assert sorted(lex) == asc and lex != asc


def test_rank_of_absent_words():
    b = oracle.spin_basis(6, 3)
    assert (oracle.rank_of(b, np.array([0, 1, 63], dtype=np.uint64)) == -1).all()


def test_table1_state_counts():
    tab = json.load(open(os.path.join(GOLDEN, "table1_dimensions.json")))
    for Ns, printed in zip(tab["Ns"], tab["N_states"]):
        du, dd, N = oracle.sector_dims(Ns, Ns // 2, Ns // 2)
        assert N == len(oracle.spin_basis(Ns, Ns // 2)) ** 2
        assert abs(N - printed) / printed < 0.05, (Ns, N, printed)


def test_table1_nnz_and_memory():
    # Eq. (22) for the all-to-all worst case, compared with Table 1 at the
    # printed precision; memory at 64 bytes per stored non-zero (four complex
    # double arrays), except the misprinted Ns=10 entry.
    tab = json.load(open(os.path.join(GOLDEN, "table1_dimensions.json")))
    for Ns, nnz_p, mem_p in zip(tab["Ns"], tab["N_nz"], tab["N_mem_GB"]):
        n = Ns // 2
        N = math.comb(Ns, n) ** 2
        nnz = N * (1 + 0.5 * n * (Ns - n) + 0.5 * n * (Ns - n))
        assert abs(nnz - nnz_p) / nnz_p < 0.05, (Ns, nnz, nnz_p)
        mem = nnz * 64 / 1e9
        if Ns == 10:
            assert abs(mem / 10 - mem_p) / mem_p < 0.1
        else:
            assert abs(mem - mem_p) / mem_p < 0.12, (Ns, mem, mem_p)
