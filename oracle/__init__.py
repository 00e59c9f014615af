"""FP64 CPU oracle for the time-dependent Hubbard ED hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (``paper_2005_13498_gb300``) and imports nothing
from it; the two meet only in the seeded inputs of ``synth``.

What it computes, following the paper (Innerberger, Worm, Prauhart, Kauch,
"Electron-light interaction in nonequilibrium: exact diagonalization for time
dependent Hubbard Hamiltonians", arXiv:2005.13498):

* ``basis``       spin bases of H^{n_up}_{n_dn} (Sec. 3.1, Eq. (18)), ranks.
* ``hamiltonian`` H(t) = T_up(t) (x) 1 + 1 (x) T_dn(t) + U sum n_up n_dn as a
                  scipy CSR matrix, with Peierls phases (Sec. 2.1-2.2,
                  Eqs. (1), (3); Sec. 3.2-3.3, Eq. (26) for the fermion sign).
* ``krylov``      fixed-m Lanczos approximation of exp(-i tau H) v
                  (Sec. 3.4, Algorithm 6), the exponential midpoint rule
                  (Eq. (32)), the trajectory with observables (Sec. 3.5,
                  Eqs. (13)-(14)), and the ground state (Sec. 3.4).
* ``spectral``    c / c^dagger maps between sectors (Sec. 3.7, Eqs. (7)-(8)),
                  the G^< / G^> overlaps of Eq. (15) and Lehmann sums (Eq. (17)).

Every function is pinned by a ``-m "not gpu"`` test against closed forms,
brute force or printed values (see tests/test_oracle_*.py).  Parity pinned for
all functions listed above.
"""
from .basis import spin_basis, rank_of, sector_dims, binom
from .hamiltonian import (pulse_A, bond_phases, spin_hopping_matrix,
                          build_H, diag_U, double_occupancy_weights,
                          single_particle_matrix)
from .krylov import (lanczos_expm, propagate, ground_state, small_expm_e1,
                     double_occupation, energy_per_site, cfet4_factors,
                     epsilon_estimate, CFET4_A, CFET4_C)
from .spectral import (broadened_transform, apply_c, apply_cdag, sector_shift, spectral_batch,
                       lehmann_overlaps)

__all__ = [
    "spin_basis", "rank_of", "sector_dims", "binom", "pulse_A", "bond_phases",
    "spin_hopping_matrix", "build_H", "diag_U", "double_occupancy_weights",
    "single_particle_matrix", "lanczos_expm", "broadened_transform", "propagate", "ground_state",
    "cfet4_factors", "epsilon_estimate", "CFET4_A", "CFET4_C",
    "small_expm_e1", "double_occupation", "energy_per_site", "apply_c",
    "apply_cdag", "sector_shift", "spectral_batch", "lehmann_overlaps",
]
