"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds geometry (bond lists), pulse parameters, workload
descriptions and seeded random vectors.  It contains none of the method's
arithmetic: no basis, no Hamiltonian, no phases, no propagation.  Both the
CPU oracle (``oracle/``) and the CUDA path consume what it produces, and
neither imports the other.

A lattice is a dict with keys

* ``Ns``       number of sites,
* ``p``, ``q`` int arrays, the two sites of every bond (0-based),
* ``t``        float array, hopping magnitude t_b of every bond,
* ``d``        (n_bonds, 3) float array, displacement r_q - r_p of the bond
               (minimum image across a periodic wrap),
* ``eps``      optional (Ns,) on-site energies, or None.

The paper encodes geometry in the hopping matrix v (Sec. 2.1, Eq. (1)); a bond
list with magnitudes and displacement vectors is the same information plus the
positions the Peierls phase of Eq. (3) needs.
"""
from .lattices import (ring, chain, torus, ladder, complete_graph, dimer,
                       triangle, lattice_from_name)
from .workloads import WORKLOADS, workload, PULSES
from .vectors import complex_normal, random_state

__all__ = [
    "ring", "chain", "torus", "ladder", "complete_graph", "dimer", "triangle",
    "lattice_from_name", "WORKLOADS", "workload", "PULSES", "complex_normal",
    "random_state",
]
