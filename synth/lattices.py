"""Bond lists for the lattices used by the tests and the benchmark.

Geometry only: site labels, bond endpoints, hopping magnitudes and bond
displacement vectors.  Sites are numbered 0..Ns-1; site i is bit i of a spin
configuration word.
"""
import numpy as np


def _pack(Ns, bonds, eps=None):
    p = np.array([b[0] for b in bonds], dtype=np.int32)
    q = np.array([b[1] for b in bonds], dtype=np.int32)
    t = np.array([b[2] for b in bonds], dtype=np.float64)
    d = np.array([b[3] for b in bonds], dtype=np.float64).reshape(len(bonds), 3)
    return {"Ns": int(Ns), "p": p, "q": q, "t": t, "d": d,
            "eps": None if eps is None else np.asarray(eps, dtype=np.float64)}


def ring(Ns, t=1.0):
    """Periodic 1D ring; bond i -> i+1 (mod Ns) has displacement +1 along x."""
    if Ns < 3:
        raise ValueError("a ring needs Ns >= 3 (use chain/dimer for 2 sites)")
    bonds = [(i, (i + 1) % Ns, t, (1.0, 0.0, 0.0)) for i in range(Ns)]
    return _pack(Ns, bonds)


def chain(Ns, t=1.0, eps=None):
    """Open 1D chain (OBC); bond i -> i+1, displacement +1 along x."""
    bonds = [(i, i + 1, t, (1.0, 0.0, 0.0)) for i in range(Ns - 1)]
    return _pack(Ns, bonds, eps)


def dimer(t=1.0):
    """Two sites, one bond (the Hubbard dimer)."""
    return chain(2, t)


def triangle(t=1.0):
    """Three sites on a closed loop (odd cycle; sign-sensitive)."""
    return ring(3, t)


def torus(Lx=4, Ly=3, t=1.0):
    """Lx x Ly square lattice, periodic in both directions, site = y*Lx + x.

    x bonds have displacement (1,0,0), y bonds (0,1,0).  Requires Lx, Ly >= 3
    so that no bond is doubled across the wrap.
    """
    if Lx < 3 or Ly < 3:
        raise ValueError("torus needs Lx, Ly >= 3")
    bonds = []
    for y in range(Ly):
        for x in range(Lx):
            s = y * Lx + x
            bonds.append((s, y * Lx + (x + 1) % Lx, t, (1.0, 0.0, 0.0)))
    for y in range(Ly):
        for x in range(Lx):
            s = y * Lx + x
            bonds.append((s, ((y + 1) % Ly) * Lx + x, t, (0.0, 1.0, 0.0)))
    return _pack(Lx * Ly, bonds)


def ladder(L=7, t_leg=1.0, t_rung=1.0):
    """Two-leg ladder, periodic along the legs, open rungs; site = leg*L + x.

    Leg bonds (leg*L+x -> leg*L+(x+1)%L) have displacement (1,0,0); rung bonds
    (x -> L+x) have displacement (0,1,0).
    """
    if L < 3:
        raise ValueError("periodic legs need L >= 3")
    bonds = []
    for leg in range(2):
        for x in range(L):
            bonds.append((leg * L + x, leg * L + (x + 1) % L, t_leg,
                          (1.0, 0.0, 0.0)))
    for x in range(L):
        bonds.append((x, L + x, t_rung, (0.0, 1.0, 0.0)))
    return _pack(2 * L, bonds)


def complete_graph(Ns, seed=1):
    """All-to-all hopping with generic magnitudes and displacements.

    Every pair of sites is bonded, so every single-electron hop is allowed; this
    is the worst case that Eq. (22) of the paper counts.
    """
    rng = np.random.default_rng(seed)
    bonds = []
    for i in range(Ns):
        for j in range(i + 1, Ns):
            bonds.append((i, j, 0.5 + rng.random(),
                          tuple(rng.standard_normal(3))))
    return _pack(Ns, bonds)


def lattice_from_name(name):
    """Named lattices of the workloads."""
    table = {
        "ring8": lambda: ring(8),
        "torus3x4": lambda: torus(4, 3),
        "ladder2x7": lambda: ladder(7),
        "torus4x4": lambda: torus(4, 4),
        "dimer": dimer,
        "triangle": triangle,
    }
    return table[name]()
