"""The benchmark workloads (lattice, sector, U, pulse, stepping).

Pulse: A(t) = A0 * exp(-(t - t0)^2 / (2 sigma^2)) * sin(Omega (t - t0)) * dir.
The field direction ``dir`` is used unnormalised, so on the 3x4 torus with
dir = (1, 1, 0) every nearest-neighbour bond carries a Peierls phase of
magnitude |A(t)|.
"""

PULSES = {
    "ring8": {"A0": 0.5, "omega": 8.0, "sigma": 2.0, "t0": 5.0,
              "dir": (1.0, 0.0, 0.0)},
    "torus3x4": {"A0": 0.5, "omega": 8.0, "sigma": 2.0, "t0": 5.0,
                 "dir": (1.0, 1.0, 0.0)},
    "ladder2x7": {"A0": 0.5, "omega": 8.0, "sigma": 2.0, "t0": 10.0,
                  "dir": (1.0, 0.0, 0.0)},
    "torus4x4": {"A0": 0.5, "omega": 8.0, "sigma": 2.0, "t0": 5.0,
                 "dir": (1.0, 1.0, 0.0)},
}

WORKLOADS = {
    # Ns=8 periodic ring, (4,4), dim 70x70
    "ring8": {"lattice": "ring8", "n_up": 4, "n_dn": 4, "U": 8.0,
              "pulse": "ring8", "dt": 0.02, "n_steps": 500, "m": 12,
              "dtypes": ["c128"]},
    # Ns=12 3x4 torus, (6,6), dim 924x924
    "torus3x4": {"lattice": "torus3x4", "n_up": 6, "n_dn": 6, "U": 8.0,
                 "pulse": "torus3x4", "dt": 0.02, "n_steps": 2000, "m": 20,
                 "dtypes": ["c128", "c64"]},
    # Ns=14 2x7 ladder, (7,7), dim 3432x3432
    "ladder2x7": {"lattice": "ladder2x7", "n_up": 7, "n_dn": 7, "U": 8.0,
                  "pulse": "ladder2x7", "dt": 0.02, "n_steps": 2000, "m": 30,
                  "dtypes": ["c128", "c64"]},
    # Ns=12 torus spectral batch: 48 vectors in (7,6),(6,7),(5,6),(6,5)
    "torus3x4_spectral": {"lattice": "torus3x4", "n_up": 6, "n_dn": 6,
                          "U": 8.0, "pulse": "torus3x4", "dt": 0.02,
                          "n_steps": 1000, "m": 20, "dtypes": ["c64"]},
    # Ns=16 4x4 torus at half filling, (8,8), dim 12870x12870 = 165,636,900:
    # the matrix-free sector beyond the paper's CSR memory limit (Sec. 4)
    "torus4x4": {"lattice": "torus4x4", "n_up": 8, "n_dn": 8, "U": 8.0,
                 "pulse": "torus4x4", "dt": 0.02, "n_steps": 2000, "m": 30,
                 "dtypes": ["c64", "c128"]},
    # Ns=14 ladder spectral batch: 56 vectors of dim 3003x3432 / 3432x3003
    "ladder2x7_spectral": {"lattice": "ladder2x7", "n_up": 7, "n_dn": 7,
                           "U": 8.0, "pulse": "ladder2x7", "dt": 0.02,
                           "n_steps": 1000, "m": 20, "dtypes": ["c64"]},
}


def workload(name):
    w = dict(WORKLOADS[name])
    w["pulse_params"] = dict(PULSES[w["pulse"]])
    return w
