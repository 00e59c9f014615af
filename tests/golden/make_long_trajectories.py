"""Write the oracle reference values of the full-length parity tests.

    python tests/golden/make_long_trajectories.py torus2000     # ~50 min
    python tests/golden/make_long_trajectories.py ladder_prefix # ~5 min
    python tests/golden/make_long_trajectories.py ladder_site   # ~5 min

Calls only ``oracle`` (float64 NumPy/SciPy) and ``synth`` (lattices, pulses,
seeded vectors); nothing here touches the CUDA library.

* ``torus2000``  -> torus3x4_2000.json: the 3x4 torus, (6,6), U = 8, from the
  oracle's ground state of H(A = 0) at t = 0, 2000 midpoint steps (Eq. (32))
  of dt = 0.02 with fixed Krylov dimension m = 20 (Algorithm 6) under the
  torus pulse; <d>(t_n) (Eq. (13)) and |psi(t_n)|^2 for n = 0..2000.
* ``ladder_prefix`` -> ladder2x7_prefix.json: the 2x7 ladder, (7,7), U = 8,
  from the seed-11 complex-normal state at t = 9.6 (inside the pulse), 10
  midpoint steps, m = 30; <d> and |psi|^2 for n = 0..10 and the amplitudes of
  the final state at 1024 seeded indices (D = 11,778,624 is too large to
  store).
* ``ladder_site`` -> ladder2x7_spectral_site3.json: the Green's functions of
  Eq. (15) for site 3, both spins, from the seed-31 complex-normal state of
  the ladder's (7,7) sector at the reference time 9.6: c / c^+ applied, the
  four vectors and psi propagated 2 steps (dt = 0.02, m = 20), G^< and G^>
  for n = 0..2.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _write(name, obj):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(obj, f, indent=0)


def torus2000():
    w = synth.workload("torus3x4")
    lat = synth.lattice_from_name(w["lattice"])
    t = time.time()
    E0, psi0, gap = oracle.ground_state(lat, 6, 6, 8.0)
    r = oracle.propagate(lat, 6, 6, 8.0, psi0, w["pulse_params"], 0.02, 2000, 20)
    _write("torus3x4_2000.json", {
        "generator": "tests/golden/make_long_trajectories.py torus2000",
        "lattice": "torus3x4", "n_up": 6, "n_dn": 6, "U": 8.0, "dt": 0.02,
        "n_steps": 2000, "m": 20, "t_start": 0.0, "pulse": w["pulse_params"],
        "start": "oracle.ground_state of H(A=0)", "E0": E0, "gap": gap,
        "docc": r["docc"].tolist(), "norm2": r["norm2"].tolist(),
        "m_eff_min": int(min(r["m_eff"])), "seconds": time.time() - t})


def ladder_prefix():
    w = synth.workload("ladder2x7")
    lat = synth.lattice_from_name(w["lattice"])
    D = 3432 * 3432
    psi0 = synth.complex_normal(D, 11)
    t = time.time()
    r = oracle.propagate(lat, 7, 7, 8.0, psi0, w["pulse_params"], 0.02, 10, 30,
                         t_start=9.6, form="kron")
    idx = np.sort(np.random.default_rng(12345).choice(D, 1024, replace=False))
    amp = r["psi"][idx]
    _write("ladder2x7_prefix.json", {
        "generator": "tests/golden/make_long_trajectories.py ladder_prefix",
        "lattice": "ladder2x7", "n_up": 7, "n_dn": 7, "U": 8.0, "dt": 0.02,
        "n_steps": 10, "m": 30, "t_start": 9.6, "pulse": w["pulse_params"],
        "start": "synth.complex_normal(D, 11)",
        "docc": r["docc"].tolist(), "norm2": r["norm2"].tolist(),
        "index": idx.tolist(), "psi_re": amp.real.tolist(), "psi_im": amp.imag.tolist(),
        "m_eff": [int(x) for x in r["m_eff"]], "seconds": time.time() - t})


def ladder_site():
    w = synth.workload("ladder2x7")
    lat = synth.lattice_from_name(w["lattice"])
    psi0 = synth.complex_normal(3432 * 3432, 31)
    t = time.time()
    r = oracle.spectral_batch(lat, 7, 7, 8.0, psi0, w["pulse_params"], 0.02, 2, 20,
                              t_start=9.6, sites=[3], form="kron")
    gl, gg = r["G_less"][:, 3, :], r["G_greater"][:, 3, :]
    _write("ladder2x7_spectral_site3.json", {
        "generator": "tests/golden/make_long_trajectories.py ladder_site",
        "lattice": "ladder2x7", "n_up": 7, "n_dn": 7, "U": 8.0, "dt": 0.02,
        "n_steps": 2, "m": 20, "t_ref": 9.6, "pulse": w["pulse_params"], "site": 3,
        "start": "synth.complex_normal(D, 31)",
        "G_less_re": gl.real.tolist(), "G_less_im": gl.imag.tolist(),
        "G_greater_re": gg.real.tolist(), "G_greater_im": gg.imag.tolist(),
        "seconds": time.time() - t})


if __name__ == "__main__":
    {"torus2000": torus2000, "ladder_prefix": ladder_prefix,
     "ladder_site": ladder_site}[sys.argv[1]]()
