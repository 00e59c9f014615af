"""Write ground_energies.json: oracle ground-state energies of the workload
sectors (H at A = 0), used by the full-size GPU ground-state test.

    python tests/golden/make_ground_energies.py

Calls only ``oracle`` (scipy eigsh on the Kronecker-structured operator) and
``synth`` (the lattices).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

CASES = [("ladder2x7", 7, 7, 8.0), ("torus3x4", 6, 6, 8.0), ("ring8", 4, 4, 8.0)]


def main():
    out = {"generator": "tests/golden/make_ground_energies.py (oracle.ground_state)",
           "cases": []}
    for name, nu, nd, U in CASES:
        t = time.time()
        E0, psi, gap = oracle.ground_state(synth.lattice_from_name(name), nu, nd, U)
        out["cases"].append({"lattice": name, "n_up": nu, "n_dn": nd, "U": U,
                             "E0": E0, "gap": gap, "seconds": time.time() - t})
        print(out["cases"][-1], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                           "ground_energies.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
