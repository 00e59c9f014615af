"""Host check of the apply's CTA order (no GPU).

The apply takes the up-spin rows in the order ``block_order(T, 1)`` returns,
a reverse Cuthill-McKee order of the graph in which two rows are adjacent
when one gathers from the other, and gives nr consecutive rows of that order
to each CTA.  Every row must appear exactly once (each row of w is written
by one CTA), and CTAs that run together (a window of consecutive CTAs) must
gather from fewer distinct rows than in natural order: that is the working
set the L2 has to hold.  The check is compiled from
``tests/host/block_order_check.cpp`` against ``tables.cpp``.
"""
import os
import shutil
import subprocess

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2005_13498_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    from paper_2005_13498_gb300 import build
    inc = os.path.join(build.cuda_home(), "include")
    exe = str(tmp_path_factory.mktemp("bo") / "block_order_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", CSRC, "-I", inc,
                    os.path.join(ROOT, "tests", "host", "block_order_check.cpp"),
                    os.path.join(CSRC, "tables.cpp"), "-o", exe], check=True)
    return exe


def run(exe, lat, n, nrs):
    p, q, t, d = lat["p"], lat["q"], lat["t"], lat["d"]
    lines = [f"{lat['Ns']} {n} {len(p)}"]
    for b in range(len(p)):
        dx, dy, dz = (float(v) for v in d[b])
        lines.append(f"{int(p[b])} {int(q[b])} {float(t[b]):.17g} {dx:.17g} {dy:.17g} {dz:.17g}")
    lines.append(" ".join(str(x) for x in nrs))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True,
                         text=True, check=True).stdout
    res = []
    for ln in out.strip().splitlines():
        a = ln.split()
        res.append((int(a[0]), int(a[1]), int(a[2]), float(a[3]), float(a[4]), int(a[5])))
    return res


@pytest.mark.parametrize("name,n", [("ladder2x7", 7), ("torus3x4", 6), ("ring8", 4)])
def test_block_order_is_a_permutation_with_a_smaller_working_set(checker, name, n):
    lat = synth.lattice_from_name(name)
    for nr, nblk, perm, u_nat, u_ord, maps_ok in run(checker, lat, n, [1, 2, 4]):
        assert perm == 1, (name, nr)
        assert maps_ok == 1, (name, nr)   # block maps cover every row (and chunk) once
        assert nblk > 1
        assert 0 < u_ord <= u_nat, (name, nr, u_nat, u_ord)
        if name == "ladder2x7":
            # the Ns=14 ladder: natural order touches about 82 % of the rows
            assert u_ord < 0.75 * u_nat, (nr, u_nat, u_ord)
