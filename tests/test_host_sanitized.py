"""The table builder (tables.cpp) under AddressSanitizer and
UndefinedBehaviorSanitizer, on the host (no GPU): every particle number of
several lattices up to Ns=16, each table checked against its definition
(tests/host/tables_check.cpp): basis order and combinadic ranks, every
entry a hop of a bond with its Jordan-Wigner sign and every hop present,
padded rows, the warp-tiled ELL column by column, the CTA order, the c / c+
maps, and conjugate coefficient pairs."""
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
    exe = str(tmp_path_factory.mktemp("tc") / "tables_check")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-g", "-fno-omit-frame-pointer",
                        "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                        "-I", CSRC, "-I", inc,
                        os.path.join(ROOT, "tests", "host", "tables_check.cpp"),
                        os.path.join(CSRC, "tables.cpp"), "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtime not available: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr
    return exe


LATS = [("ring8", synth.ring(8)), ("torus3x4", synth.lattice_from_name("torus3x4")),
        ("ladder2x5", synth.ladder(5)), ("complete7", synth.complete_graph(7, seed=2)),
        ("triangle", synth.triangle()), ("chain5", synth.chain(5)), ("dimer", synth.dimer()),
        ("torus4x4", synth.lattice_from_name("torus4x4"))]


@pytest.mark.parametrize("name,lat", LATS, ids=[x[0] for x in LATS])
def test_tables_under_sanitizers(checker, name, lat):
    lines = [f"{lat['Ns']} {len(lat['p'])}"]
    for b in range(len(lat["p"])):
        dx, dy, dz = (float(v) for v in lat["d"][b])
        lines.append(f"{int(lat['p'][b])} {int(lat['q'][b])} {float(lat['t'][b]):.17g} "
                     f"{dx:.17g} {dy:.17g} {dz:.17g}")
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([checker], input="\n".join(lines) + "\n", capture_output=True,
                       text=True, env=env, timeout=600)
    assert r.returncode == 0, (r.stdout[-500:], r.stderr[-2000:])
    assert r.stdout.startswith("ok "), r.stdout
    assert int(r.stdout.split()[1]) > 100
