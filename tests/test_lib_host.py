"""The C-ABI library on the host (no GPU): symbols, basis, tables, errors.

Basis words and connection tables are compared bit-exactly with the oracle:
the sparsity pattern of the tables equals that of the oracle's per-spin
hopping matrices, and at a generic vector potential every entry's group and
sign reproduce the oracle's value.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ed():
    from paper_2005_13498_gb300 import build
    build.build()
    from paper_2005_13498_gb300 import ed as mod
    return mod


def header_functions(name="ed.h"):
    src = open(os.path.join(ROOT, "include", name)).read()
    return sorted(set(re.findall(r"^\s*(?:ed_status|const char\*|int)\s+(ed_\w+)\s*\(",
                                 src, re.M)))


def test_library_exports_every_declared_symbol(ed):
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert headers == ["ed.h", "ed_probes.h"]
    names = header_functions("ed.h")
    assert len(names) >= 16
    for n in names:
        assert hasattr(ed.lib, n), n
    assert "sm_103a" in ed.ed_version()
    from paper_2005_13498_gb300 import probes
    for n in header_functions("ed_probes.h"):
        assert hasattr(probes.lib, n), n


def test_errors_without_gpu_work(ed):
    with pytest.raises(ed.EDError) as e:
        ed.ed_build_basis(17, 3, 3)
    assert e.value.status == 5
    with pytest.raises(ed.EDError) as e:
        ed.ed_build_basis(6, 7, 3)
    assert e.value.status == 1
    ctx = ed.ed_build_basis(4, 2, 2)
    bad = {"Ns": 4, "p": [0], "q": [0], "t": [1.0], "d": [[1, 0, 0]], "eps": None}
    with pytest.raises(ed.EDError) as e:
        ed.ed_set_lattice(ctx, bad, 1.0)
    assert e.value.status == 1 and "p == q" in str(e.value)
    bad = {"Ns": 4, "p": [0], "q": [9], "t": [1.0], "d": [[1, 0, 0]], "eps": None}
    with pytest.raises(ed.EDError):
        ed.ed_set_lattice(ctx, bad, 1.0)
    # calls before the lattice is set
    psi = np.zeros(36, dtype=np.complex128)
    with pytest.raises(ed.EDError) as e:
        ed.ed_propagate(ctx, psi, ed.ED_C128, None, 0.0, 0.01, 1, 4)
    assert e.value.status == 6
    ed.ed_set_lattice(ctx, synth.ring(4), 2.0)
    with pytest.raises(ed.EDError) as e:
        ed.ed_propagate(ctx, psi, ed.ED_C128, None, 0.0, 0.01, 1, 65)
    assert e.value.status == 5
    with pytest.raises(ed.EDError) as e:
        ed.ed_propagate(ctx, psi, ed.ED_C128, None, 0.0, 0.01, 1, 0)
    assert e.value.status == 1
    ed.ed_destroy(ctx)


@pytest.mark.parametrize("Ns", [1, 2, 5, 8, 12, 14, 16])
def test_basis_words_match_oracle(ed, Ns):
    for n in sorted({0, 1, Ns // 2, Ns - 1, Ns}):
        if not 0 <= n <= Ns:
            continue
        ctx = ed.ed_build_basis(Ns, n, max(0, Ns - n))
        du, dd = ed.ed_dims(ctx)
        assert du == len(oracle.spin_basis(Ns, n))
        assert np.array_equal(ed.ed_get_basis(ctx, 0).astype(np.uint64),
                              oracle.spin_basis(Ns, n))
        assert np.array_equal(ed.ed_get_basis(ctx, 1).astype(np.uint64),
                              oracle.spin_basis(Ns, max(0, Ns - n)))
        ed.ed_destroy(ctx)


def table_matrix(off, ent, coefs):
    """Dense matrix of a connection table: M[r, src] += sign * coef[group]."""
    dim = len(off) - 1
    M = np.zeros((dim, dim), dtype=complex)
    for r in range(dim):
        for e in ent[off[r]:off[r + 1]]:
            src = int(e) & 0xFFFF
            g = (int(e) >> 16) & 0xFF
            sgn = -1.0 if (int(e) >> 31) & 1 else 1.0
            M[r, src] += sgn * coefs[g]
    return M


def class_coefficients(lat, A):
    """Coefficients per group in the table's class order (first-seen order of
    distinct (t, d) bonds)."""
    classes = []
    for b in range(len(lat["p"])):
        key = (lat["t"][b], *lat["d"][b])
        if key not in classes:
            classes.append(key)
    c = []
    for key in classes:
        phi = np.dot(key[1:], A)
        c += [-key[0] * np.exp(-1j * phi), -key[0] * np.exp(1j * phi)]
    return np.array(c)


LATTICES = [
    ("ring8", synth.ring(8), [(4, 4), (3, 5)]),
    ("torus3x4", synth.torus(4, 3), [(6, 6), (5, 7)]),
    ("ladder2x7", synth.ladder(7), [(7, 7), (6, 8)]),
    ("complete6", synth.complete_graph(6, seed=4), [(3, 2)]),
    ("triangle", synth.triangle(), [(2, 1)]),
    ("chain5_eps", synth.chain(5, eps=[0.1, 0.2, -0.3, 0.0, 0.5]), [(2, 3)]),
]


@pytest.mark.parametrize("name,lat,sectors", LATTICES, ids=[x[0] for x in LATTICES])
def test_tables_match_oracle_bit_exact(ed, name, lat, sectors):
    A = np.array([0.31, -0.17, 0.23])
    for (nu, nd) in sectors:
        ctx = ed.ed_build_basis(lat["Ns"], nu, nd)
        ed.ed_set_lattice(ctx, lat, 3.0)
        for spin, n in ((0, nu), (1, nd)):
            off, ent, ncl = ed.ed_get_table(ctx, spin)
            T = oracle.spin_hopping_matrix(lat, n, A)
            dim = T.shape[0]
            if dim > 1000:
                # pattern and values row by row without a dense matrix
                coefs = class_coefficients(lat, A)
                Tc = T.tocsr()
                for r in range(0, dim, 7):
                    row = {}
                    for e in ent[off[r]:off[r + 1]]:
                        src = int(e) & 0xFFFF
                        g = (int(e) >> 16) & 0xFF
                        sgn = -1.0 if (int(e) >> 31) & 1 else 1.0
                        row[src] = row.get(src, 0) + sgn * coefs[g]
                    ref = dict(zip(Tc.indices[Tc.indptr[r]:Tc.indptr[r + 1]],
                                   Tc.data[Tc.indptr[r]:Tc.indptr[r + 1]]))
                    assert set(row) == set(ref)
                    for k in row:
                        assert abs(row[k] - ref[k]) < 1e-14
                continue
            M = table_matrix(off, ent, class_coefficients(lat, A))
            Td = T.toarray()
            assert np.array_equal(M != 0, Td != 0)
            assert np.abs(M - Td).max() < 1e-14
            # rows sorted by (group, source)
            for r in range(dim):
                es = [(int(e) >> 16 & 0xFF, int(e) & 0xFFFF) for e in ent[off[r]:off[r + 1]]]
                assert es == sorted(es)
        ed.ed_destroy(ctx)


def test_connection_counts_complete_graph(ed):
    # every single-electron hop allowed: n (Ns - n) entries per state (Eq. (22))
    Ns = 8
    lat = synth.complete_graph(Ns, seed=2)
    for n in range(Ns + 1):
        ctx = ed.ed_build_basis(Ns, n, 0)
        ed.ed_set_lattice(ctx, lat, 1.0)
        off, ent, ncl = ed.ed_get_table(ctx, 0)
        assert np.all(np.diff(off) == n * (Ns - n))
        ed.ed_destroy(ctx)


def test_apply_config_table_and_switch(ed):
    """The H v configuration table, and the process-wide switch that pins an
    entry (no GPU work: only the table and argument checks run here)."""
    n = ed.ed_apply_config_count()
    assert n >= 4
    seen = set()
    for c in range(n):
        i = ed.ed_apply_config_info(c)
        assert i["fp64"] in (0, 1) and i["split"] in (0, 1) and i["tma"] in (0, 1)
        assert i["rows_per_cta"] >= 1 and i["pairs_per_thread"] >= 1 and i["ctas_per_sm"] >= 1
        assert i["mv"] in (0, 1) and not (i["mv"] and (i["split"] or i["tma"]))
        seen.add((i["fp64"], i["split"]))
        if i["mv"]:
            seen.add(("mv", i["fp64"]))
    assert seen == {(0, 0), (0, 1), (1, 0), (1, 1), ("mv", 0), ("mv", 1)}
    for bad in (-2, n):
        with pytest.raises(ed.EDError) as e:
            ed.ed_set_apply_config(bad)
        assert e.value.status == 1
    with pytest.raises(ed.EDError):
        ed.ed_apply_config_info(n)
    ed.ed_set_apply_config(n - 1)
    ed.ed_set_apply_config(-1)
    h = ed.Hubbard(synth.ring(6), 3, 3, 2.0)
    assert ed.ed_get_apply_config(h.ctx) == (-1, -1)   # nothing set up yet
    h.close()


def test_krylov_tolerance_argument_checks(ed):
    h = ed.Hubbard(synth.ring(6), 3, 3, 2.0)
    ed.ed_set_krylov_tol(h.ctx, 1e-8)
    ed.ed_set_krylov_tol(h.ctx, 0.0)
    for bad in (-1e-3, float("nan"), float("inf")):
        with pytest.raises(ed.EDError) as e:
            ed.ed_set_krylov_tol(h.ctx, bad)
        assert e.value.status == 1
    h.close()


def test_integrator_argument_checks(ed):
    h = ed.Hubbard(synth.ring(6), 3, 3, 2.0)
    ed.ed_set_integrator(h.ctx, ed.ED_CFET4)
    ed.ed_set_integrator(h.ctx, "midpoint")
    with pytest.raises(ed.EDError) as e:
        ed.ed_set_integrator(h.ctx, 7)
    assert e.value.status == 1
    h.close()


def test_spectral_function_host_transform_matches_oracle(ed):
    """ed_spectral_function (host code of the library) against the oracle's
    broadened transform of Eq. (37)."""
    rng = np.random.default_rng(1)
    G = rng.standard_normal((101, 3, 2)) + 1j * rng.standard_normal((101, 3, 2))
    nu = np.linspace(-5, 5, 17)
    A = ed.ed_spectral_function(G, 0.05, 0.1, nu)
    ref = oracle.broadened_transform(G, 0.05, 0.1, nu)
    assert A.shape == ref.shape == (17, 3, 2)
    assert np.abs(A - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    for bad in ((0.0, 0.1), (0.05, -1.0)):
        with pytest.raises(ed.EDError):
            ed.ed_spectral_function(G, bad[0], bad[1], nu)


def test_device_verdict_refuses_foreign_devices(tmp_path):
    """Every GPU entry point refuses to launch when the current device is not
    the one the context's tables live on (ED_ERR_STATE) or when a caller's
    device buffer lives on another device (ED_ERR_ARG): the decision, compiled
    from csrc/device_guard.h and run on the host (one GPU cannot make the
    devices differ)."""
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    csrc = os.path.join(ROOT, "paper_2005_13498_gb300", "csrc")
    exe = str(tmp_path / "device_guard_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", csrc,
                    os.path.join(ROOT, "tests", "host", "device_guard_check.cpp"), "-o", exe],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = [tuple(int(x) for x in ln.split()) for ln in out if ln.strip()]
    ok, wrong_current, foreign = 0, 1, 2
    want = {(0, 0, -1): ok, (0, 0, 0): ok, (1, 1, 1): ok, (1, 1, -1): ok,
            (0, 1, -1): wrong_current, (1, 0, 0): wrong_current, (0, 1, 1): wrong_current,
            (0, 0, 1): foreign, (1, 1, 0): foreign, (2, 2, 3): foreign}
    assert len(got) == len(want)
    for c0, c1, c2, v in got:
        assert want[(c0, c1, c2)] == v, (c0, c1, c2, v)


def test_new_control_calls_validate_arguments(ed):
    ctx = ed.ed_build_basis(4, 2, 2)
    with pytest.raises(ed.EDError) as e:
        ed.ed_set_workspace_limit(ctx, -1)
    assert e.value.status == 1
    ed.ed_set_workspace_limit(ctx, 0)
    with pytest.raises(ed.EDError) as e:
        ed.ed_set_wait_fault(-2, 0)
    assert e.value.status == 1
    with pytest.raises(ed.EDError) as e:
        ed.ed_set_wait_fault(-1, -5)
    assert e.value.status == 1
    ed.ed_set_wait_fault(-1, 0)
    ed.ed_destroy(ctx)


STEP_CASES = [
    ("ring8", synth.lattice_from_name("ring8"), synth.workload("ring8")["pulse_params"]),
    ("torus3x4", synth.lattice_from_name("torus3x4"), synth.workload("torus3x4")["pulse_params"]),
    ("ladder2x7", synth.lattice_from_name("ladder2x7"),
     synth.workload("ladder2x7")["pulse_params"]),
    ("complete6", synth.complete_graph(6, seed=4),
     {"A0": 0.9, "omega": 3.0, "sigma": 0.7, "t0": 0.3, "dir": (0.3, -1.0, 0.5)}),
    ("triangle-cos-phase", synth.triangle(),
     {"A0": 0.8, "omega": 4.0, "sigma": 1.0, "t0": 0.5, "dir": (1.0, 0.0, 0.0),
      "shape": "cos_phase", "b": 0.3}),
]


@pytest.mark.parametrize("name,lat,pulse", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_step_coefficients_match_oracle(ed, name, lat, pulse):
    """The per-step hopping coefficients (S1) the propagation uploads, per
    bond, against the oracle's one-electron Hamiltonian h[q, p] at the
    midpoints (Eq. (32)) and, for CFET4, its two-field combinations: the
    sub-step tau times the coefficient equals dt (a2 h(A1) + a1 h(A2)), then
    dt (a1 h(A1) + a2 h(A2))."""
    ctx = ed.ed_build_basis(lat["Ns"], 1, 1)
    ed.ed_set_lattice(ctx, lat, 2.0)
    p, q = np.asarray(lat["p"]), np.asarray(lat["q"])
    nb = len(p)
    t0, dt, n = 0.13, 0.05, 7
    coef, tau = ed.ed_step_coefficients(ctx, nb, pulse, t0, dt, n)
    assert coef.shape == (n, nb) and tau == dt
    for s in range(n):
        h = oracle.single_particle_matrix(lat, oracle.pulse_A(t0 + (s + 0.5) * dt, pulse))
        assert np.abs(coef[s] - h[q, p]).max() <= 1e-15
    ed.ed_set_integrator(ctx, "cfet4")
    coef, tau = ed.ed_step_coefficients(ctx, nb, pulse, t0, dt, n)
    assert coef.shape == (2 * n, nb) and abs(tau - dt / 2) <= 1e-18
    (c1, c2), (a1, a2) = oracle.krylov.CFET4_C, oracle.krylov.CFET4_A
    for s in range(n):
        h1 = oracle.single_particle_matrix(lat, oracle.pulse_A(t0 + (s + c1) * dt, pulse))
        h2 = oracle.single_particle_matrix(lat, oracle.pulse_A(t0 + (s + c2) * dt, pulse))
        first, second = a2 * h1 + a1 * h2, a1 * h1 + a2 * h2
        assert np.abs(tau * coef[2 * s] - dt * first[q, p]).max() <= 1e-15
        assert np.abs(tau * coef[2 * s + 1] - dt * second[q, p]).max() <= 1e-15
    # no pulse: the bare hoppings -t_b
    ed.ed_set_integrator(ctx, "midpoint")
    coef, _ = ed.ed_step_coefficients(ctx, nb, None, 0.0, dt, 2)
    assert np.array_equal(coef, np.tile(-np.asarray(lat["t"], dtype=np.complex128), (2, 1)))
    ed.ed_destroy(ctx)


def test_step_coefficients_and_tridiag_expm_validate_arguments(ed):
    ctx = ed.ed_build_basis(4, 2, 2)
    with pytest.raises(ed.EDError) as e:
        ed.ed_step_coefficients(ctx, 4, None, 0.0, 0.02, 3)
    assert e.value.status == 6          # ED_ERR_STATE: no lattice yet
    ed.ed_set_lattice(ctx, synth.ring(4), 2.0)
    for n_steps, dt in ((0, 0.02), (3, float("nan"))):
        with pytest.raises(ed.EDError) as e:
            ed.ed_step_coefficients(ctx, 4, None, 0.0, dt, n_steps)
        assert e.value.status == 1
    bad_pulse = {"A0": 1.0, "omega": 1.0, "sigma": 0.0, "t0": 0.0, "dir": (1.0, 0, 0)}
    with pytest.raises(ed.EDError) as e:
        ed.ed_step_coefficients(ctx, 4, bad_pulse, 0.0, 0.02, 3)
    assert e.value.status == 1
    ed.ed_destroy(ctx)
    # the exponential checks its arguments before any device work
    for alpha, beta in ((np.zeros((1, 65)), np.zeros((1, 64))),
                        (np.array([[1.0, np.nan]]), np.array([[0.5]])),
                        (np.array([[1.0, 2.0]]), np.array([[np.inf]]))):
        with pytest.raises(ed.EDError) as e:
            ed.ed_tridiag_expm(alpha, beta, 0.1)
        assert e.value.status == 1
    with pytest.raises(ed.EDError) as e:
        ed.ed_tridiag_expm(np.array([[1.0]]), np.zeros((1, 0)), float("inf"))
    assert e.value.status == 1
