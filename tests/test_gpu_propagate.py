"""GPU parity of ed_propagate against the oracle's midpoint-rule trajectory.

Same discrete scheme on both sides (fixed m, same breakdown rule, same pulse
at the midpoints), so complex128 agrees to rounding: state relative L2 and
<d> within 1e-10.  complex64 (float32 vectors, float64 Lanczos scalars):
<d> within 1e-5 and norm drift within 1e-6 of the complex128 oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import LATTICES, torch_cuda, to_dev, from_dev, rel_l2, ed_dtype

pytestmark = pytest.mark.gpu


def run_gpu(ed, torch, lat, nu, nd, U, psi0, pulse, dt, n, m, dtype, energy=False,
            host=False, profile=False):
    h = ed.Hubbard(lat, nu, nd, U)
    if host == "pinned":
        # pinned host memory: read and written by the library's permutation
        # kernel over the host link
        x = torch.from_numpy(np.array(psi0, dtype=np.complex128 if dtype == "c128"
                                      else np.complex64, copy=True)).pin_memory()
        out = ed.ed_propagate(h.ctx, x, ed_dtype(ed, dtype), pulse, 0.0, dt, n, m,
                              energy=energy, profile=profile)
        psi = x.numpy().astype(np.complex128)
    elif host:
        # a private copy: the library writes the result into this buffer
        x = np.array(psi0, dtype=np.complex128 if dtype == "c128" else np.complex64,
                     copy=True)
        out = ed.ed_propagate(h.ctx, x, ed_dtype(ed, dtype), pulse, 0.0, dt, n, m,
                              energy=energy, profile=profile)
        psi = x.astype(np.complex128)
    else:
        xd = to_dev(torch, psi0, dtype)
        out = ed.ed_propagate(h.ctx, xd, ed_dtype(ed, dtype), pulse, 0.0, dt, n, m,
                              energy=energy, profile=profile)
        torch.cuda.synchronize()
        psi = from_dev(xd)
    h.close()
    return psi, out


def test_ring8_full_trajectory_c128(ed_lib, parity_log):
    """Ns=8 ring, (4,4), U=8, 500 steps dt=0.02, m=12, pulse A0=0.5 Omega=8
    sigma=2 t0=5: the whole trajectory against the oracle."""
    torch = torch_cuda()
    w = synth.workload("ring8")
    lat = LATTICES["ring8"]
    E0, psi0, gap = oracle.ground_state(lat, 4, 4, 8.0)
    ref = oracle.propagate(lat, 4, 4, 8.0, psi0, w["pulse_params"], 0.02, 500, 12,
                           with_energy=True)
    psi, out = run_gpu(ed_lib, torch, lat, 4, 4, 8.0, psi0, w["pulse_params"], 0.02,
                       500, 12, "c128", energy=True)
    parity_log("ring8_500_c128", state_rel_l2=rel_l2(psi, ref["psi"]),
               docc_max_err=np.abs(out["docc"] - ref["docc"]).max(),
               norm2_max_err=np.abs(out["norm2"] - ref["norm2"]).max(),
               energy_max_err=np.abs(out["energy"] - ref["energy"]).max())
    assert rel_l2(psi, ref["psi"]) <= 1e-10
    assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-10
    assert np.abs(out["norm2"] - ref["norm2"]).max() <= 1e-10
    assert np.abs(out["energy"] - ref["energy"]).max() <= 1e-10
    assert np.array_equal(out["m_eff"], np.array(ref["m_eff"]))
    assert np.ptp(ref["docc"]) > 1e-3  # the pulse really excites the system


def test_ring8_trajectory_c64(ed_lib, parity_log):
    torch = torch_cuda()
    w = synth.workload("ring8")
    lat = LATTICES["ring8"]
    E0, psi0, gap = oracle.ground_state(lat, 4, 4, 8.0)
    ref = oracle.propagate(lat, 4, 4, 8.0, psi0, w["pulse_params"], 0.02, 500, 12)
    psi, out = run_gpu(ed_lib, torch, lat, 4, 4, 8.0, psi0, w["pulse_params"], 0.02,
                       500, 12, "c64")
    parity_log("ring8_500_c64", state_rel_l2=rel_l2(psi, ref["psi"]),
               docc_max_err=np.abs(out["docc"] - ref["docc"]).max(),
               norm_drift=np.abs(out["norm2"] - out["norm2"][0]).max())
    assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-5
    assert np.abs(out["norm2"] - out["norm2"][0]).max() <= 1e-6
    assert rel_l2(psi, ref["psi"]) <= 1e-4


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_torus_prefix(ed_lib, dtype, parity_log):
    """Ns=12 3x4 torus, (6,6), m=20, dt=0.02: first 12 steps (D = 853,776)."""
    torch = torch_cuda()
    w = synth.workload("torus3x4")
    lat = LATTICES["torus3x4"]
    psi0 = synth.complex_normal(924 * 924, 7)
    # start late in the pulse so the field is strong
    pulse = dict(w["pulse_params"], t0=0.1)
    ref = oracle.propagate(lat, 6, 6, 8.0, psi0, pulse, 0.02, 12, 20)
    psi, out = run_gpu(ed_lib, torch, lat, 6, 6, 8.0, psi0, pulse, 0.02, 12, 20, dtype)
    parity_log(f"torus_prefix12_{dtype}", state_rel_l2=rel_l2(psi, ref["psi"]),
               docc_max_err=np.abs(out["docc"] - ref["docc"]).max(),
               norm_drift=np.abs(out["norm2"] - out["norm2"][0]).max())
    if dtype == "c128":
        assert rel_l2(psi, ref["psi"]) <= 1e-10
        assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-10
    else:
        assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-5
        assert np.abs(out["norm2"] - out["norm2"][0]).max() <= 1e-6
        assert rel_l2(psi, ref["psi"]) <= 1e-5


def test_ladder_full_size_one_step(ed_lib, parity_log):
    """Ns=14 ladder, (7,7), m=30: one full midpoint step at t=10 (pulse
    maximum region) in both dtypes against the oracle, every element."""
    torch = torch_cuda()
    w = synth.workload("ladder2x7")
    lat = LATTICES["ladder2x7"]
    psi0 = synth.complex_normal(3432 * 3432, 11)
    t_start = 9.6
    ref = oracle.propagate(lat, 7, 7, 8.0, psi0, w["pulse_params"], 0.02, 1, 30,
                           t_start=t_start)
    for dtype, tol in (("c128", 1e-10), ("c64", 2e-6)):
        h = ed_lib.Hubbard(lat, 7, 7, 8.0)
        xd = to_dev(torch, psi0, dtype)
        out = ed_lib.ed_propagate(h.ctx, xd, ed_dtype(ed_lib, dtype), w["pulse_params"],
                                  t_start, 0.02, 1, 30)
        torch.cuda.synchronize()
        parity_log(f"ladder_one_step_{dtype}", state_rel_l2=rel_l2(from_dev(xd), ref["psi"]),
                   docc_err=abs(out["docc"][1] - ref["docc"][1]))
        assert rel_l2(from_dev(xd), ref["psi"]) <= tol, dtype
        assert abs(out["docc"][1] - ref["docc"][1]) <= (1e-10 if dtype == "c128" else 1e-6)
        h.close()


def test_atomic_limit_breakdown(ed_lib):
    """t = 0: exact phases exp(-i U w_d t) and the same breakdown as the oracle."""
    torch = torch_cuda()
    lat = synth.ring(6, t=0.0)
    D = oracle.sector_dims(6, 3, 3)[2]
    psi0 = synth.complex_normal(D, 2)
    psi, out = run_gpu(ed_lib, torch, lat, 3, 3, 8.0, psi0, None, 0.02, 25, 12, "c128")
    w = oracle.double_occupancy_weights(6, 3, 3)
    assert np.abs(psi - np.exp(-1j * 8.0 * w * 0.5) * psi0).max() <= 1e-12
    assert out["m_eff"].max() <= 4


def test_stationary_ground_state(ed_lib):
    torch = torch_cuda()
    lat = LATTICES["ring6"]
    E0, psi0, gap = oracle.ground_state(lat, 3, 3, 4.0)
    psi, out = run_gpu(ed_lib, torch, lat, 3, 3, 4.0, psi0, None, 0.05, 40, 12, "c128",
                       energy=True)
    assert np.abs(psi - np.exp(-1j * E0 * 2.0) * psi0).max() <= 1e-11
    assert np.ptp(out["docc"]) <= 1e-12
    assert np.abs(out["energy"] - E0 / 6).max() <= 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_host_pointer_and_profile_paths(ed_lib, dtype):
    """Pageable host buffers (copied in and out by the library), pinned host
    buffers (read and written by its permutation kernel) and the profiled
    launch path give the same result as device buffers with a CUDA graph."""
    torch = torch_cuda()
    lat = LATTICES["triangle"]
    pulse = {"A0": 0.7, "omega": 3.0, "sigma": 1.0, "t0": 0.3, "dir": (1.0, 0, 0)}
    psi0 = synth.complex_normal(3 * 3, 5)
    a, oa = run_gpu(ed_lib, torch, lat, 2, 1, 2.0, psi0, pulse, 0.05, 20, 6, dtype)
    b, ob = run_gpu(ed_lib, torch, lat, 2, 1, 2.0, psi0, pulse, 0.05, 20, 6, dtype, host=True)
    c, oc = run_gpu(ed_lib, torch, lat, 2, 1, 2.0, psi0, pulse, 0.05, 20, 6, dtype,
                    profile=True)
    d, od = run_gpu(ed_lib, torch, lat, 2, 1, 2.0, psi0, pulse, 0.05, 20, 6, dtype,
                    host="pinned")
    assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, d)
    assert np.array_equal(oa["docc"], ob["docc"]) and np.array_equal(oa["docc"], od["docc"])
    assert oc["kernel_launches"][0] > 0 and oc["kernel_ms"][0] > 0


@pytest.mark.parametrize("name,nu,nd,dtype", [("ladder2x7", 7, 7, "c64"),
                                               ("ring7", 3, 2, "c128")])
def test_pinned_host_state_equals_device_state(ed_lib, name, nu, nd, dtype):
    """A pinned host state, read and written by the permutation kernel over
    the host link, ends bit-equal to the same state kept on the device: the
    Ns=14 ladder (rows of 3432 columns, every column moved by the hop order)
    and a 7-site ring with rows of 21 columns."""
    torch = torch_cuda()
    if name == "ring7":
        lat = synth.ring(7)
        pulse = {"A0": 0.5, "omega": 8.0, "sigma": 2.0, "t0": 0.2, "dir": (1.0, 0, 0)}
    else:
        lat = LATTICES[name]
        pulse = synth.workload(name)["pulse_params"]
    D = oracle.sector_dims(lat["Ns"], nu, nd)[2]
    psi0 = synth.complex_normal(D, 21)
    a, oa = run_gpu(ed_lib, torch, lat, nu, nd, 8.0, psi0, pulse, 0.02, 2, 12, dtype)
    b, ob = run_gpu(ed_lib, torch, lat, nu, nd, 8.0, psi0, pulse, 0.02, 2, 12, dtype,
                    host="pinned")
    assert np.array_equal(a, b)
    assert np.array_equal(oa["docc"], ob["docc"]) and np.array_equal(oa["norm2"], ob["norm2"])


def test_repeated_calls_reuse_and_resume(ed_lib):
    """Two calls of 10 steps equal one call of 20 steps (same graph reused;
    the scheme is Markov in (psi, t_n))."""
    torch = torch_cuda()
    lat = LATTICES["ring8"]
    pulse = synth.workload("ring8")["pulse_params"]
    psi0 = synth.complex_normal(4900, 1)
    h = ed_lib.Hubbard(lat, 4, 4, 8.0)
    x1 = to_dev(torch, psi0, "c128")
    ed_lib.ed_propagate(h.ctx, x1, ed_lib.ED_C128, pulse, 4.0, 0.02, 20, 12)
    x2 = to_dev(torch, psi0, "c128")
    ed_lib.ed_propagate(h.ctx, x2, ed_lib.ED_C128, pulse, 4.0, 0.02, 10, 12)
    ed_lib.ed_propagate(h.ctx, x2, ed_lib.ED_C128, pulse, 4.2, 0.02, 10, 12)
    torch.cuda.synchronize()
    assert rel_l2(from_dev(x2), from_dev(x1)) <= 1e-13
    h.close()


def test_zero_steps_and_observables(ed_lib):
    torch = torch_cuda()
    lat = LATTICES["chain6_eps"]
    psi0 = synth.complex_normal(oracle.sector_dims(6, 3, 3)[2], 8) * 1.3
    psi, out = run_gpu(ed_lib, torch, lat, 3, 3, 2.5, psi0, None, 0.02, 0, 5, "c128")
    w = oracle.double_occupancy_weights(6, 3, 3)
    assert abs(out["docc"][0] - oracle.double_occupation(psi0, w, 6)) <= 1e-13
    assert abs(out["norm2"][0] - 1.69) <= 1e-12
    assert np.array_equal(psi, psi0)
