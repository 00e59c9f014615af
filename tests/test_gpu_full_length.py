"""Parity at the workloads' full lengths and sizes.

* 3x4 torus, (6,6), D = 853,776: 2000 midpoint steps (dt = 0.02, m = 20)
  from the oracle's ground state under the torus pulse, against the oracle's
  complex128 trajectory (tests/golden/torus3x4_2000.json, written by
  make_long_trajectories.py): complex128 <d> within 1e-10 and |psi|^2 within
  1e-10 at every step; complex64 (float32 vectors, float64 Lanczos scalars)
  <d> within 1e-5 at every step and norm drift within 1e-6, the bounds the
  float32 form has to meet.
* 2x7 ladder, (7,7), D = 11,778,624:
  - a 10-step prefix (m = 30, from a seeded state inside the pulse) against
    the oracle (tests/golden/ladder2x7_prefix.json): <d> and |psi|^2 at every
    step, and the final state at 1024 seeded indices (relative L2 over the
    sample: 1e-10 in complex128; 1e-5 in complex64, ten steps of float32
    rounding of about 1e-6 each);
  - 2000 steps from the ground state: complex64 <d> within 1e-5 of the
    complex128 path at every step (that path is pinned to the oracle by the
    prefix), complex64 norm drift within 1e-6, complex128 norm drift within
    1e-10.
  - the Green's functions of Eq. (15) for one site, both spins, all four
    operators, in the batch of 56 c / c^+ vectors plus psi, 2 steps from the
    reference time 9.6, against the oracle
    (tests/golden/ladder2x7_spectral_site3.json), complex64 within 1e-5.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import LATTICES, torch_cuda, to_dev, from_dev, ed_dtype

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_torus_2000_steps_against_oracle(ed_lib, parity_log):
    torch = torch_cuda()
    ed = ed_lib
    g = golden("torus3x4_2000.json")
    lat = LATTICES["torus3x4"]
    E0, psi0, gap = oracle.ground_state(lat, 6, 6, 8.0)
    assert abs(E0 - g["E0"]) <= 1e-10 * abs(E0)
    ref_docc, ref_n2 = np.array(g["docc"]), np.array(g["norm2"])
    h = ed.Hubbard(lat, 6, 6, 8.0)
    for dtype in ("c128", "c64"):
        x = to_dev(torch, psi0, dtype)
        out = ed.ed_propagate(h.ctx, x, ed_dtype(ed, dtype), g["pulse"], 0.0, g["dt"],
                              g["n_steps"], g["m"])
        torch.cuda.synchronize()
        e_d = float(np.abs(out["docc"] - ref_docc).max())
        drift = float(np.abs(out["norm2"] - out["norm2"][0]).max())
        parity_log(f"torus2000_{dtype}", docc_max_err=e_d, norm_drift=drift,
                   norm2_max_err=float(np.abs(out["norm2"] - ref_n2).max()),
                   drift_at_1000=out["norm2"][1000] - out["norm2"][0],
                   drift_at_2000=out["norm2"][2000] - out["norm2"][0])
        if dtype == "c128":
            assert e_d <= 1e-10
            assert np.abs(out["norm2"] - ref_n2).max() <= 1e-10
        else:
            assert e_d <= 1e-5
            assert drift <= 1e-6
    assert np.ptp(ref_docc) > 1e-3   # the pulse really drives the system
    h.close()


def test_ladder_prefix_against_oracle(ed_lib, parity_log):
    torch = torch_cuda()
    ed = ed_lib
    g = golden("ladder2x7_prefix.json")
    lat = LATTICES["ladder2x7"]
    psi0 = synth.complex_normal(3432 * 3432, 11)
    idx = np.array(g["index"])
    ref_amp = np.array(g["psi_re"]) + 1j * np.array(g["psi_im"])
    h = ed.Hubbard(lat, 7, 7, 8.0)
    for dtype, tol_state, tol_d in (("c128", 1e-10, 1e-10), ("c64", 1e-5, 1e-5)):
        x = to_dev(torch, psi0, dtype)
        out = ed.ed_propagate(h.ctx, x, ed_dtype(ed, dtype), g["pulse"], g["t_start"], g["dt"],
                              g["n_steps"], g["m"])
        torch.cuda.synchronize()
        amp = from_dev(x[torch.from_numpy(idx).cuda()])
        e_s = float(np.linalg.norm(amp - ref_amp) / np.linalg.norm(ref_amp))
        e_d = float(np.abs(out["docc"] - np.array(g["docc"])).max())
        drift = float(np.abs(out["norm2"] - out["norm2"][0]).max())
        parity_log(f"ladder_prefix10_{dtype}", state_sample_rel_l2=e_s, docc_max_err=e_d,
                   norm_drift=drift)
        assert e_s <= tol_state, dtype
        assert e_d <= tol_d, dtype
        assert np.abs(out["norm2"] - np.array(g["norm2"])).max() <= (1e-10 if dtype == "c128"
                                                                      else 1e-6)
        assert list(out["m_eff"]) == g["m_eff"]
    h.close()


def test_ladder_2000_steps_c64_against_c128(ed_lib, parity_log):
    torch = torch_cuda()
    ed = ed_lib
    w = synth.workload("ladder2x7")
    lat = LATTICES["ladder2x7"]
    h = ed.Hubbard(lat, 7, 7, 8.0)
    g = torch.zeros(h.D, dtype=torch.complex128, device="cuda")
    ed.ed_ground_state(h.ctx, g, tol=1e-10, max_iter=3000)
    outs = {}
    for dtype in ("c128", "c64"):
        x = g.clone() if dtype == "c128" else g.to(torch.complex64)
        outs[dtype] = ed.ed_propagate(h.ctx, x, ed_dtype(ed, dtype), w["pulse_params"], 0.0,
                                      w["dt"], w["n_steps"], w["m"])
        torch.cuda.synchronize()
        del x
    d128, d64 = outs["c128"]["docc"], outs["c64"]["docc"]
    e_d = float(np.abs(d64 - d128).max())
    drift64 = float(np.abs(outs["c64"]["norm2"] - outs["c64"]["norm2"][0]).max())
    drift128 = float(np.abs(outs["c128"]["norm2"] - outs["c128"]["norm2"][0]).max())
    n64 = outs["c64"]["norm2"] - outs["c64"]["norm2"][0]
    parity_log("ladder2000_c64_vs_c128", docc_max_err=e_d, norm_drift_c64=drift64,
               norm_drift_c128=drift128, drift_c64_at_500=n64[500], drift_c64_at_1000=n64[1000],
               drift_c64_at_2000=n64[2000], max_step_change_c64=np.abs(np.diff(n64)).max())
    assert len(d128) == 2001
    assert e_d <= 1e-5
    assert drift64 <= 1e-6
    assert drift128 <= 1e-10
    assert np.ptp(d128) > 1e-3
    h.close()


def test_ladder_spectral_site_against_oracle(ed_lib, parity_log):
    torch_cuda()
    ed = ed_lib
    g = golden("ladder2x7_spectral_site3.json")
    lat = LATTICES["ladder2x7"]
    psi0 = synth.complex_normal(3432 * 3432, 31)
    h = ed.Hubbard(lat, 7, 7, 8.0)
    Gl, Gg = ed.ed_spectral_propagate_at(h.ctx, psi0, g["t_ref"], ed.ED_C64, g["pulse"],
                                         g["dt"], g["n_steps"], g["m"], 14)
    i = g["site"]
    rl = np.array(g["G_less_re"]) + 1j * np.array(g["G_less_im"])
    rg = np.array(g["G_greater_re"]) + 1j * np.array(g["G_greater_im"])
    e_l = float(np.abs(Gl[:, i, :] - rl).max())
    e_g = float(np.abs(Gg[:, i, :] - rg).max())
    parity_log("ladder_spectral_site3_c64", G_less_max_err=e_l, G_greater_max_err=e_g)
    assert e_l <= 1e-5 and e_g <= 1e-5
    # sum rule at the reference time on every site: L(0) + G(0) = <psi|psi>
    n2 = float(np.vdot(psi0, psi0).real)
    for site in range(14):
        for s in (0, 1):
            assert abs(Gl[0, site, s] / 1j + Gg[0, site, s] / -1j - n2) <= 1e-5
    h.close()
