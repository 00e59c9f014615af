"""The error paths of the propagation calls, made to happen without faulting
or hanging the GPU, each followed by a normal call on the same context.

* A non-finite state: the observation kernel finds |psi|^2 not finite and
  the call returns ED_ERR_NUMERIC.
* A workspace cap below what the Krylov storage needs: ED_ERR_OOM before
  anything is allocated (propagation and ground state).
* A bounded device-side wait that runs out: with the test hook of
  ed_set_wait_fault, the producer warp of a TMA configuration of the H v
  kernel stops before one T_up row copy, the consumer warps' wait for it
  gives up after a few thousand polls, and ed_propagate returns
  ED_ERR_TIMEOUT.  No copy is left in flight (the producer waits for the
  copies it issued), so the context stays usable: the next call, on the same
  TMA configuration, matches the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import LATTICES, torch_cuda, to_dev, from_dev, rel_l2

pytestmark = pytest.mark.gpu

PULSE = {"A0": 0.6, "omega": 5.0, "sigma": 1.0, "t0": 0.2, "dir": (1.0, 1.0, 0.0)}


def test_non_finite_state_is_reported_and_context_recovers(ed_lib):
    torch = torch_cuda()
    ed = ed_lib
    lat = LATTICES["ring8"]
    h = ed.Hubbard(lat, 4, 4, 8.0)
    psi0 = synth.complex_normal(h.D, 3)
    bad = psi0.copy()
    bad[5] = np.nan
    x = to_dev(torch, bad, "c128")
    with pytest.raises(ed.EDError) as e:
        ed.ed_propagate(h.ctx, x, ed.ED_C128, PULSE, 0.0, 0.02, 2, 8)
    assert e.value.status == 7
    ref = oracle.propagate(lat, 4, 4, 8.0, psi0, PULSE, 0.02, 2, 8)
    x = to_dev(torch, psi0, "c128")
    out = ed.ed_propagate(h.ctx, x, ed.ED_C128, PULSE, 0.0, 0.02, 2, 8)
    torch.cuda.synchronize()
    assert rel_l2(from_dev(x), ref["psi"]) <= 1e-10
    assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-10
    h.close()


def test_workspace_cap_returns_oom_and_context_recovers(ed_lib):
    torch = torch_cuda()
    ed = ed_lib
    lat = LATTICES["ring8"]
    h = ed.Hubbard(lat, 4, 4, 8.0)
    psi0 = synth.complex_normal(h.D, 4)
    # m = 12 complex128: 11 Krylov slots + one scratch vector of 4900 elements
    ed.ed_set_workspace_limit(h.ctx, 11 * 16 * h.D)
    x = to_dev(torch, psi0, "c128")
    with pytest.raises(ed.EDError) as e:
        ed.ed_propagate(h.ctx, x, ed.ED_C128, PULSE, 0.0, 0.02, 2, 12)
    assert e.value.status == 3 and "workspace limit" in str(e.value)
    g = torch.zeros(h.D, dtype=torch.complex128, device="cuda")
    ed.ed_set_workspace_limit(h.ctx, 4 * 16 * h.D)        # fewer than two Lanczos vectors
    with pytest.raises(ed.EDError) as e:
        ed.ed_ground_state(h.ctx, g, tol=1e-10)
    assert e.value.status == 3
    ed.ed_set_workspace_limit(h.ctx, 12 * 16 * h.D)       # exactly enough
    ref = oracle.propagate(lat, 4, 4, 8.0, psi0, PULSE, 0.02, 2, 12)
    out = ed.ed_propagate(h.ctx, x, ed.ED_C128, PULSE, 0.0, 0.02, 2, 12)
    torch.cuda.synchronize()
    assert rel_l2(from_dev(x), ref["psi"]) <= 1e-10
    assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-10
    ed.ed_set_workspace_limit(h.ctx, 0)
    h.close()


def _tma_config(ed, fp64):
    for i in range(ed.ed_apply_config_count()):
        info = ed.ed_apply_config_info(i)
        if info["tma"] and info["fp64"] == fp64 and not info["split"]:
            return i
    pytest.skip("no TMA configuration in the table")


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_tma_wait_timeout_returns_status_and_context_recovers(ed_lib, dtype):
    torch = torch_cuda()
    ed = ed_lib
    lat = LATTICES["torus3x4"]
    code = ed.ED_C128 if dtype == "c128" else ed.ED_C64
    cfg = _tma_config(ed, 1 if dtype == "c128" else 0)
    psi0 = synth.complex_normal(924 * 924, 17)
    h = ed.Hubbard(lat, 6, 6, 8.0)           # dim_dn = 924: even rows, TMA allowed
    try:
        ed.ed_set_apply_config(cfg)
        ed.ed_set_wait_fault(3, 2000)
        x = to_dev(torch, psi0, dtype)
        with pytest.raises(ed.EDError) as e:
            ed.ed_propagate(h.ctx, x, code, PULSE, 0.0, 0.02, 1, 4)
        assert e.value.status == 4
        ed.ed_set_wait_fault(-1, 0)
        x = to_dev(torch, psi0, dtype)
        out = ed.ed_propagate(h.ctx, x, code, PULSE, 0.0, 0.02, 1, 4)
        torch.cuda.synchronize()
        assert ed.ed_get_apply_config(h.ctx)[0] == cfg
        ref = oracle.propagate(lat, 6, 6, 8.0, psi0, PULSE, 0.02, 1, 4)
        tol = 1e-10 if dtype == "c128" else 2e-6
        assert rel_l2(from_dev(x), ref["psi"]) <= tol
        assert abs(out["docc"][1] - ref["docc"][1]) <= (1e-10 if dtype == "c128" else 1e-6)
    finally:
        ed.ed_set_wait_fault(-1, 0)
        ed.ed_set_apply_config(-1)
        h.close()
