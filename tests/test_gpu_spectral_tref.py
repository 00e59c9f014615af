"""GPU parity of the Green's functions at a reference time t_ref > 0
(ed_spectral_propagate_at, Eq. (15)) with the paper's own hopping phase of
Eq. (4) (pulse shape "cos_phase"), and of A(nu, t_ref) of Eq. (37) through
the library's transform, against the oracle.
complex128: 1e-9 on G, 1e-8 on A.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import LATTICES, torch_cuda, to_dev

pytestmark = pytest.mark.gpu


def test_spectral_at_reference_time_matches_oracle(ed_lib):
    torch = torch_cuda()
    ed = ed_lib
    lat = LATTICES["ring6"]
    U, dt, t_ref, n_ref, n = 4.0, 0.05, 0.4, 8, 12
    pulse = {"A0": 0.6, "omega": 5.0, "sigma": 1.0, "t0": 0.5, "dir": (1.0, 0.0, 0.0),
             "shape": "cos_phase", "b": float(np.cos(5.0 * 0.5))}
    E0, psi0, _ = oracle.ground_state(lat, 3, 3, U)
    # oracle: psi(t_ref) by the midpoint rule, then the batch from t_ref
    pr = oracle.propagate(lat, 3, 3, U, psi0, pulse, dt, n_ref, 16)["psi"]
    ref = oracle.spectral_batch(lat, 3, 3, U, pr, pulse, dt, n, 16, t_start=t_ref)
    # the same two stages through the C ABI
    h = ed.Hubbard(lat, 3, 3, U)
    x = to_dev(torch, psi0, "c128")
    ed.ed_propagate(h.ctx, x, ed.ED_C128, pulse, 0.0, dt, n_ref, 16)
    Gl, Gg = ed.ed_spectral_propagate_at(h.ctx, x, t_ref, ed.ED_C128, pulse, dt, n, 16, 6)
    torch.cuda.synchronize()
    h.close()
    assert np.abs(Gl - ref["G_less"]).max() <= 1e-9
    assert np.abs(Gg - ref["G_greater"]).max() <= 1e-9
    assert np.abs(ref["G_less"][1:] - ref["G_less"][0]).max() > 1e-3   # not trivial
    nu = np.linspace(-10.0, 10.0, 41)
    A = ed.ed_spectral_function(Gl, dt, 0.3, nu) + ed.ed_spectral_function(Gg, dt, 0.3, nu)
    Ar = (oracle.broadened_transform(ref["G_less"], dt, 0.3, nu) +
          oracle.broadened_transform(ref["G_greater"], dt, 0.3, nu))
    assert np.abs(A - Ar).max() <= 1e-8
