"""The small exponential of Algorithm 6 (the float64 device routine of the
propagation's exponential kernel) against the oracle's eigendecomposition
form, on random real symmetric tridiagonals: orders 1 to 64, time steps
that need one or many Taylor sub-steps, wide and narrow spectra, and the
near-eigenvector case of a Lanczos step (tiny off-diagonals)."""
import numpy as np
import pytest

import oracle
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _batch(rng, batch, n, a_scale, b_scale, b_min=0.0):
    alpha = rng.normal(0.0, a_scale, (batch, n))
    beta = np.abs(rng.normal(0.0, b_scale, (batch, max(0, n - 1)))) + b_min
    return alpha, beta


@pytest.mark.parametrize("n", [1, 2, 3, 12, 20, 30, 33, 64])
@pytest.mark.parametrize("tau,a_scale,b_scale", [(0.02, 3.0, 1.5), (0.5, 3.0, 1.5),
                                                 (3.0, 10.0, 4.0), (0.02, 40.0, 0.3)])
def test_tridiag_expm_matches_oracle(ed_lib, n, tau, a_scale, b_scale):
    torch_cuda()
    rng = np.random.default_rng(1000 * n + int(100 * tau))
    alpha, beta = _batch(rng, 7, n, a_scale, b_scale)
    y = ed_lib.ed_tridiag_expm(alpha, beta, tau)
    for b in range(alpha.shape[0]):
        ref = oracle.small_expm_e1(alpha[b], beta[b], tau)
        # float64 rounding of the series and of the shift's phase, times the
        # number of sub-steps (tau * spectral half width / 0.5)
        half = 0.5 * (np.ptp(alpha[b]) + 4 * (beta[b].max() if n > 1 else 0.0)) + 1.0
        tol = 1e-14 * max(1.0, tau * half)
        assert np.abs(y[b] - ref).max() <= tol, (b, np.abs(y[b] - ref).max(), tol)
        assert abs(np.linalg.norm(y[b]) - 1.0) <= tol


def test_tridiag_expm_near_eigenvector(ed_lib):
    """A Lanczos step from a near-eigenvector: beta_1 ~ 1e-7 relative, the
    rest of T arbitrary.  The tiny component y_2 (of the order of tau beta_1)
    is resolved and the norm stays 1 to rounding."""
    torch_cuda()
    rng = np.random.default_rng(7)
    n, tau = 30, 0.02
    alpha = rng.normal(0.0, 4.0, (1, n))
    beta = np.abs(rng.normal(0.0, 2.0, (1, n - 1)))
    beta[0, 0] = 7e-7
    y = ed_lib.ed_tridiag_expm(alpha, beta, tau)[0]
    ref = oracle.small_expm_e1(alpha[0], beta[0], tau)
    assert np.abs(y - ref).max() <= 1e-14
    assert abs(y[1] - ref[1]) <= 1e-6 * abs(ref[1])
    assert 0.5 * tau * 7e-7 < abs(y[1]) < 2.0 * tau * 7e-7
    assert abs(np.linalg.norm(y) - 1.0) <= 1e-15
