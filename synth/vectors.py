"""Seeded random vectors (inputs only)."""
import numpy as np


def complex_normal(D, seed=0):
    """D standard normals for the real part, then D for the imaginary part.

    Drawn from ``numpy.random.default_rng(seed)`` in that order and scaled to
    unit 2-norm in float64.
    """
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(D)
    im = rng.standard_normal(D)
    v = re + 1j * im
    return v / np.sqrt(np.vdot(v, v).real)


def random_state(dim_up, dim_dn, seed=0, nvec=1):
    """Unit-norm complex128 vectors shaped (nvec, dim_up, dim_dn)."""
    out = np.empty((nvec, dim_up, dim_dn), dtype=np.complex128)
    for k in range(nvec):
        out[k] = complex_normal(dim_up * dim_dn, seed + k).reshape(dim_up, dim_dn)
    return out
