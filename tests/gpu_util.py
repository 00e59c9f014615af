"""Helpers shared by the GPU parity tests (not collected as tests)."""
import numpy as np

import synth


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def to_dev(torch, x, dtype):
    """numpy complex -> contiguous CUDA tensor of complex128 / complex64."""
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128))
    if dtype == "c64":
        t = t.to(torch.complex64)
    return t.cuda().contiguous()


def from_dev(t):
    return t.detach().cpu().to(dtype=t.dtype).numpy().astype(np.complex128)


def rel_l2(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_el(a, b):
    """Largest element error relative to the largest reference element:
    max_k |a_k - b_k| / max_k |b_k| (a local error, e.g. in a few rows,
    cannot hide under the norm of a large vector)."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# Per-element bound of the apply tests, relative to max |w|: complex128 ~
# rounding of a sum of at most 2 * 19 + 1 terms; complex64 about 40 float32
# roundings of 6e-8 on terms no larger than the largest |w|, with margin.
TOL_EL = {"c128": 1e-13, "c64": 5e-6}


def ed_dtype(ed, name):
    return ed.ED_C128 if name == "c128" else ed.ED_C64


LATTICES = {
    "ring8": synth.ring(8),
    "torus3x4": synth.torus(4, 3),
    "ladder2x7": synth.ladder(7),
    "triangle": synth.triangle(),
    "dimer": synth.dimer(),
    "chain6_eps": synth.chain(6, eps=[0.2, -0.1, 0.0, 0.3, -0.4, 0.1]),
    "complete7": synth.complete_graph(7, seed=3),
    "ring6": synth.ring(6),
    "ring16": synth.ring(16),
}
