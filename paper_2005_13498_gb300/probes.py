"""ctypes binding of libed_probes.so (include/ed_probes.h): measured on-chip
ceilings of the current device, reported by the benchmark beside the
roofline of the H v kernel.  Argument marshalling only."""
import ctypes
import os

from . import build as _build


class ed_ceilings(ctypes.Structure):
    _fields_ = [("l2_read_gbs", ctypes.c_double), ("hbm_read_gbs", ctypes.c_double),
                ("smem_read_gbs", ctypes.c_double), ("fp32_fma_tflops", ctypes.c_double),
                ("fp32x2_fma_tflops", ctypes.c_double), ("fp64_fma_tflops", ctypes.c_double),
                ("sms", ctypes.c_int)]


def _load():
    path = _build.probes_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2005_13498_gb300.build`")
    lib = ctypes.CDLL(path)
    lib.ed_probe_ceilings.argtypes = [ctypes.POINTER(ed_ceilings)]
    lib.ed_probe_ceilings.restype = ctypes.c_int
    lib.ed_probe_shared_loads.argtypes = []
    lib.ed_probe_shared_loads.restype = ctypes.c_int
    return lib


lib = _load()


def ed_probe_ceilings():
    """dict of the measured ceilings (see include/ed_probes.h)."""
    c = ed_ceilings()
    rc = lib.ed_probe_ceilings(ctypes.byref(c))
    if rc != 0:
        raise RuntimeError(f"ed_probe_ceilings failed with CUDA error {rc}")
    return {k: getattr(c, k) for k, _ in ed_ceilings._fields_}


def ed_probe_shared_loads():
    """Launch the four shared-memory load-pattern kernels (include/ed_probes.h)."""
    rc = lib.ed_probe_shared_loads()
    if rc != 0:
        raise RuntimeError(f"ed_probe_shared_loads failed with CUDA error {rc}")
