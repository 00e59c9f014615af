"""The on-chip probes of libed_probes.so (include/ed_probes.h) run on the GPU
and return plausible figures: every rate positive and ordered as the memory
hierarchy orders them (shared memory above L2 above DRAM), float32 FMA above
float64, the multiprocessor count of the device; the shared-memory pattern
kernels launch and finish without error."""
import pytest

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def test_ceilings_are_ordered():
    torch = torch_cuda()
    from paper_2005_13498_gb300 import probes
    c = probes.ed_probe_ceilings()
    for k in ("l2_read_gbs", "hbm_read_gbs", "smem_read_gbs", "fp32_fma_tflops",
              "fp32x2_fma_tflops", "fp64_fma_tflops"):
        assert c[k] > 0.0, k
    assert c["smem_read_gbs"] > c["l2_read_gbs"] > c["hbm_read_gbs"]
    assert c["fp32_fma_tflops"] > c["fp64_fma_tflops"]
    assert c["sms"] == torch.cuda.get_device_properties(0).multi_processor_count


def test_shared_load_patterns_run():
    torch_cuda()
    from paper_2005_13498_gb300 import probes
    probes.ed_probe_shared_loads()
