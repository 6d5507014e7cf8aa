"""The FP32 FMA probe behind the measured roofline denominator: it runs, its
output is finite, and its rate is within a plausible range of the SM count x
128 lanes x 2 flop x clock figure."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_fma_probe_rate():
    import torch
    from paper_2104_00359_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda:0")
    blocks = 152 * 8
    out = torch.empty(blocks * 256, device=dev)
    assert lib.shs_fp32_fma_probe(0, 10, _lib.ptr(out), None) == 1
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    times = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _lib.check(lib.shs_fp32_fma_probe(blocks, 1 << 15, _lib.ptr(out), sp), "probe")
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    assert np.all(np.isfinite(out.cpu().numpy()))
    tflops = 16.0 * (1 << 15) * blocks * 256 / (min(times) * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    assert 0.3 * nominal < tflops < 2.5 * nominal, (tflops, nominal)
