"""The pipe-throughput microbenchmarks (synax_pipe_peak) that give the march's
roofline denominators: every pipe reports a positive rate below the
instruction-issue bound of the device, the paired FMA does two element
operations per instruction, and an unknown pipe is rejected."""
import ctypes

import pytest

from paper_2410_01136_gb300 import _native

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    return _t


def test_every_pipe_reports_a_bounded_rate(torch):
    import paper_2410_01136_gb300 as sx
    r = sx.pipe_peaks(iters=2048, repeats=2)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    # issue bound: 4 schedulers x 32 lanes per SM per clock, at most ~3 GHz
    bound = sms * 128 * 3.0e9
    for name in _native.PIPES:
        assert 0.0 < r[name] <= (2 if name == "ffma2" else 1) * bound, (name, r[name])
    # the SFU is narrower than the FP32 pipe, and its conversions share it
    for name in ("ex2", "lg2", "sin", "cos", "rcp", "rsqrt", "frnd", "f2i"):
        assert r[name] < r["ffma"], name


def test_ops_count_and_validation(torch):
    L = _native.lib()
    sink = torch.empty(4 * 256, dtype=torch.float32, device="cuda")
    ops = ctypes.c_longlong(0)
    h = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.synax_pipe_peak(_native.PIPES["ffma2"], 4, 10, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops), h) == 0
    assert ops.value == 4 * 256 * 10 * 8 * 2          # 8 chains, two elements per paired FMA
    assert L.synax_pipe_peak(_native.PIPES["f2i"], 4, 10, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops), h) == 0
    assert ops.value == 4 * 256 * 10 * 8
    torch.cuda.synchronize()
    assert bool(torch.isfinite(sink).all())
    assert L.synax_pipe_peak(10, 4, 10, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops), h) == _native.SYNAX_EINVAL
    assert L.synax_pipe_peak(0, 0, 10, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops), h) == _native.SYNAX_EINVAL
