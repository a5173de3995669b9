"""tkf_probe_alu, the measured denominators of the ALU rooflines: the rates it reports lie
between a tenth and a few times the GB300's nominal figures (FP32 FMA 152 SMs x 128 lanes x
2 x 2.07 GHz = 80.5 TFLOP/s; FP64 1.25 TFLOP/s; special-function unit 16 per SM and clock =
5.0 T/s), FP32 runs far ahead of FP64, and a null output is refused."""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1702_06359_gb300 import tkf  # noqa: E402


def test_probe_rates_are_plausible():
    r = tkf.probe_alu()
    assert 8.0 < r["fp32_tflops"] < 200.0, r
    assert 0.1 < r["fp64_tflops"] < 20.0, r
    assert 0.5 < r["sfu_tops"] < 20.0, r
    assert r["fp32_tflops"] > 8 * r["fp64_tflops"]


def test_probe_refuses_null_outputs():
    d = C.c_double()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert tkf.lib().tkf_probe_alu(s, None, C.byref(d), C.byref(d)) == tkf.ERR_INVALID
