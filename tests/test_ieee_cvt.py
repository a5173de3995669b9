"""The integer-only conversions between binary32 and binary64 (csrc/ieee_cvt.cuh) that the
mixed-precision Kalman update uses instead of the GPU's scarce double-precision units, compiled
as host C++ and held to the C conversions, which follow IEEE 754 (float -> double exact; double
-> float rounded to nearest, ties to even): bit for bit on random values over the whole float
range, on values just beside rounding ties, and on the special cases (zero, infinities, NaN,
the largest float, values that round up to it or overflow).  Subnormal floats are flushed to a
signed zero, as the library's single-precision arithmetic flushes them."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1702_06359_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "ieee_cvt.cuh"
int main()
{
    char kind;
    unsigned long long bits;
    while (std::scanf(" %c %llx", &kind, &bits) == 2) {
        if (kind == 'f') {  // binary32 in, binary64 bits out
            const uint32_t u = (uint32_t)bits;
            float f;
            std::memcpy(&f, &u, 4);
            const double d = tkf::f32_to_f64_bits(f);
            uint64_t o;
            std::memcpy(&o, &d, 8);
            std::printf("%016llx\n", (unsigned long long)o);
        } else {  // binary64 in, binary32 bits out
            double d;
            std::memcpy(&d, &bits, 8);
            const float f = tkf::f64_to_f32_bits(d);
            uint32_t o;
            std::memcpy(&o, &f, 4);
            std::printf("%08x\n", o);
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    d = tmp_path_factory.mktemp("cvt")
    src = d / "cvt.cpp"
    src.write_text(PROGRAM)
    exe = d / "cvt"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.check_call([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", cuda_inc, str(src), "-o", str(exe)])
    return str(exe)


def _run(exe, items):
    inp = "\n".join("%s %x" % kv for kv in items)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    return [int(x, 16) for x in out]


def _f32_bits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def _f64_bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def test_float_to_double_is_exact(prog):
    rng = np.random.default_rng(1)
    u = rng.integers(0, 2 ** 32, size=20000, dtype=np.uint64).astype(np.uint32)
    specials = np.array([0, 0x80000000, 0x00800000, 0x80800000, 0x7F7FFFFF, 0x3F800000, 0x7F800000, 0xFF800000,
                         0x7FC00000, 0x00000001, 0x807FFFFF], dtype=np.uint32)
    u = np.concatenate([u, specials])
    got = _run(prog, [("f", int(x)) for x in u])
    for x, g in zip(u, got):
        f = np.array([x], dtype=np.uint32).view(np.float32)[0]
        e = (int(x) >> 23) & 0xFF
        if e == 0:  # zero and subnormals: signed zero
            want = (int(x) & 0x80000000) << 32
        elif e == 0xFF and int(x) & 0x7FFFFF:  # NaN stays NaN
            assert (g >> 52) & 0x7FF == 0x7FF and g & ((1 << 52) - 1), hex(int(x))
            continue
        else:
            want = _f64_bits(float(f))
        assert g == want, (hex(int(x)), hex(g), hex(want))


def test_double_to_float_rounds_to_nearest_even(prog):
    rng = np.random.default_rng(2)
    # random doubles over (a little beyond) the float range, both signs
    mant = rng.uniform(1.0, 2.0, size=20000)
    expo = rng.integers(-130, 130, size=20000)
    d = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], size=20000)
    # exact halfway points between neighbouring floats, and their neighbours one double ulp away
    f = rng.uniform(1e-30, 1e30, size=3000).astype(np.float32)
    lo = f.astype(np.float64)
    hi = np.nextafter(f, np.float32(np.inf)).astype(np.float64)
    mid = 0.5 * (lo + hi)
    ties = np.concatenate([mid, np.nextafter(mid, -np.inf), np.nextafter(mid, np.inf)])
    fmax = float(np.finfo(np.float32).max)
    specials = np.array([0.0, -0.0, 1.0, -1.0, fmax, np.nextafter(fmax, np.inf), fmax * (1 + 2 ** -25),
                         fmax * (1 + 2 ** -24), 3.4e38, 1e39, -1e39, np.inf, -np.inf, 2.0 ** -126,
                         2.0 ** -126 * (1 - 2 ** -30), 1e-40, 1e-300])
    d = np.concatenate([d, ties, specials])
    got = _run(prog, [("d", _f64_bits(float(x))) for x in d])
    with np.errstate(over="ignore"):
        ref = d.astype(np.float32)
    for x, g, r in zip(d, got, ref):
        want = _f32_bits(float(r))
        if ((want >> 23) & 0xFF) == 0:  # subnormal or zero result: signed zero
            want &= 0x80000000
        assert g == want, (repr(float(x)), hex(g), hex(want))
    nan = _run(prog, [("d", 0x7FF8000000000001)])[0]
    assert (nan >> 23) & 0xFF == 0xFF and nan & 0x7FFFFF
