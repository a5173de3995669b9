"""The generated congruence products (paper_1702_06359_gb300/csrc/gen_sparse.py ->
sparse_gen.cuh; the Matriplex code-generator idea of Sec. 2.1): the committed header is what
the generator writes, and its functions (cylinder and plane transports, measured rows),
compiled as host C++ in double, equal the dense products A P A^T of random sparse matrices of
the declared patterns (numpy, 1e-12)."""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1702_06359_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_sparse  # noqa: E402

PROGRAM = r"""
#include <cstdio>
#include "sparse_gen.cuh"
int main()
{
    double j[17], m[9], q[11], P[21], S[21], S2[3], S3[21];
    for (double &v : j) if (std::scanf("%lf", &v) != 1) return 1;
    for (double &v : m) if (std::scanf("%lf", &v) != 1) return 1;
    for (double &v : q) if (std::scanf("%lf", &v) != 1) return 1;
    for (double &v : P) if (std::scanf("%lf", &v) != 1) return 1;
    tkf::transport_cov<double>(j[0], j[1], j[2], j[3], j[4], j[5], j[6], j[7], j[8], j[9], j[10], j[11], j[12],
                               j[13], j[14], j[15], j[16], P, S);
    tkf::measured_cov<double>(m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7], m[8], P, S2);
    tkf::plane_cov<double>(q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], q[8], q[9], q[10], P, S3);
    for (double v : S) std::printf("%.17g\n", v);
    for (double v : S2) std::printf("%.17g\n", v);
    for (double v : S3) std::printf("%.17g\n", v);
    return 0;
}
"""


def test_committed_header_is_what_the_generator_writes():
    with open(os.path.join(CSRC, "sparse_gen.cuh")) as f:
        assert f.read() == gen_sparse.render()


def _dense(pattern, values):
    A = np.zeros((len(pattern), 6))
    for i, row in enumerate(pattern):
        for k, e in enumerate(row):
            A[i, k] = 0.0 if e == "0" else (1.0 if e == "1" else values[e])
    return A


def _packed(S):
    return np.array([S[i, j] for i in range(S.shape[0]) for j in range(i + 1)])


def test_generated_products_equal_dense_products(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    src = tmp_path / "prog.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "prog"
    subprocess.check_call([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])
    rng = np.random.default_rng(1702)
    jnames = ["a0", "a1", "a3", "a4", "b0", "b1", "b3", "b4", "c0", "c1", "c3", "c4", "c5", "f0", "f1", "f3", "f4"]
    mnames = ["m0", "m1", "m3", "m4", "v0", "v1", "v3", "v4", "v5"]
    qnames = ["a2", "a3", "a4", "a5", "b2", "b3", "b4", "b5", "f2", "f3", "f5"]
    for _ in range(20):
        jv = dict(zip(jnames, rng.normal(size=len(jnames))))
        mv = dict(zip(mnames, rng.normal(size=len(mnames))))
        qv = dict(zip(qnames, rng.normal(size=len(qnames))))
        X = rng.normal(size=(6, 6))
        P = X @ X.T + 0.1 * np.eye(6)
        inp = " ".join("%.17g" % v for v in [*(jv[k] for k in jnames), *(mv[k] for k in mnames),
                                             *(qv[k] for k in qnames), *_packed(P)])
        out = np.array(subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True)
                       .stdout.split(), dtype=float)
        J = _dense(gen_sparse.TRANSPORT, jv)
        M = _dense(gen_sparse.MEASURED, mv)
        Jp = _dense(gen_sparse.PLANE, qv)
        want = np.concatenate([_packed(J @ P @ J.T), _packed(M @ P @ M.T), _packed(Jp @ P @ Jp.T)])
        assert np.allclose(out, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    # a planted mistake in the pattern (a dropped entry) is caught by the same comparison
    bad = [row[:] for row in gen_sparse.TRANSPORT]
    bad[0][3] = "0"
    assert not np.allclose(_packed(_dense(bad, jv) @ P @ _dense(bad, jv).T), want[:21], rtol=1e-6)
    bad = [row[:] for row in gen_sparse.PLANE]
    bad[4][5] = "0"
    assert not np.allclose(_packed(_dense(bad, qv) @ P @ _dense(bad, qv).T), want[24:], rtol=1e-6)
