"""Writes sparse_gen.cuh: congruence products S = A P A^T of a symmetric 6x6 covariance P with a
matrix A of known sparsity, written out term by term -- known zeros skipped, known ones not
multiplied.  This is the Matriplex code-generator idea of Sec. 2.1 of arXiv:1702.06359, for
the products of the Kalman-filter kernels:

  transport_cov   P' = J P J^T with the helix transport Jacobian J (propagation to a cylinder);
  plane_cov       P' = J P J^T for the propagation to a plane z = const (an endcap disk);
  measured_cov    the 2x2 block M P M^T with M = H J, the two measured rows of the transported
                  state (the two-step propagation's per-hit chi2).

    python gen_sparse.py            # rewrites sparse_gen.cuh beside this file
    python gen_sparse.py --check    # exit status 1 if sparse_gen.cuh is out of date

An entry of a pattern is "0", "1" or the name of a scalar argument.  P and S are packed lower
triangles in row order (element (i, j), i >= j, at i (i + 1) / 2 + j).  For each row i of A
that is not a unit row, the generated code forms the row T_i = A_i P, summing over the nonzero
entries in column order; a unit row e_m takes row m of P; a zero row gives zeros.  It then forms S_ik = T_i . A_k over
the nonzero entries of A_k in column order, and a unit row A_k = e_m takes T_i[m].  Products
are written as (entry) * (operand), left to right, so that the compiler's multiply-add
contraction sees the same expression trees as a hand-written form in that order.
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "sparse_gen.cuh")

# helix transport Jacobian d(state out)/d(state in) at fixed transverse path plus the path's
# dependence on the start (rows and columns x, y, z, q/pT, phi, theta)
TRANSPORT = [
    ["a0", "a1", "0", "a3", "a4", "0"],      # x
    ["b0", "b1", "0", "b3", "b4", "0"],      # y
    ["c0", "c1", "1", "c3", "c4", "c5"],     # z
    ["0", "0", "0", "1", "0", "0"],          # q/pT
    ["f0", "f1", "0", "f3", "f4", "0"],      # phi
    ["0", "0", "0", "0", "0", "1"],          # theta
]
# helix transport to a plane z = const (an endcap disk): the path depends on z and theta only,
# so rows x, y, phi gain columns z and theta and lose the x, y dependence of the path; row z is
# zero (the plane's z is fixed)
PLANE = [
    ["1", "0", "a2", "a3", "a4", "a5"],      # x
    ["0", "1", "b2", "b3", "b4", "b5"],      # y
    ["0", "0", "0", "0", "0", "0"],          # z
    ["0", "0", "0", "1", "0", "0"],          # q/pT
    ["0", "0", "f2", "f3", "1", "f5"],       # phi
    ["0", "0", "0", "0", "0", "1"],          # theta
]
# the two measured rows of the transported state: u (along the hit's tangent) and z
MEASURED = [
    ["m0", "m1", "0", "m3", "m4", "0"],      # u = -sin(phi_h) x + cos(phi_h) y
    ["v0", "v1", "1", "v3", "v4", "v5"],     # v = z
]


def _sym(i, j):
    return i * (i + 1) // 2 + j if i >= j else j * (j + 1) // 2 + i


def _zero(row):
    return all(e == "0" for e in row)


def _unit(row):
    """Index m when row is the unit row e_m, else None."""
    nz = [k for k, e in enumerate(row) if e != "0"]
    return nz[0] if len(nz) == 1 and row[nz[0]] == "1" else None


def _sum(terms):
    return " + ".join(terms) if terms else "R(0)"


def sandwich(name, pattern, doc):
    rows = len(pattern)
    args = [e for row in pattern for e in row if e not in ("0", "1")]
    seen = []
    for a in args:
        if a not in seen:
            seen.append(a)
    out_n = rows * (rows + 1) // 2
    sig = ", ".join("R %s" % a for a in seen)
    lines = ["// " + ln for ln in doc.split("\n")]
    lines.append("template <class R>")
    lines.append("TKF_HD void %s(%s, const R P[21], R S[%d])" % (name, sig, out_n))
    lines.append("{")
    # T_i = A_i P for the non-unit rows
    trow = {}
    for i, row in enumerate(pattern):
        if _zero(row):
            trow[i] = ("Z", i)
            continue
        m = _unit(row)
        if m is not None:
            trow[i] = ("P", m)
            continue
        trow[i] = ("T", i)
        lines.append("    R T%d[6];" % i)
    lines.append("#pragma unroll")
    lines.append("    for (int j = 0; j < 6; ++j) {")
    for i, row in enumerate(pattern):
        if trow[i][0] != "T":
            continue
        terms = []
        for k, e in enumerate(row):
            if e == "0":
                continue
            p = "P[tkf_gen_sym(%d, j)]" % k
            terms.append(p if e == "1" else "%s * %s" % (e, p))
        lines.append("        T%d[j] = %s;" % (i, _sum(terms)))
    lines.append("    }")
    # S_ik = T_i . A_k, lower triangle
    for i in range(rows):
        for k in range(i + 1):
            if _zero(pattern[i]) or _zero(pattern[k]):  # a zero row of A gives a zero row of S
                lines.append("    S[%d] = R(0);" % _sym(i, k))
                continue

            def t_at(m):
                kind, idx = trow[i]
                return "T%d[%d]" % (i, m) if kind == "T" else "P[%d]" % _sym(idx, m)

            mk = _unit(pattern[k])
            if mk is not None:
                expr = t_at(mk)
            else:
                terms = []
                for m, e in enumerate(pattern[k]):
                    if e == "0":
                        continue
                    terms.append(t_at(m) if e == "1" else "%s * %s" % (t_at(m), e))
                expr = _sum(terms)
            lines.append("    S[%d] = %s;" % (_sym(i, k), expr))
    lines.append("}")
    return "\n".join(lines)


def render():
    head = """// GENERATED by gen_sparse.py from the sparsity patterns declared there -- do not edit; run
// `python gen_sparse.py` after changing a pattern.  Congruence products S = A P A^T of a
// packed symmetric 6x6 P with a sparse A, term by term (Sec. 2.1 of arXiv:1702.06359: the
// Matriplex code generator's skipping of known zeros and ones).  Packed lower triangles in
// row order.
#pragma once

#ifdef __CUDACC__
#define TKF_HD __host__ __device__ __forceinline__
#else
#define TKF_HD inline
#endif

namespace tkf {

TKF_HD constexpr int tkf_gen_sym(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }
"""
    body = [
        sandwich("transport_cov", TRANSPORT,
                 "P' = J P J^T for the helix transport Jacobian J: rows x, y, phi have entries in columns\n"
                 "x, y, q/pT, phi; row z also in columns z (1) and theta; rows q/pT and theta are unit rows."),
        sandwich("plane_cov", PLANE,
                 "P' = J P J^T for the transport to a plane z = const: rows x, y, phi have entries in\n"
                 "columns z, q/pT, phi, theta (x, y on their own column); row z is zero; q/pT, theta unit rows."),
        sandwich("measured_cov", MEASURED,
                 "[[Suu], [Suv, Svv]] = M P M^T for the two measured rows M of a transported state: u in\n"
                 "columns x, y, q/pT, phi; v = z in every column, 1 in column z."),
    ]
    return head + "\n" + "\n\n".join(body) + "\n\n}  // namespace tkf\n"


def main():
    text = render()
    if "--check" in sys.argv:
        with open(OUT) as f:
            ok = f.read() == text
        if not ok:
            print("sparse_gen.cuh is out of date: run python gen_sparse.py")
        sys.exit(0 if ok else 1)
    with open(OUT, "w") as f:
        f.write(text)


if __name__ == "__main__":
    main()
