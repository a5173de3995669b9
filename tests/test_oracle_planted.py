"""Plausible mistakes planted in a compiled copy of the oracle (on the CPU): each must make one
of the pins of the part it sits in fail.  This checks the pins, not the oracle: a pin that a
dropped term, a wrong sign or a swapped index passes would not pin anything.  (The seeding
pins have their own planted set in test_oracle_seeding.py.)"""
import os
import shutil
import subprocess
import sys

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (pins file, exact text in tkf_oracle.c, planted replacement)
PLANTED = {
    "helix: phi turns the wrong way": ("test_oracle_propagation.py", "const double phi1 = phi0 + kappa * s;",
                                       "const double phi1 = phi0 - kappa * s;"),
    "Jacobian: d phi / d(q/pT) halved": ("test_oracle_propagation.py", "F[4 * 6 + 3] = s * dkdw;",
                                         "F[4 * 6 + 3] = 0.5 * s * dkdw;"),
    "Highland: beta for beta^2 in the log": ("test_oracle_fit.py", "log(t / (beta * beta))", "log(t / beta)"),
    "scattering: q/pT kick sign": ("test_oracle_fit.py", "{-w * cot, 0}", "{w * cot, 0}"),
    "update: Joseph form without K V K^T": ("test_oracle_fit.py",
                                            "P[i * 6 + j] = APAt[i * 6 + j] + KVKt[i * 6 + j];",
                                            "P[i * 6 + j] = APAt[i * 6 + j];"),
    "measurement: z residual sign": ("test_oracle_fit.py", "r[1] = h->z - p[2];", "r[1] = p[2] - h->z;"),
    "seed: cot(theta) from the wrong hit": ("test_oracle_fit.py", "const double cot = (h3->z - h1->z) / s13;",
                                            "const double cot = (h3->z - h2->z) / s13;"),
    "ranking: chi2 descending": ("test_oracle_build.py", "return x->chi2 < y->chi2 ? -1 : 1;",
                                 "return x->chi2 > y->chi2 ? -1 : 1;"),
    "index: eta of the first layer's radius": ("test_oracle_build.py", "asinh(z / g->radius[layer])",
                                               "asinh(z / g->radius[0])"),
    "window: z half-width from the r-phi variance": ("test_oracle_build.py",
                                                     "    double W = sqrt(g->chi2_cut * S[3])",
                                                     "    double W = sqrt(g->chi2_cut * S[0])"),
    "backward: theta not reversed": ("test_oracle_backward.py", "b[5] = ORC_PI - a[5];", "b[5] = a[5];"),
    "disks: path to the plane": ("test_oracle_disks.py", "const double s = (Zp - pin[2]) / cot_th;",
                                 "const double s = (Zp - pin[2]) * cot_th;"),
    "modules: states kept on the average radius": ("test_oracle_two_step.py",
                                                   "return (g->hit_dr > 0.0 && h) ? sqrt(h->x * h->x + h->y * h->y) "
                                                   ": g->radius[layer];",
                                                   "return g->radius[layer];"),
}


@pytest.mark.parametrize("name", sorted(PLANTED))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    pins, old, new = PLANTED[name]
    src_dir = os.path.dirname(O.__file__)
    text = open(os.path.join(src_dir, "tkf_oracle.c")).read()
    assert text.count(old) == 1, "the planted text is no longer (or not only once) in the oracle"
    shutil.copy(os.path.join(src_dir, "tkf_oracle.h"), tmp_path)
    (tmp_path / "tkf_oracle.c").write_text(text.replace(old, new))
    so = str(tmp_path / "liborc_planted.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", so, str(tmp_path / "tkf_oracle.c"),
                           "-lm"])
    env = dict(os.environ, ORC_LIBRARY=so)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins), "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    # exit code 1: a pin failed (2 and above would be an error of the run itself)
    assert r.returncode == 1, "no pin in %s caught '%s':\n%s" % (pins, name, r.stdout[-2000:])
