"""Pins of the oracle's seeding from hit triplets (layers 0, 1, 2, confirmed on layer 3).

Sec. 2 names seeding as the stage that gives the first estimate from a few inner hits and leaves
it unspecified; the oracle's reading is a brute-force definition (tkf_oracle.c).  References used
instead of the oracle itself:
- closed forms of circle geometry: the curvature of the circle through the beam line point and
  two hits from the inscribed-angle theorem, the power of a point of a circle with known centre
  and radius, the distance of a point placed at a known offset from a circle;
- the generator's truth on noise-free tracks (curvature from pT and the field, the circle's
  centre from the momentum direction at the vertex);
- each cut planted just inside and just outside its limit on a clean track; the confirmation
  hit's residuals entering the score (a worse triplet with a better confirmation wins);
- symmetries (rotation about the beam line, y -> -y, z -> -z) under which the picks must not move;
- on the seeding workload (pixel inner layers), the own triplet of nearly every track.
Eight plausible mistakes planted in a compiled copy of the oracle each fail one of these pins."""
import math

import numpy as np
import pytest

import oracle as O
from synth import Detector, EventSpec, generate
from synth.events import K_B

PIX = Detector(pixel_layers=4)


def _hit(x, y, z, layer):
    return O.make_hit(x, y, z, 4e-6, 2.5e-5, layer)


def _on_circle(ux, uy, rho, r, branch=1):
    """A point at transverse radius r on the circle of centre (ux, uy) and radius rho."""
    D = math.hypot(ux, uy)
    a = (r * r - rho * rho + D * D) / (2 * D)
    h = math.sqrt(r * r - a * a)
    ex, ey = ux / D, uy / D
    return a * ex - branch * h * ey, a * ey + branch * h * ex


def test_circle_quantities_closed_forms():
    g = O.make_geom(PIX)
    cuts = O.SeedCuts(pt_min=0.01, z_vertex=50.0, d0_max=5.0, dz_max=5.0, conf_rphi=5.0, conf_z=5.0)
    ux, uy, rho = 30.0, -40.0, 48.0  # |U| = 50: the beam line point lies 2 cm outside the circle
    pts = [_on_circle(ux, uy, rho, r) for r in (4.0, 8.0, 12.0)]
    z0, t = 0.7, 0.9  # hits on the r-z line z = z0 + t r
    a, b, c = (_hit(x, y, z0 + t * r, l) for l, ((x, y), r) in enumerate(zip(pts, (4.0, 8.0, 12.0))))
    delta = 0.013  # the layer-3 hit 0.13 mm outside the circle, radially from its centre
    ex, ey = _on_circle(ux, uy, rho, 16.0)
    k = (rho + delta) / rho
    e = _hit(ux + k * (ex - ux), uy + k * (ey - uy), 0.0, 3)
    re = math.hypot(e.x, e.y)
    e.z = z0 + t * re  # on the r-z line of b and c
    ok, q = O.seed_eval(g, cuts, a, b, c, e)
    assert ok
    assert q.kappa == pytest.approx(1 / rho, rel=1e-12)
    assert q.d0 == pytest.approx((50.0 ** 2 - rho ** 2) / (2 * rho), rel=1e-12)  # power / diameter
    assert q.f3 == pytest.approx(delta + delta * delta / (2 * rho), rel=1e-9)
    assert abs(q.zv - z0) < 1e-12 and abs(q.dz) < 1e-12 and abs(q.dz3) < 1e-12
    # curvature through the beam line point: chord AB = 2 rho' sin(angle AOB) (inscribed angle)
    ang = math.atan2(a.x * b.y - a.y * b.x, a.x * b.x + a.y * b.y)
    chord = math.hypot(b.x - a.x, b.y - a.y)
    assert q.kappa01 == pytest.approx(2 * math.sin(ang) / chord, rel=1e-12)
    assert q.chord01 == pytest.approx(chord, rel=1e-15)
    # z offsets enter with their sign and at their own hit
    c.z += 0.02
    e.z -= 0.03
    _, q2 = O.seed_eval(g, cuts, a, b, c, e)
    assert q2.dz == pytest.approx(0.02, abs=1e-12)
    slope = (c.z - b.z) / (math.hypot(c.x, c.y) - math.hypot(b.x, b.y))
    assert q2.dz3 == pytest.approx(e.z - (b.z + slope * (re - math.hypot(b.x, b.y))), abs=1e-12)


def test_truth_of_noise_free_tracks():
    det = Detector(pixel_layers=4, x_over_x0=(0.0,) * 10)
    b = generate(EventSpec(seed=71, n_tracks=40, noise_frac=0.0, scatter=False, smear=False, keep_f64=True,
                           vertex_sigma=(0.02, 0.02, 1.0)), det)
    g = O.make_geom(det)
    hits = O.hits_of(b, exact=True)
    cuts = O.SeedCuts(d0_max=0.2)
    pk = O.find_seeds(g, cuts, hits)
    th = b.trk_hits
    for t in range(b.n_tracks):
        vx, vy, _, w, phi, _ = b.vertex_state[t]
        kappa = K_B * det.bz * abs(w)
        rho = 1 / kappa
        h0 = hits[th[t, 0]]
        # the centre lies rho away from the vertex, perpendicular to the momentum; the side is
        # the one whose circle holds the first hit
        cands = [(vx - s * rho * math.sin(phi), vy + s * rho * math.cos(phi)) for s in (1, -1)]
        ux, uy = min(cands, key=lambda u: abs(math.hypot(h0["x"] - u[0], h0["y"] - u[1]) - rho))
        assert abs(math.hypot(h0["x"] - ux, h0["y"] - uy) - rho) < 1e-9
        ok, q = O.seed_eval(g, cuts, *(O.make_hit(*hits[th[t, l]][["x", "y", "z", "var_u", "var_v"]], l)
                                       for l in range(4)))
        assert ok
        assert q.kappa == pytest.approx(kappa, rel=1e-9)
        assert q.d0 == pytest.approx((ux * ux + uy * uy - rho * rho) / (2 * rho), abs=1e-9)
        assert abs(q.f3) < 1e-9
        p = pk[th[t, 0]]
        assert (p["h1"], p["h2"], p["h3"]) == (th[t, 1], th[t, 2], th[t, 3])


def _clean_track():
    det = Detector(pixel_layers=4, x_over_x0=(0.0,) * 10)
    b = generate(EventSpec(seed=72, n_tracks=1, noise_frac=0.0, scatter=False, keep_f64=True), det)
    hits = O.hits_of(b, exact=True)
    return O.make_geom(det), hits, b.trk_hits[0]


@pytest.mark.parametrize("field", ["pt_min", "z_vertex", "d0_max", "dz_max", "conf_rphi", "conf_z"])
def test_each_cut_planted_inside_and_outside(field):
    g, hits, th = _clean_track()
    cuts = O.SeedCuts()
    ok, q = O.seed_eval(g, cuts, *(O.make_hit(*hits[th[l]][["x", "y", "z", "var_u", "var_v"]], l) for l in range(4)))
    assert ok
    value = {"pt_min": None, "z_vertex": abs(q.zv), "d0_max": abs(q.d0), "dz_max": abs(q.dz),
             "conf_rphi": abs(q.f3), "conf_z": abs(q.dz3)}[field]
    for scale, seeded in ((1.001, True), (0.999, False)):
        c = O.SeedCuts()
        if field == "pt_min":
            # kappa_max = K_B Bz / pt_min (1 + slack) just above / below the larger curvature
            kap = max(abs(q.kappa01), q.kappa)
            setattr(c, field, K_B * 3.8 * (1 + c.kappa_slack) / (kap * scale))
        else:
            setattr(c, field, value * scale)
        pk = O.find_seeds(g, c, hits)
        assert (pk[th[0]]["h1"] == th[1]) == seeded, (field, scale)


def test_far_crossing_is_not_a_pair():
    """A hit where a low-pT circle through the beam line and the first hit crosses layer 1 again,
    after looping, passes the curvature cut but not the chord cut."""
    g = O.make_geom(PIX)
    cuts = O.SeedCuts()
    rho = 1 / (0.9 * O.seed_kappa_max(g, cuts))
    ux, uy = rho * math.cos(0.3), rho * math.sin(0.3)  # a circle through the origin
    a = _hit(*_on_circle(ux, uy, rho, 4.0, 1), 0.4, 0)
    near = _hit(*_on_circle(ux, uy, rho, 8.0, 1), 0.8, 1)
    far = _hit(*_on_circle(ux, uy, rho, 8.0, -1), 0.8, 1)
    ok_near, qn = O.seed_eval(g, cuts, a, near)
    ok_far, qf = O.seed_eval(g, cuts, a, far)
    assert ok_near and not ok_far
    assert abs(qf.kappa01) == pytest.approx(abs(qn.kappa01), rel=1e-9)  # the same circle
    assert qf.chord01 > 2 * (g.radius[1] - g.radius[0])


def test_best_triplet_and_ties():
    g, hits, th = _clean_track()
    cuts = O.SeedCuts()
    # a second layer-2 hit 0.3 mm off in z (a worse score), then an exact copy (the same score,
    # a larger id)
    h = np.concatenate([hits, hits[[th[2], th[2]]]])
    i_extra, i_dup = len(hits), len(hits) + 1
    h["z"][i_extra] += 0.03
    pk = O.find_seeds(g, cuts, h)[th[0]]
    assert (pk["h1"], pk["h2"], pk["n_pass"]) == (th[1], th[2], 3)
    assert pk["gap"] == 0.0  # the copy ties
    h2 = h.copy()
    h2["layer"][th[2]] = 5  # remove the own hit from layer 2: the copy (same score) is next
    pk2 = O.find_seeds(g, cuts, h2)[th[0]]
    assert pk2["h2"] == i_dup and pk2["score"] == pytest.approx(pk["score"], rel=1e-12)
    h2["layer"][i_dup] = 5
    pk3 = O.find_seeds(g, cuts, h2)[th[0]]
    assert pk3["h2"] == i_extra and pk3["score"] > pk["score"]
    # without confirmation required the layer-3 hit does not matter
    h3 = h.copy()
    h3["layer"][th[3]] = 5
    assert O.find_seeds(g, cuts, h3)[th[0]]["h1"] == -1
    c0 = O.SeedCuts(confirm=0)
    assert O.find_seeds(g, c0, h3)[th[0]]["h2"] == th[2]


def test_confirmation_quality_enters_the_score():
    """The track's own layer-3 hit moved onto the r-z line of a second layer-2 candidate 0.35 mm
    above the own one: the own triplet keeps the better triplet term but is now confirmed only
    0.7 mm off in z, the second one exactly; the second wins on the sum."""
    g, hits, th = _clean_track()
    cuts = O.SeedCuts()
    h = np.concatenate([hits, hits[[th[2], th[3]]]])
    i_c, i_e = len(hits), len(hits) + 1
    rb, rc, re = (float(np.hypot(h["x"][k], h["y"][k])) for k in (th[1], th[2], th[3]))
    h["z"][i_c] += 0.035
    h["z"][i_e] += 0.035 * (re - rb) / (rc - rb)  # on the r-z line of b and the second candidate
    h["layer"][th[3]] = 5  # the own layer-3 hit replaced by the moved one
    pk = O.find_seeds(g, cuts, h)[th[0]]
    assert (pk["h2"], pk["h3"], pk["n_pass"]) == (i_c, i_e, 2)
    q = {k: O.seed_eval(g, cuts, *(O.make_hit(*h[i][["x", "y", "z", "var_u", "var_v"]], l)
                                   for l, i in enumerate((th[0], th[1], k))))[1] for k in (th[2], i_c)}
    s2 = {k: (q[k].d0 / cuts.d0_max) ** 2 + (q[k].dz / cuts.dz_max) ** 2 for k in q}
    assert s2[th[2]] < s2[i_c] <= pk["score"]


def _transform(hits, f):
    h = hits.copy()
    h["x"], h["y"], h["z"] = f(hits["x"], hits["y"], hits["z"])
    return h


def test_symmetries():
    b = generate(EventSpec(seed=73, n_tracks=250, noise_frac=0.3, keep_f64=True), PIX)
    g = O.make_geom(PIX)
    hits = O.hits_of(b, exact=True)
    cuts = O.SeedCuts()
    ref = O.find_seeds(g, cuts, hits)
    l0 = hits["layer"] == 0
    assert (ref["h1"][l0] >= 0).sum() > 200
    robust = l0 & (ref["margin"] > 1e-9) & (ref["gap"] > 1e-9)
    ca, sa = math.cos(2.1), math.sin(2.1)
    for f in (lambda x, y, z: (ca * x - sa * y, sa * x + ca * y, z), lambda x, y, z: (x, -y, z),
              lambda x, y, z: (x, y, -z)):
        pk = O.find_seeds(g, cuts, _transform(hits, f))
        for k in ("h1", "h2", "h3", "n_pass"):
            assert np.array_equal(pk[k][robust], ref[k][robust]), k
        assert np.allclose(pk["score"][robust], ref["score"][robust], rtol=1e-9, atol=1e-12)


def test_own_triplets_on_pixel_layers():
    """On the seeding workload's detector nearly every track's own triplet is its first hit's
    pick, and seeds barely outnumber tracks."""
    b = generate(EventSpec(seed=74, n_tracks=600, noise_frac=0.3), PIX)
    g = O.make_geom(PIX)
    pk = O.find_seeds(g, O.SeedCuts(), O.hits_of(b))
    th = b.trk_hits
    own = np.mean([(pk[th[t, 0]]["h1"], pk[th[t, 0]]["h2"]) == (th[t, 1], th[t, 2]) for t in range(b.n_tracks)])
    n_seeds = (pk["h1"] >= 0).sum()
    assert own >= 0.99
    assert n_seeds <= 1.05 * b.n_tracks


def test_cuts_keep_true_triplets():
    """The default cuts sit above the true triplets' distributions on the seeding detector (with
    smearing and scattering): at least 99.5 % of 3 000 tracks pass every cut with their own
    hits, and each quantity's 99th percentile stays inside its cut."""
    b = generate(EventSpec(seed=75, n_tracks=3000, noise_frac=0.0), PIX)
    g = O.make_geom(PIX)
    cuts = O.SeedCuts()
    hits = O.hits_of(b)
    th = b.trk_hits
    kmax = O.seed_kappa_max(g, cuts)
    ok, ratios = [], []
    for t in range(b.n_tracks):
        passed, q = O.seed_eval(g, cuts, *(O.make_hit(*hits[th[t, l]][["x", "y", "z", "var_u", "var_v"]], l)
                                           for l in range(4)))
        ok.append(passed)
        ratios.append([abs(q.kappa01) / kmax, abs(q.zv) / cuts.z_vertex, q.kappa / kmax, abs(q.d0) / cuts.d0_max,
                       abs(q.dz) / cuts.dz_max, abs(q.f3) / cuts.conf_rphi, abs(q.dz3) / cuts.conf_z])
    assert np.mean(ok) >= 0.995
    assert np.all(np.percentile(np.array(ratios), 99, axis=0) < 1.0)


# Plausible mistakes planted in a copy of the oracle's seeding code: each must fail one of the
# pins above (the copy is compiled on the CPU and swapped in for the committed library).
PLANTED = {
    "d0 over rho": ("q->d0 = (*ux * *ux + *uy * *uy - *rho * *rho) / (2.0 * *rho);",
                    "q->d0 = (*ux * *ux + *uy * *uy - *rho * *rho) / (*rho);"),
    "dz at the wrong radius": ("(b->z - a->z) * (rc - ra) / (rb - ra)", "(b->z - a->z) * (rc - rb) / (rb - ra)"),
    "f over rho": ("q->f3 = ((e->x - ux) * (e->x - ux) + (e->y - uy) * (e->y - uy) - rho * rho) / (2.0 * rho);",
                   "q->f3 = ((e->x - ux) * (e->x - ux) + (e->y - uy) * (e->y - uy) - rho * rho) / (rho);"),
    "dz3 at the wrong radius": ("(cc->z - b->z) * (re - rb) / (rc - rb)", "(cc->z - b->z) * (re - rc) / (rc - rb)"),
    "z vertex from the wrong radius": ("q->zv = a->z - ra * (b->z - a->z) / (rb - ra);",
                                       "q->zv = a->z - rb * (b->z - a->z) / (rb - ra);"),
    "pair curvature sign": ("(a->x * b->y - a->y * b->x > 0.0 ? 1.0 : -1.0)",
                            "(a->x * b->y - a->y * b->x < 0.0 ? 1.0 : -1.0)"),
    "score without the confirmation": ("(q.dz / c->dz_max) * (q.dz / c->dz_max) + c3;",
                                       "(q.dz / c->dz_max) * (q.dz / c->dz_max);"),
    "chord limit of one layer gap": ("q->chord01 <= 2.0 * (g->radius[1] - g->radius[0])",
                                     "q->chord01 <= 1.0 * (g->radius[1] - g->radius[0])"),
}


def _pins():
    yield test_circle_quantities_closed_forms
    yield test_truth_of_noise_free_tracks
    for f in ("pt_min", "z_vertex", "d0_max", "dz_max", "conf_rphi", "conf_z"):
        yield lambda f=f: test_each_cut_planted_inside_and_outside(f)
    yield test_far_crossing_is_not_a_pair
    yield test_best_triplet_and_ties
    yield test_confirmation_quality_enters_the_score
    yield test_symmetries
    yield test_own_triplets_on_pixel_layers


@pytest.mark.parametrize("name", sorted(PLANTED))
def test_planted_mistake_fails_a_pin(name, tmp_path, monkeypatch):
    import os
    import shutil
    import subprocess
    src_dir = os.path.dirname(O.__file__)
    text = open(os.path.join(src_dir, "tkf_oracle.c")).read()
    old, new = PLANTED[name]
    assert text.count(old) == 1, "the planted line is no longer in the oracle"
    shutil.copy(os.path.join(src_dir, "tkf_oracle.h"), tmp_path)
    (tmp_path / "tkf_oracle.c").write_text(text.replace(old, new))
    so = str(tmp_path / "liborc_planted.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", so, str(tmp_path / "tkf_oracle.c"),
                           "-lm"])
    monkeypatch.setattr(O, "_lib", O.load_library(so))
    failed = []
    for pin in _pins():
        try:
            pin()
        except (AssertionError, ValueError, ZeroDivisionError, FloatingPointError):
            failed.append(pin)
            break
    assert failed, "no pin caught the planted mistake: %s" % name
