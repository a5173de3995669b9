"""Pins of the oracle's Kalman update, scattering noise, seed estimate and track fit (Sec. 2).

References used instead of the oracle itself: a hand-worked chi2 for a diagonal covariance,
noise-free tracks (the filter must return the truth exactly), the batch weighted
least-squares information matrix built from the event generator's own helix code (the
Kalman filter must reproduce it), symmetric positive-definite covariances, unit-width pulls
and a flat chi2 p-value on simulated tracks, and the generator's simulated scattering kicks.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from synth import Detector, EventSpec, generate
from synth.events import K_B, _helix_to_cylinder


def _wrap(a):
    return (np.asarray(a) + math.pi) % (2 * math.pi) - math.pi


def test_chi2_and_update_hand_worked_case():
    """Prediction at (R, 0, 0) pointing along +x: the tangent is +y, so u = y_h and v = z_h.
    With P = diag(a, b, c, ...) the innovation covariance is diag(b + su2, c + sv2)."""
    a, b, c = 0.04, 0.09, 0.25
    P = np.diag([a, b, c, 0.01, 0.0004, 0.0009])
    p = np.array([10.0, 0.0, 0.0, 0.5, 0.0, 1.0])
    su2, sv2 = 0.01, 0.0225
    hit = O.make_hit(10.0 * math.cos(0.03), 10.0 * math.sin(0.03), 0.2, su2, sv2)
    # tangent at the hit is (-sin 0.03, cos 0.03): u = 10 sin(0.03)  (hit and prediction on r = 10)
    u = 10.0 * math.sin(0.03)
    Suu = math.sin(0.03) ** 2 * a + math.cos(0.03) ** 2 * b + su2
    Svv = c + sv2
    expect = u * u / Suu + 0.2 * 0.2 / Svv
    assert O.chi2(p, P, hit) == pytest.approx(expect, rel=1e-13)
    st, p1, P1, c2 = O.update(p, P, hit)
    assert st == 0 and c2 == pytest.approx(expect, rel=1e-13)
    # z decouples: the scalar Kalman update z <- z + c/(c+sv2) v, var <- c sv2/(c+sv2)
    assert p1[2] == pytest.approx(0.2 * c / Svv, rel=1e-13)
    assert P1[2, 2] == pytest.approx(c * sv2 / Svv, rel=1e-13)
    # untouched parameters keep their values and variances
    for i in (3, 5):
        assert p1[i] == p[i] and P1[i, i] == P[i, i]


def _fit_event(det, spec, settings=O.Settings()):
    b = generate(spec, det)
    g = O.make_geom(det, settings)
    hits = O.hits_of(b, exact=spec.keep_f64)
    par0, cov0 = O.seed_estimate(g, hits, b.trk_hits[:, :3])
    po, co, c2, nh, st = O.fit(g, hits, par0, cov0, b.trk_hits, 0, det.n_layers - 1)
    assert np.all(st == 0)
    return b, g, hits, (par0, cov0), (po, co, c2, nh)


def test_noise_free_tracks_return_truth():
    det = Detector(x_over_x0=(0.0,) * 10)
    b, g, hits, (par0, _), (po, co, c2, nh) = _fit_event(det, EventSpec(seed=21, n_tracks=400, scatter=False,
                                                                        smear=False, keep_f64=True))
    # the three-hit estimate of an exact helix is the exact state at the first hit
    d0 = par0 - b.truth[:, 0]
    d0[:, 4] = _wrap(d0[:, 4])
    assert np.max(np.abs(d0)) < 1e-9
    d = po - b.truth[:, -1]
    d[:, 4] = _wrap(d[:, 4])
    assert np.max(np.abs(d)) < 1e-9
    assert np.max(c2) < 1e-12
    assert np.all(nh == det.n_layers)


def test_covariance_equals_batch_least_squares_information():
    """Noise-free track, filter started at the truth: the final covariance must equal
    J (P0^-1 + sum_l A_l^T V^-1 A_l)^-1 J^T, with A_l = d(u_l, v_l)/d(state at layer 1) and
    J = d(state at layer 10)/d(state at layer 1) taken by central differences of the event
    generator's helix crossing (code independent of the oracle)."""
    det = Detector(x_over_x0=(0.0,) * 10)
    b = generate(EventSpec(seed=22, n_tracks=12, scatter=False, smear=False, keep_f64=True), det)
    g = O.make_geom(det)
    hits = O.hits_of(b, exact=True)
    kb = K_B * det.bz
    P0 = np.diag(np.square(O.Settings().prior_sigma))
    V = np.diag([det.sigma_rphi ** 2, det.sigma_z ** 2]).astype(np.float32).astype(np.float64)

    def forward(p1):
        """measurements (u_l, v_l) at every layer and the final state, from state p1 on layer 1"""
        x, y, z, w, phi, th = [np.array([v]) for v in p1]
        meas, state = [], None
        for l in range(det.n_layers):
            if l > 0:
                x, y, z, phi = _helix_to_cylinder(x, y, z, w, phi, th, det.radii[l], kb)
            meas.append((x[0], y[0], z[0]))
            state = np.array([x[0], y[0], z[0], w[0], phi[0], th[0]])
        return meas, state

    for t in range(b.n_tracks):
        p1 = b.truth[t, 0].copy()
        ids = b.trk_hits[t]
        po, co, c2, nh, st = O.fit(g, hits, p1[None], P0[None], ids[None], 0, det.n_layers - 1)
        A = np.zeros((det.n_layers, 2, 6))
        Jf = np.zeros((6, 6))
        for j in range(6):
            h = 1e-6 if j in (0, 1, 2) else 1e-7
            pp, pm = p1.copy(), p1.copy()
            pp[j] += h
            pm[j] -= h
            mp, sp = forward(pp)
            mm, sm = forward(pm)
            for l in range(det.n_layers):
                hx, hy = hits["x"][ids[l]], hits["y"][ids[l]]
                ph = math.atan2(hy, hx)
                tx, ty = -math.sin(ph), math.cos(ph)
                up = tx * mp[l][0] + ty * mp[l][1]
                um = tx * mm[l][0] + ty * mm[l][1]
                A[l, 0, j] = (up - um) / (2 * h)
                A[l, 1, j] = (mp[l][2] - mm[l][2]) / (2 * h)
            d = sp - sm
            d[4] = _wrap(d[4])
            Jf[:, j] = d / (2 * h)
        info = np.linalg.inv(P0)
        for l in range(det.n_layers):
            info += A[l].T @ np.linalg.inv(V) @ A[l]
        Pb = Jf @ np.linalg.inv(info) @ Jf.T
        rel = np.abs(co[0] - Pb) / np.sqrt(np.outer(np.diag(Pb), np.diag(Pb)) + 1e-30)
        assert np.max(rel) < 1e-5, (t, np.max(rel))


def test_covariances_stay_symmetric_positive_definite():
    """After every layer P is symmetric and positive semi-definite.  Once a state has been
    propagated onto a cylinder its only null direction is the radial position offset at the
    predicted crossing, because the crossing point cannot leave the cylinder (the update then
    moves the position along that tangent, so the output radial direction differs from it by
    the small angle correction/R); on the orthogonal 5-dimensional complement P must be
    positive definite."""
    det = Detector()
    b = generate(EventSpec(seed=23, n_tracks=500, pt_max=100.0), det)
    g = O.make_geom(det)
    hits = O.hits_of(b)
    par0, cov0 = O.seed_estimate(g, hits, b.trk_hits[:, :3])
    for last in range(det.n_layers):
        po, co, _, _, st = O.fit(g, hits, par0, cov0, b.trk_hits, 0, last)
        assert np.all(st == 0)
        assert np.array_equal(co, np.transpose(co, (0, 2, 1)))
        if last == 0:
            np.linalg.cholesky(co)
            continue
        r = np.hypot(po[:, 0], po[:, 1])
        n = np.zeros((len(po), 6))
        n[:, 0], n[:, 1] = po[:, 0] / r, po[:, 1] / r
        scale = np.max(np.abs(co), axis=(1, 2))
        ev, evec = np.linalg.eigh(co)
        assert np.all(ev[:, 0] > -1e-12 * scale)
        assert np.all(np.abs(np.einsum("ni,ni->n", evec[:, :, 0], n)) > 0.99)
        # orthonormal basis of the complement of n: rotate (x, y) into (radial, tangential)
        B = np.zeros((len(po), 5, 6))
        B[:, 0, 0], B[:, 0, 1] = -n[:, 1], n[:, 0]
        for k in range(2, 6):
            B[:, k - 1, k] = 1.0
        Pc = np.einsum("nai,nij,nbj->nab", B, co, B)
        np.linalg.cholesky(Pc)
        assert np.min(np.linalg.eigvalsh(Pc)) > 0.0


@pytest.mark.parametrize("scatter", [True, False])
def test_pulls_and_chi2(scatter):
    """Over 1e4 simulated tracks the fitted parameters at the last layer have pulls of mean
    0 +- 0.03 and width 1 +- 0.05, and chi2 (ndf = 2 nHits - 5) has a flat p-value.
    The position pull is taken along the cylinder's tangent, the direction in which the
    covariance at the cylinder has its support."""
    stats = pytest.importorskip("scipy.stats")
    det = Detector() if scatter else Detector(x_over_x0=(0.0,) * 10)
    b, g, hits, _, (po, co, c2, nh) = _fit_event(det, EventSpec(seed=24, n_tracks=10000, scatter=scatter))
    tr = b.truth[:, -1]
    ph = np.arctan2(po[:, 1], po[:, 0])
    t = np.stack([-np.sin(ph), np.cos(ph)], 1)
    du = np.sum(t * (po[:, :2] - tr[:, :2]), 1)
    su = np.sqrt(np.einsum("ni,nij,nj->n", t, co[:, :2, :2], t))
    res = po - tr
    res[:, 4] = _wrap(res[:, 4])
    sd = np.sqrt(np.diagonal(co, axis1=1, axis2=2))
    pulls = np.column_stack([du / su, res[:, 2:] / sd[:, 2:]])
    assert np.all(np.abs(pulls.mean(0)) < 0.03), pulls.mean(0)
    assert np.all(np.abs(pulls.std(0) - 1.0) < 0.05), pulls.std(0)
    ndf = 2 * nh - 5
    assert abs(np.mean(c2 / ndf) - 1.0) < 0.03
    pv = stats.chi2.sf(c2, ndf)
    assert stats.kstest(pv, "uniform").pvalue > 1e-3


def test_scattering_noise_matches_simulated_kicks():
    """Whitened kicks of the generator (state after minus before the kick on one layer) must
    have the covariance Q the oracle adds: unit variance in theta and phi, and the q/pT
    change tied to the theta change by -(q/pT) cot(theta)."""
    det = Detector(x_over_x0=(0.0, 0.0, 0.05, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0))
    b = generate(EventSpec(seed=25, n_tracks=100000, smear=False), det)
    g = O.make_geom(det)
    l = 2
    before, after = b.truth[:, l], b.truth_after[:, l]
    d = after - before
    d[:, 4] = _wrap(d[:, 4])
    zth = np.empty(len(d))
    zph = np.empty(len(d))
    zw = np.empty(len(d))
    for i in range(len(d)):
        Q = O.scatter(g, l, before[i], np.zeros((6, 6)))
        zth[i] = d[i, 5] / math.sqrt(Q[5, 5])
        zph[i] = d[i, 4] / math.sqrt(Q[4, 4])
        zw[i] = d[i, 3] / math.sqrt(Q[3, 3]) * np.sign(Q[3, 5]) if Q[3, 3] > 0 else 0.0
    assert abs(np.var(zth) - 1.0) < 0.02
    assert abs(np.var(zph) - 1.0) < 0.02
    assert abs(np.mean(zth * zph)) < 0.01
    # the q/pT kick is (to first order) -(q/pT) cot(theta) times the theta kick: correlation 1
    # (away from cot(theta) = 0, where the first-order term vanishes)
    cot = 1.0 / np.tan(before[:, 5])
    m = np.abs(cot) > 0.2
    assert np.corrcoef(zw[m], zth[m])[0, 1] > 0.999


HIGHLAND = os.path.join(os.path.dirname(__file__), "golden", "highland.txt")


def test_scattering_width_hand_worked():
    """The width and the covariance terms of the scattering noise against cases worked by hand
    from the PDG's Highland formula (tests/golden/highland.txt, every step shown there): theta0 =
    sqrt(Q_theta_theta), and each of the four non-zero terms, to 1e-12 relative."""
    n = 0
    for line in open(HIGHLAND):
        if line.startswith("#") or not line.strip():
            continue
        x, y, z, w, phi, th, xx0, mass, th0, qww, qtw, qpp, qtt = (float(v) for v in line.split())
        det = Detector(x_over_x0=(xx0,) * 10, mass=mass)
        g = O.make_geom(det)
        Q = O.scatter(g, 4, np.array([x, y, z, w, phi, th]), np.zeros((6, 6)))
        assert math.sqrt(Q[5, 5]) == pytest.approx(th0, rel=1e-12, abs=0), line
        for (i, j), ref in (((3, 3), qww), ((5, 3), qtw), ((4, 4), qpp), ((5, 5), qtt)):
            assert Q[i, j] == pytest.approx(ref, rel=1e-12, abs=1e-43), (line, i, j)
            assert Q[j, i] == Q[i, j]
        # nothing else is touched: position rows and the phi-(w, theta) terms stay zero
        mask = np.ones((6, 6), bool)
        for i, j in ((3, 3), (5, 3), (3, 5), (4, 4), (5, 5)):
            mask[i, j] = False
        assert np.all(Q[mask] == 0.0)
        n += 1
    assert n == 4
