"""Pins of the oracle's backward (inward) pass over a fitted track's hits, the refinement of the
final fit towards the production point (Sec. 2; the next row after building and fitting).

References used instead of the oracle itself: noise-free tracks (the pass must return the
generator's truth on the innermost layer), the batch weighted least-squares information on the
innermost layer built by central differences of a backward helix crossing written in the
test (the inward filter must reproduce it), unit-width pulls on simulated tracks with scattering, and a round trip outward and back
inward that must return the starting state and covariance."""
import math

import numpy as np
import pytest

import oracle as O
from synth import Detector, EventSpec, generate
from synth.events import K_B


def _wrap(a):
    return (np.asarray(a) + math.pi) % (2 * math.pi) - math.pi


def _forward_then_backward(det, spec, scale, settings=O.Settings()):
    b = generate(spec, det)
    g = O.make_geom(det, settings)
    hits = O.hits_of(b, exact=spec.keep_f64)
    L = det.n_layers
    par0, cov0 = O.seed_estimate(g, hits, b.trk_hits[:, :3])
    pf, cf, _, _, st = O.fit(g, hits, par0, cov0, b.trk_hits, 0, L - 1)
    assert np.all(st == 0)
    pb, cb, c2, nh, st = O.fit_backward(g, hits, pf, cf, b.trk_hits, L - 1, 0, scale)
    assert np.all(st == 0)
    return b, g, hits, (pf, cf), (pb, cb, c2, nh)


def test_noise_free_tracks_return_truth_on_the_innermost_layer():
    det = Detector(x_over_x0=(0.0,) * 10)
    b, g, hits, _, (pb, cb, c2, nh) = _forward_then_backward(
        det, EventSpec(seed=31, n_tracks=400, scatter=False, smear=False, keep_f64=True), scale=100.0)
    d = pb - b.truth[:, 0]
    d[:, 4] = _wrap(d[:, 4])
    assert np.max(np.abs(d)) < 1e-9
    assert np.max(c2) < 1e-12
    assert np.all(nh == det.n_layers)
    # a pass that stops on an intermediate layer returns the truth there
    L = det.n_layers
    p4, _, _, nh4, st = O.fit_backward(g, hits, b.truth[:, -1], np.tile(np.eye(6), (b.n_tracks, 1, 1)), b.trk_hits,
                                       L - 1, 4, 1.0)
    d4 = p4 - b.truth[:, 4]
    d4[:, 4] = _wrap(d4[:, 4])
    assert np.all(st == 0) and np.max(np.abs(d4)) < 1e-9 and np.all(nh4 == L - 4)


def _backward_crossing(state, radius, kb):
    """The previous crossing of r = radius (< the state's radius) along the helix through
    `state`: the negative transverse path s closest to 0 with |(x(s), y(s))| = radius, bracketed
    by steps back along the helix, then bisected and polished by Newton's method (written here,
    independently of the oracle's reversal of the track)."""
    x, y, z, w, phi, th = state
    kappa = -kb * w

    def pos(s):
        ang = phi + kappa * s
        return x + (math.sin(ang) - math.sin(phi)) / kappa, y - (math.cos(ang) - math.cos(phi)) / kappa, ang

    def excess(s):
        xs, ys, _ = pos(s)
        return xs * xs + ys * ys - radius * radius

    step = 0.2  # cm of transverse path: finer than the dip of r(s) near a track's origin
    hi, lo = 0.0, -step
    while excess(lo) > 0.0:
        hi, lo = lo, lo - step
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if excess(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    s = 0.5 * (lo + hi)
    for _ in range(2):
        xs, ys, ang = pos(s)
        s -= excess(s) / (2.0 * (xs * math.cos(ang) + ys * math.sin(ang)))
    xs, ys, ang = pos(s)
    assert s < 0 and abs(math.hypot(xs, ys) - radius) < 1e-9
    return np.array([xs, ys, z + s * math.cos(th) / math.sin(th), w, math.atan2(math.sin(ang), math.cos(ang)), th])


@pytest.mark.parametrize("scale", [1.0, 3e3])
def test_covariance_equals_batch_least_squares_information(scale):
    """Noise-free track, no material, pass started at the truth on the outermost layer with
    covariance P_s and covariance scale c: the covariance on the innermost layer must equal
    T ((c P_s)^-1 + sum_l B_l^T V^-1 B_l)^-1 T^T, with B_l = d(u_l, v_l)/d(start state) and
    T = d(state on layer 1)/d(start state) taken by central differences of a backward helix
    crossing written in this test (not the oracle's reversal of the track)."""
    det = Detector(x_over_x0=(0.0,) * 10)
    b = generate(EventSpec(seed=32, n_tracks=10, scatter=False, smear=False, keep_f64=True), det)
    g = O.make_geom(det)
    hits = O.hits_of(b, exact=True)
    L = det.n_layers
    kb = K_B * det.bz
    Ps = np.diag(np.square([0.05, 0.05, 0.5, 0.02, 0.01, 0.01]))
    V = np.diag([det.sigma_rphi ** 2, det.sigma_z ** 2]).astype(np.float32).astype(np.float64)

    def inward(ps):
        """positions on layers L-1..0 and the state on layer 0, from the start state ps"""
        meas = {L - 1: ps[:3].copy()}
        st = ps
        for l in range(L - 2, -1, -1):
            st = _backward_crossing(ps, det.radii[l], kb)
            meas[l] = st[:3]
        return meas, st

    for t in range(b.n_tracks):
        ps = b.truth[t, -1].copy()
        ids = b.trk_hits[t]
        pb, cb, _, _, st = O.fit_backward(g, hits, ps[None], Ps[None], ids[None], L - 1, 0, scale)
        assert st[0] == 0
        B = np.zeros((L, 2, 6))
        T = np.zeros((6, 6))
        for j in range(6):
            h = 1e-6 if j in (0, 1, 2) else 1e-7
            pp, pm = ps.copy(), ps.copy()
            pp[j] += h
            pm[j] -= h
            mp, sp = inward(pp)
            mm, sm = inward(pm)
            for l in range(L):
                ph = math.atan2(hits["y"][ids[l]], hits["x"][ids[l]])
                tx, ty = -math.sin(ph), math.cos(ph)
                B[l, 0, j] = (tx * (mp[l][0] - mm[l][0]) + ty * (mp[l][1] - mm[l][1])) / (2 * h)
                B[l, 1, j] = (mp[l][2] - mm[l][2]) / (2 * h)
            d = sp - sm
            d[4] = _wrap(d[4])
            T[:, j] = d / (2 * h)
        info = np.linalg.inv(scale * Ps)
        for l in range(L):
            info += B[l].T @ np.linalg.inv(V) @ B[l]
        Pb = T @ np.linalg.inv(info) @ T.T
        rel = np.abs(cb[0] - Pb) / np.sqrt(np.outer(np.diag(Pb), np.diag(Pb)) + 1e-30)
        assert np.max(rel) < 1e-5, (t, np.max(rel))
        d = pb[0] - b.truth[t, 0]
        d[4] = _wrap(d[4])
        assert np.max(np.abs(d)) < 1e-9


def test_pulls_and_chi2_on_the_innermost_layer():
    """Over 1e4 simulated tracks with scattering, the backward state on layer 1 has pulls of
    mean 0 +- 0.03 and width 1 +- 0.05 against the generator's truth there (the position pull
    along the cylinder's tangent), and chi2 / (2 nHits - 5) averages 1 +- 0.05 (the starting
    state's information is discounted by the scale 1e4)."""
    det = Detector()
    b, g, hits, _, (pb, cb, c2, nh) = _forward_then_backward(det, EventSpec(seed=33, n_tracks=10000), scale=1e4)
    tr = b.truth[:, 0]
    ph = np.arctan2(pb[:, 1], pb[:, 0])
    t = np.stack([-np.sin(ph), np.cos(ph)], 1)
    du = np.sum(t * (pb[:, :2] - tr[:, :2]), 1)
    su = np.sqrt(np.einsum("ni,nij,nj->n", t, cb[:, :2, :2], t))
    res = pb - tr
    res[:, 4] = _wrap(res[:, 4])
    sd = np.sqrt(np.diagonal(cb, axis1=1, axis2=2))
    pulls = np.column_stack([du / su, res[:, 2:] / sd[:, 2:]])
    assert np.all(np.abs(pulls.mean(0)) < 0.03), pulls.mean(0)
    assert np.all(np.abs(pulls.std(0) - 1.0) < 0.05), pulls.std(0)
    assert abs(np.mean(c2 / (2 * nh - 5)) - 1.0) < 0.05


def test_reversal_is_exact_for_the_propagation():
    """Carrying a state outward over four layers and back inward with no hits and no material
    returns it and its covariance (the same helix run backwards; the two transports are inverse
    maps between the cylinders)."""
    det = Detector(x_over_x0=(0.0,) * 10)
    b = generate(EventSpec(seed=35, n_tracks=200, scatter=False, smear=False, keep_f64=True), det)
    g = O.make_geom(det)
    hits = O.hits_of(b, exact=True)
    ids = np.full_like(b.trk_hits, -1)
    # a covariance on the cylinder (no radial position spread, which a crossing cannot keep)
    ph = np.arctan2(b.truth[:, 2, 1], b.truth[:, 2, 0])
    tang = np.stack([-np.sin(ph), np.cos(ph)], 1)
    P0 = np.tile(np.diag(np.square([0.0, 0.0, 0.1, 0.01, 0.001, 0.001])), (b.n_tracks, 1, 1))
    P0[:, :2, :2] = 0.01 ** 2 * np.einsum("ni,nj->nij", tang, tang)
    po, co, _, _, st = O.fit(g, hits, b.truth[:, 2], P0, ids, 2, 6)
    assert np.all(st == 0)
    pb, cbk, _, nh, st = O.fit_backward(g, hits, po, co, ids, 6, 2, 1.0)
    assert np.all(st == 0) and np.all(nh == 0)
    d = pb - b.truth[:, 2]
    d[:, 4] = _wrap(d[:, 4])
    assert np.max(np.abs(d)) < 1e-9
    # without hits and material the covariance returns too
    scale_ = np.sqrt(np.einsum("nii,njj->nij", P0, P0)) + 1e-30
    assert np.max(np.abs(cbk - P0) / np.maximum(scale_, 1e-12)) < 1e-6
