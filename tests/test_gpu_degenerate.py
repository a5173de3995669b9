"""Degenerate tracks the method has to report rather than compute: curling tracks that cannot
reach the next cylinder.  The fit marks them TKF_TRACK_NOREACH where the oracle's propagation
reports no crossing, the building drops every candidate of a seed that cannot reach the first
building layer (TKF_TRACK_LOST, the oracle's zero candidates), and the backward pass marks a
track whose circle never comes back to the inner cylinder.  Every other track of the same
launch keeps its parity with the oracle."""
import math

import numpy as np
import pytest

import oracle as O
from _gpu import device_hits, device_tracks, host_tracks, param_violations, rounded
from synth import Detector, EventSpec, generate
from synth.events import K_B

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1702_06359_gb300 import tkf  # noqa: E402

PRECS = [tkf.FP32, tkf.FP64]
PNAME = {tkf.FP32: "fp32", tkf.FP64: "fp64"}


@pytest.fixture(scope="module")
def det():
    return Detector()


def _curl(det, radius_of_curvature):
    """q/pT (1/GeV, positive) of a track with the given radius of curvature in cm."""
    return 1.0 / (K_B * det.bz * radius_of_curvature)


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
def test_fit_reports_tracks_that_cannot_reach_a_cylinder(det, prec):
    """States on layer 1 without hits, every third one turned into a curler of radius 4.4 cm
    (it reaches at most 10.3 cm from the origin: layer 2 at 8 cm, not layer 3 at 12 cm)."""
    b = generate(EventSpec(seed=51, n_tracks=300), det)
    g = O.make_geom(det)
    hits = O.hits_of(b)
    L = det.n_layers
    par = b.truth[:, 0].copy()
    curl = np.arange(b.n_tracks) % 3 == 0
    par[curl, 3] = np.sign(par[curl, 3]) * _curl(det, 4.4)
    cov = np.tile(np.diag(np.square([0.01, 0.01, 0.1, 0.01, 0.001, 0.001])), (b.n_tracks, 1, 1))
    par, cov = rounded(par, prec), rounded(cov, prec)
    ids = np.full((b.n_tracks, L), -1, dtype=np.int32)
    ref = O.fit(g, hits, par, cov, ids, 0, L - 1)
    assert np.all(ref[4][curl] == 1) and np.all(ref[4][~curl] == 0)  # ORC_ERR_NOREACH
    ctx = tkf.Context(tkf.default_config(precision=prec))
    out = tkf.DeviceTracks.empty(b.n_tracks, L, prec)
    ctx.fit(device_hits(b), device_tracks(par, cov, np.zeros(b.n_tracks), np.zeros(b.n_tracks), ids, precision=prec),
            0, L - 1, out)
    ctx.sync_status()
    got = host_tracks(out)
    assert np.all(got["nhits"][curl] == tkf.TRACK_NOREACH)
    assert np.all(got["nhits"][~curl] == 0)
    assert not param_violations(got["par"][~curl], ref[0][~curl])[0].any()
    ctx.close()


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
def test_building_drops_seeds_that_cannot_reach_the_first_building_layer(det, prec):
    """Seeds on layer 3 turned into curlers of radius 1.76 cm (at most 13.9 cm from the origin,
    the first building layer is at 16 cm): every candidate is dropped, as in the oracle; the
    other seeds of the launch build as usual."""
    b = generate(EventSpec(seed=52, n_tracks=400, noise_frac=0.2), det)
    g = O.make_geom(det)
    hits = O.hits_of(b)
    L = det.n_layers
    from _helpers import oracle_seeds
    sp, sP, sc2, snh, sh = oracle_seeds(g, hits, b.trk_hits)
    curl = np.arange(b.n_tracks) % 4 == 1
    sp = sp.copy()
    sp[curl, 3] = np.sign(sp[curl, 3]) * _curl(det, 1.76)
    sp, sP, sc2 = rounded(sp, prec), rounded(sP, prec), rounded(sc2, prec)
    ref = O.build(g, O.hit_index(g, hits), sp, sP, sc2, snh, sh)
    assert np.all(ref.n_cand[curl] == 0)
    ctx = tkf.Context(tkf.default_config(precision=prec))
    idx = ctx.build_hit_index(device_hits(b))
    out = tkf.DeviceTracks.empty(b.n_tracks, L, prec)
    ctx.build_tracks(idx, device_tracks(sp, sP, sc2, snh, sh, precision=prec), out)
    ctx.sync_status()
    got = host_tracks(out)
    assert np.all(got["nhits"][curl] == tkf.TRACK_LOST)
    assert np.all(got["hit_idx"][curl][:, 3:] == -1) and np.array_equal(got["hit_idx"][curl][:, :3], sh[curl][:, :3])
    live = ~curl & (ref.n_cand > 0)
    same = np.all(got["hit_idx"] == ref.hits[:, 0, :], axis=1) & live
    assert same.sum() >= 0.95 * live.sum()
    assert not param_violations(got["par"][same], ref.par[same, 0])[0].any()
    ctx.close()


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
def test_backward_pass_reports_a_circle_that_never_returns_inward(det, prec):
    """States on layer 3 (12 cm) moving along the cylinder with a 3 cm radius of curvature
    centred outside it (15 cm from the origin): going back along the track the circle never
    comes within 12 cm of the beam line, so layer 2 (8 cm) is out of reach."""
    L = det.n_layers
    n = 64
    ang = np.linspace(-math.pi, math.pi, n, endpoint=False)
    par = np.zeros((n, 6))
    par[:, 0], par[:, 1] = 12.0 * np.cos(ang), 12.0 * np.sin(ang)
    par[:, 2] = 1.0
    par[:, 4] = np.arctan2(np.sin(ang + math.pi / 2), np.cos(ang + math.pi / 2))  # along the cylinder, counter-clockwise
    par[:, 3] = _curl(det, 3.0)  # q/pT > 0: curvature -K Bz q/pT < 0, centre on the outer side
    par[:, 5] = 1.2
    normal = np.arange(n) % 2 == 0  # half of them: an ordinary outgoing 2 GeV track
    par[normal, 4] = np.arctan2(np.sin(ang[normal]), np.cos(ang[normal]))
    par[normal, 3] = 0.5
    cov = np.tile(np.diag(np.square([0.01, 0.01, 0.1, 0.01, 0.001, 0.001])), (n, 1, 1))
    par, cov = rounded(par, prec), rounded(cov, prec)
    b = generate(EventSpec(seed=53, n_tracks=1), det)  # any hits: the pass uses none of them
    g = O.make_geom(det)
    ids = np.full((n, L), -1, dtype=np.int32)
    ref = O.fit_backward(g, O.hits_of(b), par, cov, ids, 2, 0, 1.0)
    assert np.all(ref[4][~normal] == 1) and np.all(ref[4][normal] == 0)
    ctx = tkf.Context(tkf.default_config(precision=prec))
    out = tkf.DeviceTracks.empty(n, L, prec)
    ctx.fit_backward(device_hits(b), device_tracks(par, cov, np.zeros(n), np.zeros(n), ids, precision=prec), 2, 0,
                     out, cov_scale=1.0)
    ctx.sync_status()
    got = host_tracks(out)
    assert np.all(got["nhits"][~normal] == tkf.TRACK_NOREACH)
    assert np.all(got["nhits"][normal] == 0)
    assert not param_violations(got["par"][normal], ref[0][normal])[0].any()
    ctx.close()


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
def test_two_step_fit_reports_a_module_out_of_reach(prec):
    """Hits on modules off the cylinders (hit_dr = 0.5 cm), layers at 6.9 and 8 cm: curlers of
    radius 4.05 cm from the origin reach at most 8.1 cm, past the 8 cm layer's average radius
    and its inner modules (7.5 cm) but short of its outer modules (8.5 cm).  A track whose
    second hit lies on an outer module is reported TKF_TRACK_NOREACH, as the oracle finds no
    crossing of the hit's radius; with the hit on an inner module it is fitted, at parity.
    (The first layer sits close to the second so that the step stays within the straight-line
    start of the GPU's Newton solve: a 4 cm radius of curvature is 46 MeV of pT.)"""
    radii = (6.9,) + tuple(4.0 * (l + 1) for l in range(1, 10))
    det = Detector(radii=radii, x_over_x0=(0.0,) * 10, module_dr=1.0)
    g = O.make_geom(det)
    L = det.n_layers
    n = 64
    w = 1.0 / (K_B * det.bz * 4.05)
    start = np.zeros((n, 6))
    hits = np.zeros(2 * n, dtype=O.HIT_DTYPE)
    ids = np.full((n, L), -1, dtype=np.int32)
    outer = np.arange(n) % 2 == 1
    for t in range(n):
        v = np.array([0.0, 0.0, 0.0, w if t % 4 < 2 else -w, -math.pi + 2 * math.pi * t / n, 1.2])
        st, p1, _ = O.propagate(g, v, radii[0])
        assert st == 0
        start[t] = p1
        st, p2, _ = O.propagate(g, p1, 7.5)  # the crossing of the inner module radius
        assert st == 0
        r2 = 8.5 if outer[t] else 7.5
        ph = math.atan2(p2[1], p2[0])
        hits[2 * t] = (p1[0], p1[1], p1[2], det.sigma_rphi ** 2, det.sigma_z ** 2, 0, 0)
        hits[2 * t + 1] = (r2 * math.cos(ph), r2 * math.sin(ph), p2[2], det.sigma_rphi ** 2, det.sigma_z ** 2, 1, 0)
        ids[t, 0], ids[t, 1] = 2 * t, 2 * t + 1
    # the oracle on the float-rounded hits the GPU reads
    for k in ("x", "y", "z", "var_u", "var_v"):
        hits[k] = hits[k].astype(np.float32)
    cov = np.tile(np.diag(np.square([0.01, 0.01, 0.1, 0.01, 0.001, 0.001])), (n, 1, 1))
    start, cov = rounded(start, prec), rounded(cov, prec)
    ref = O.fit(g, hits, start, cov, ids, 0, 1)
    assert np.all(ref[4][outer] == 1) and np.all(ref[4][~outer] == 0)  # ORC_ERR_NOREACH

    class _Hits:
        x, y, z = hits["x"], hits["y"], hits["z"]
        var_u, var_v, layer = hits["var_u"], hits["var_v"], hits["layer"]
        hit_off = np.array([0, 2 * n])
    ctx = tkf.Context(tkf.default_config(precision=prec, hit_dr=0.5, radius=radii, x_over_x0=det.x_over_x0))
    out = tkf.DeviceTracks.empty(n, L, prec)
    ctx.fit(device_hits(_Hits), device_tracks(start, cov, np.zeros(n), np.zeros(n), ids, precision=prec), 0, 1, out)
    ctx.sync_status()
    got = host_tracks(out)
    assert np.all(got["nhits"][outer] == tkf.TRACK_NOREACH)
    assert np.all(got["nhits"][~outer] == 2)
    assert not param_violations(got["par"][~outer], ref[0][~outer])[0].any()
    ctx.close()
