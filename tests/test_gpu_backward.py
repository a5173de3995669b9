"""Parity of tkf_fit_backward (the inward pass over a fitted track's hits, carrying the final
fit to the production point) with the oracle's backward pass, from the same states on the
outermost layer, in FP32, MIXED and FP64; holes, partial layer ranges, failed inputs, bad hit
ids and argument errors."""
import numpy as np
import pytest

import oracle as O
from _gpu import chi2_violations, device_hits, device_tracks, host_tracks, param_violations, rounded
from synth import Detector, EventSpec, generate

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1702_06359_gb300 import tkf  # noqa: E402

PRECS = [tkf.FP32, tkf.MIXED, tkf.FP64]
PNAME = {tkf.FP32: "fp32", tkf.MIXED: "mixed", tkf.FP64: "fp64"}


@pytest.fixture(scope="module")
def det():
    return Detector()


def _forward(det, n, seed, pt_max=10.0, holes=0.0, eta_max=1.0):
    """Generated tracks and the oracle's forward fit over all layers (the backward pass's input)."""
    b = generate(EventSpec(seed=seed, n_tracks=n, pt_max=pt_max, eta_max=eta_max), det)
    g = O.make_geom(det)
    hits = O.hits_of(b)
    ids = b.trk_hits.copy()
    if holes:
        h = np.random.default_rng(seed).random(ids.shape) < holes
        h[:, :3] = False
        ids[h] = -1
    par0, cov0 = O.seed_estimate(g, hits, ids[:, :3])
    pf, cf, c2, nh, st = O.fit(g, hits, par0, cov0, ids, 0, det.n_layers - 1)
    assert np.all(st == 0)
    return b, g, hits, ids, pf, cf, nh


def _gpu_backward(det, b, ids, par, cov, nhits, prec, last, first, scale, **cfg):
    ctx = tkf.Context(tkf.default_config(precision=prec, **cfg))
    init = device_tracks(par, cov, np.zeros(len(par)), nhits, ids, precision=prec)
    out = tkf.DeviceTracks.empty(len(par), det.n_layers, prec)
    ctx.fit_backward(device_hits(b), init, last, first, out, cov_scale=scale)
    ctx.sync_status()
    got = host_tracks(out)
    ctx.close()
    return got


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
@pytest.mark.parametrize("scale", [1.0, 1e4])
@pytest.mark.parametrize("pt_max", [10.0, 100.0])
def test_backward_parity(det, prec, scale, pt_max):
    """1000 tracks (the plain-fit workload's shapes): the pass from the forward fit's states on
    layer 10 to layer 1, against the oracle from the same (precision-rounded) states."""
    L = det.n_layers
    b, g, hits, ids, pf, cf, nh = _forward(det, 1000, 11, pt_max)
    pf, cf = rounded(pf, prec), rounded(cf, prec)
    ref = O.fit_backward(g, hits, pf, cf, ids, L - 1, 0, scale)
    assert np.all(ref[4] == 0)
    got = _gpu_backward(det, b, ids, pf, cf, nh, prec, L - 1, 0, scale)
    assert np.array_equal(got["nhits"], ref[3])
    bad, worst = param_violations(got["par"], ref[0])
    assert not bad.any(), worst
    bad, worst = chi2_violations(got["chi2"], ref[2])
    assert not bad.any(), worst
    if prec == tkf.FP64:  # the oracle's arithmetic type: far inside the stated bound
        assert param_violations(got["par"], ref[0], rel=1e-8)[1] <= 1.0
    assert np.array_equal(got["hit_idx"], ids)


@pytest.mark.parametrize("prec", [tkf.FP32, tkf.MIXED], ids=lambda p: PNAME[p])
def test_backward_with_holes_and_partial_range(det, prec):
    """Tracks missing 15 % of their hits on layers 4-10; passes over layers 8..3 and 5..5 from
    the forward fits over 0..7 and 0..4."""
    b, g, hits, ids, pf, cf, nh = _forward(det, 777, 12, holes=0.15)
    par0, cov0 = O.seed_estimate(g, hits, ids[:, :3])
    for last, first in ((7, 2), (4, 4)):
        pl, cl, _, nl, st = O.fit(g, hits, par0, cov0, ids, 0, last)
        assert np.all(st == 0)
        pl, cl = rounded(pl, prec), rounded(cl, prec)
        ref = O.fit_backward(g, hits, pl, cl, ids, last, first, 100.0)
        got = _gpu_backward(det, b, ids, pl, cl, nl, prec, last, first, 100.0)
        assert np.array_equal(got["nhits"], ref[3])
        assert np.array_equal(ref[3], (ids[:, first:last + 1] >= 0).sum(1))
        assert not param_violations(got["par"], ref[0])[0].any()
        assert not chi2_violations(got["chi2"], ref[2])[0].any()


def test_backward_failed_inputs_bad_ids_and_errors(det):
    L = det.n_layers
    b, g, hits, ids, pf, cf, nh = _forward(det, 64, 13)
    nh = nh.copy()
    nh[5] = tkf.TRACK_LOST
    got = _gpu_backward(det, b, ids, pf, cf, nh, tkf.FP32, L - 1, 0, 1e4)
    assert got["nhits"][5] == tkf.TRACK_LOST and np.all(np.delete(got["nhits"], 5) == L)
    # a hit id past the end: the kernel's error bit, that track SINGULAR, the others unchanged
    bad = ids.copy()
    bad[9, 6] = b.n_hits + 5
    ctx = tkf.Context(tkf.default_config())
    init = device_tracks(pf, cf, np.zeros(64), np.full(64, L), bad)
    out = tkf.DeviceTracks.empty(64, L)
    ctx.fit_backward(device_hits(b), init, L - 1, 0, out, cov_scale=1e4)
    with pytest.raises(tkf.TkfError):
        ctx.sync_status()
    r = host_tracks(out)
    assert r["nhits"][9] == tkf.TRACK_SINGULAR and np.all(np.delete(r["nhits"], 9) == L)
    # argument errors, and an empty batch
    dh = device_hits(b)
    for last, first, scale in ((2, 5, 1.0), (L, 0, 1.0), (L - 1, -1, 1.0), (L - 1, 0, 0.0), (L - 1, 0, float("inf"))):
        with pytest.raises(tkf.TkfError):
            ctx.fit_backward(dh, init, last, first, out, cov_scale=scale)
    empty = tkf.DeviceTracks.empty(0, L)
    ctx.fit_backward(dh, empty, L - 1, 0, tkf.DeviceTracks.empty(0, L), cov_scale=1e4)
    ctx.close()


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
def test_backward_parity_on_module_geometry(prec):
    """Hits on modules 0.5 cm inside and outside the layers' radii (hit_dr = 0.5 cm, |eta| < 2):
    the inward pass takes each state to its hit's own radius, as the oracle does."""
    det = Detector(module_dr=1.0)
    L = det.n_layers
    b, g, hits, ids, pf, cf, nh = _forward(det, 1000, 14, eta_max=2.0)
    pf, cf = rounded(pf, prec), rounded(cf, prec)
    ref = O.fit_backward(g, hits, pf, cf, ids, L - 1, 0, 1e4)
    assert np.all(ref[4] == 0)
    got = _gpu_backward(det, b, ids, pf, cf, nh, prec, L - 1, 0, 1e4, hit_dr=0.5)
    assert np.array_equal(got["nhits"], ref[3])
    bad, worst = param_violations(got["par"], ref[0])
    assert not bad.any(), worst
    bad, worst = chi2_violations(got["chi2"], ref[2])
    assert not bad.any(), worst
