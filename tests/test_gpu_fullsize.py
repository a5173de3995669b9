"""Parity at the full batched size, in the launch configuration bench.py times: the 640-event
lognormal batch (2.6 M seeds, 35 M hits) through the graph-replayed pipeline with seed ordering
and the autotuned work tile, compared with the oracle on a seeded sample of seeds (the oracle
builds and fits them one event at a time), plus properties checked on every seed; then the
backward pass (tkf_fit_backward) over every fitted track, sampled against the oracle's.  The
same in MIXED precision, and for the bench's two-step case (the batch's first 160 events on
modules 0.5 cm off the layers' cylinders, hit_dr = 0.5 cm) and its endcap case (all 640 events,
each with a quarter of its tracks, on ten pairs of disks)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
from _gpu import chi2_violations, divergence_allowed, param_violations, unpack_cov
from synth import Detector

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1702_06359_gb300 import tkf  # noqa: E402

N_SAMPLE_EVENTS, SEEDS_PER_EVENT = 48, 40
# On the disks the fit takes q/pT from the small sagitta across planes 8 cm apart (a short
# radial lever arm), and FP32 rounding in the covariance carries about 1e-4 relative into it:
# 1.35e-4 at most over this sample, about 1e-3 of the estimate's own sigma.  q/pT is held to
# 2e-4 relative there (the other parameters to the barrel's 1e-4), and every track's q/pT
# difference to 5e-3 of its sigma.
ENDCAP_PAR_REL = np.array([1e-4, 1e-4, 1e-4, 2e-4, 1e-4, 1e-4])


def _batch(n_events, module_dr=0.0, forward=False):
    import bench
    with mp.get_context("spawn").Pool(min(os.cpu_count() or 1, 16)) as pool:
        return bench.workload(3, n_events, pool, module_dr=module_dr, forward=forward)


def test_full_batch_sampled_parity_and_properties():
    _check_batch(_batch(640), Detector(), {}, N_SAMPLE_EVENTS)


def test_full_batch_mixed_precision_sampled_parity_and_properties():
    """The bench's MIXED leg: the same batch and launch configuration with the FP64 innovation
    inverse and Joseph update (the block's updates packed into full warps)."""
    _check_batch(_batch(640), Detector(), {"precision": tkf.MIXED}, 24)


def test_two_step_batch_sampled_parity_and_properties():
    _check_batch(_batch(160, module_dr=1.0), Detector(module_dr=1.0), {"hit_dr": 0.5}, 32)


def test_endcap_batch_sampled_parity_and_properties():
    """The bench's endcap leg: 650 k forward tracks on the disks, the oracle with the endcap
    settings; the backward pass with covariance scale 1e2 (in FP32 a scale of 1e4 leaves too few
    digits of the forward information on the first disks, as the endcap parity tests note)."""
    import bench
    from synth import FORWARD_PRIOR, forward_detector
    det = forward_detector()
    settings = O.Settings(eta_min=-3.0, n_eta_bins=60, prior_sigma=FORWARD_PRIOR)
    _check_batch(_batch(640, forward=True), det, bench.forward_config(tkf, seed_order=1, seeds_per_block=5), 48,
                 settings=settings, cov_scale=1e2, min_live=0.99, par_rel=ENDCAP_PAR_REL, qpt_sigma_frac=5e-3)


def test_largest_event_sampled_parity_and_properties():
    """One event at the workload's largest size: 20 000 tracks (the clip of the lognormal track
    count) with 50 % noise hits (the top of the noise range), 300 000 hits."""
    from synth import EventSpec, generate
    b = generate(EventSpec(seed=99, n_events=1, n_tracks=20000, noise_frac=0.5))
    _check_batch(b, Detector(), {}, 1, seeds_per_event=400)


def _check_batch(b, det, cfg, n_sample_events, seeds_per_event=SEEDS_PER_EVENT, settings=None, cov_scale=1e4,
                 min_live=0.999, par_rel=1e-4, qpt_sigma_frac=None):
    """cfg: keyword settings of the library configuration, or a whole tkf_config."""
    L = det.n_layers
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(dev)
    hits = tkf.DeviceHits(t(b.x, torch.float32), t(b.y, torch.float32), t(b.z, torch.float32),
                          t(b.var_u, torch.float32), t(b.var_v, torch.float32), t(b.layer, torch.int32),
                          t(b.hit_off, torch.int32))
    sh, se = t(b.trk_hits[:, :3].T, torch.int32), t(b.trk_event, torch.int32)
    n = b.n_tracks
    ctx = tkf.Context(cfg if isinstance(cfg, tkf.Config) else tkf.default_config(seed_order=1, seeds_per_block=5, **cfg))
    pipe = tkf.DevicePipeline(ctx, b.n_hits, b.n_events, n, use_graph=True)
    for _ in range(2):  # capture, then a replay
        pipe.run(hits, sh, se, n)
    ctx.sync_status()
    assert pipe.captures() == 1
    _, built, fitted = pipe.outputs()
    bt, ft = tkf.tracks_tensors(built, L), tkf.tracks_tensors(fitted, L)
    hid = bt["hit_idx"][:, :n].T.cpu().numpy()
    bnh = bt["nhits"][:n].cpu().numpy()
    par = ft["par"][:, :n].double().T.cpu().numpy()
    chi2 = ft["chi2"][:n].double().cpu().numpy()
    fnh = ft["nhits"][:n].cpu().numpy()
    cov_diag = ft["cov"][[0, 2, 5, 9, 14, 20], :n].double().cpu().numpy()

    # properties of every seed
    ev = b.trk_event
    lo, hi = b.hit_off[ev], b.hit_off[ev + 1]
    ok = (hid < 0) | ((hid >= lo[:, None]) & (hid < hi[:, None]))
    assert ok.all(), "a hit id outside its seed's event"
    assert np.array_equal(hid[:, :3], b.trk_hits[:, :3]), "seed hits must stay on layers 0-2"
    live = bnh >= 0
    assert live.mean() > min_live
    assert np.array_equal((hid[live] >= 0).sum(1), bnh[live]), "nhits counts the built hits"
    # a state on a disk has its z fixed by the plane: the z variance is zero there
    on_disk = bool(np.any(np.asarray(getattr(det, "disk_z", ())) > 0))
    pos = [0, 1, 3, 4, 5] if on_disk else list(range(6))
    assert np.all(chi2[live] >= 0) and np.all(cov_diag[pos][:, live] > 0)
    if on_disk:
        assert np.all(cov_diag[2, live] >= 0)
    layers = np.where(hid >= 0, b.layer[np.maximum(hid, 0)], -1)
    assert np.all((hid < 0) | (layers == np.arange(L)[None, :])), "hit of layer l in slot l"

    # sampled seeds against the oracle, one event at a time
    g = O.make_geom(det, settings) if settings is not None else O.make_geom(det)
    rng = np.random.default_rng(1702)
    events = np.sort(rng.choice(b.n_events, n_sample_events, replace=False))
    n_cmp = n_div = 0
    bw_samples = []
    for e in events:
        h0, h1, t0, t1 = b.hit_off[e], b.hit_off[e + 1], b.trk_off[e], b.trk_off[e + 1]
        if t1 == t0:
            continue
        s = np.sort(rng.choice(np.arange(t0, t1), min(seeds_per_event, t1 - t0), replace=False))
        oh = O.hits_of(b, slice(h0, h1))
        local = b.trk_hits[s] - h0
        p0, c0 = O.seed_estimate(g, oh, local[:, :3])
        ids = np.full((len(s), L), -1, dtype=np.int32)
        ids[:, :3] = local[:, :3]
        sp, sP, sc2, snh, _ = O.fit(g, oh, p0, c0, ids, 0, 2)
        res = O.build(g, O.hit_index(g, oh), sp, sP, sc2, snh, ids)
        rh = res.hits[:, 0, :]
        gh = np.where(hid[s] >= 0, hid[s] - h0, -1)
        lost = res.n_cand == 0
        assert np.all(bnh[s[lost]] == tkf.TRACK_LOST)
        same = np.all(gh == rh, axis=1) & ~lost
        for k in np.nonzero(~same & ~lost)[0]:
            assert divergence_allowed(gh[k], res, k), ("hit list differs before any fragile decision", e, s[k])
            n_div += 1
        m = np.nonzero(same)[0]
        fpar, fcov, fchi2, fn, _ = O.fit(g, oh, p0[m], c0[m], rh[m], 0, L - 1)
        assert not param_violations(par[s[m]], fpar, rel=par_rel)[0].any(), param_violations(par[s[m]], fpar, rel=par_rel)[1]
        if qpt_sigma_frac is not None:
            assert np.all(np.abs(par[s[m], 3] - fpar[:, 3]) <= qpt_sigma_frac * np.sqrt(fcov[:, 3, 3]))
        assert not chi2_violations(chi2[s[m]], fchi2)[0].any()
        assert np.array_equal(fnh[s[m]], fn)
        n_cmp += len(s)
        bw_samples.append((oh, s[m], rh[m]))
    assert n_cmp > 0.6 * seeds_per_event * n_sample_events and n_div <= 0.05 * n_cmp, (n_cmp, n_div)

    # the backward pass over every fitted track (tkf_fit_backward, layer 10 -> 1), the sampled
    # seeds against the oracle's pass from the same (float32) states
    class _Raw:  # the pipeline's output struct where the binding expects a DeviceTracks
        def __init__(self, t):
            self.t = t

        def struct(self):
            return self.t
    back = tkf.DeviceTracks.empty(n, L)
    ctx.fit_backward(hits, _Raw(fitted), L - 1, 0, back, cov_scale=cov_scale, hit_idx=bt["hit_idx"])
    ctx.sync_status()
    bk = dict(par=back.par, cov=back.cov, chi2=back.chi2, nhits=back.nhits)
    bnh2 = bk["nhits"][:n].cpu().numpy()
    live = fnh >= 0
    assert np.array_equal(bnh2[live], fnh[live]) and np.all(bnh2[~live] < 0)
    assert np.all(bk["chi2"][:n].cpu().numpy()[live] >= 0)
    assert np.all(bk["cov"][[0, 2, 5, 9, 14, 20], :n].cpu().numpy()[pos][:, live] > 0)
    bpar = bk["par"][:, :n].double().T.cpu().numpy()
    bchi2 = bk["chi2"][:n].double().cpu().numpy()
    fcov_all = ft["cov"][:, :n]
    n_bw = 0
    for oh, idx, rh in bw_samples:
        if not len(idx):
            continue
        init_cov = unpack_cov(fcov_all[:, idx].double().cpu().numpy())
        rp, _, rc2, rn, rst = O.fit_backward(g, oh, par[idx], init_cov, rh, L - 1, 0, cov_scale)
        assert np.all(rst == 0)
        assert np.array_equal(bnh2[idx], rn)
        assert not param_violations(bpar[idx], rp, rel=par_rel)[0].any(), param_violations(bpar[idx], rp, rel=par_rel)[1]
        assert not chi2_violations(bchi2[idx], rc2)[0].any()
        n_bw += len(idx)
    assert n_bw > 0.6 * seeds_per_event * n_sample_events
    pipe.close()
    ctx.close()
    pipe.close()
    ctx.close()
