"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded
inputs.  Tolerances: parameters |d| <= 1e-4 max(|ref|, floor) with floors
(1, 1, 1 cm, 0.1 GeV^-1, 1, 1 rad), chi2 |d| <= 1e-3 max(chi2, 1), phi compared modulo 2 pi;
hit assignment identical except for seeds whose oracle decisions were fragile (two ranked
chi2 within 1e-3 of each other, or a chi2 within 1e-3 of the cut) at or before the first
differing layer."""
import numpy as np
import pytest

import oracle as O
from _gpu import (chi2_violations, device_hits, device_tracks, divergence_allowed, host_tracks, param_violations,
                  rounded)
from _helpers import oracle_seeds, select_events, small_event
from synth import Detector, EventSpec, event_sizes, generate

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


def _ctx(prec=tkf.FP32, **kw):
    return tkf.Context(tkf.default_config(precision=prec, **kw))


# ------------------------------------------------------------------ hit index

def test_hit_index_matches_oracle_bins(det):
    """Same bin contents as the oracle's index (bit for bit, up to hits within rounding of a
    bin edge); inside a bin the GPU orders hits by (phi sixteenth of the bin, id) instead of by
    id, and records where each sixteenth starts."""
    b = generate(EventSpec(seed=41, n_events=3, n_tracks=[1500, 0, 2500], noise_frac=0.3), det)
    ctx = _ctx()
    idx = ctx.build_hit_index(device_hits(b))
    torch.cuda.synchronize()
    ctx.sync_status()
    v = idx.view()
    n, L, NB = b.n_hits, det.n_layers, v.n_bins
    xyzi = _copy_dev(v.hit_xyzi, n * 4, torch.float32).view(n, 4).cpu().numpy()
    nbt = b.n_events * L * NB
    sub = _copy_dev(v.bin_sub, nbt * 4, torch.int32).view(nbt, 4).cpu().numpy().view(np.uint32)
    off = _copy_dev(v.bin_off, nbt + 1, torch.int32).cpu().numpy()
    pos = _copy_dev(v.pos_of_hit, n, torch.int32).cpu().numpy()
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 0)
    ids = xyzi[:, 3].view(np.int32)
    starts = np.zeros((nbt, 17), dtype=np.int64)  # start of each of the 16 phi sixteenths, and the count
    for t in range(1, 16):
        starts[:, t] = (sub[:, (t - 1) // 4] >> (8 * ((t - 1) % 4))) & 0xFF
    starts[:, 16] = np.diff(off)
    g = O.make_geom(det)
    n_edge = 0
    for e in range(b.n_events):
        h0, h1 = b.hit_off[e], b.hit_off[e + 1]
        hits = O.hits_of(b, slice(h0, h1))
        oi = O.hit_index(g, hits)
        for l in range(L):
            for bb in range(NB):
                k = (e * L + l) * NB + bb
                got = ids[off[k]:off[k + 1]]
                cnt = len(got)
                assert np.all(pos[h0 + got] == np.arange(off[k], off[k + 1]))
                if cnt:
                    # sixteenths: recorded starts are monotone and every hit lies in its own
                    assert np.all(np.diff(starts[k]) >= 0) and starts[k, 16] == cnt
                    coord = (np.arctan2(b.y[h0 + got].astype(np.float64), b.x[h0 + got]) + np.pi) * 63 / (2 * np.pi)
                    frac = np.clip((coord - bb % 63) * 16, 0, 15.999999)
                    sb = np.floor(frac).astype(int)
                    for j in range(cnt):
                        lo, hi = starts[k, sb[j]], starts[k, sb[j] + 1]
                        if not (lo <= j < hi):
                            assert abs(frac[j] - round(frac[j])) < 1e-4, (k, j, frac[j])
                    for t in range(16):
                        seg_ids = got[starts[k, t]:starts[k, t + 1]]
                        assert np.all(np.diff(seg_ids) > 0)
                ref = oi.order[oi.bin_off[l, bb]:oi.bin_off[l, bb + 1]]
                if not np.array_equal(np.sort(got), ref):
                    # only hits within rounding of a bin edge may land in the neighbouring bin
                    for hid in np.setxor1d(got, ref):
                        h = hits[hid]
                        eta = (np.arcsinh(h["z"] / det.radii[l]) + 2.0) / 0.1
                        ph = (np.arctan2(h["y"], h["x"]) + np.pi) / (2 * np.pi) * 63
                        edge = min(abs(eta - round(eta)), abs(ph - round(ph)))
                        assert edge < 1e-4, (e, l, bb, hid, eta, ph)
                        n_edge += 1
    assert n_edge <= 4


def test_hit_index_one_block_per_event_equals_multi_launch_index(det):
    """A batch with at least twice as many events as SMs takes the one-block-per-event kernel, a
    smaller one the multi-launch path (global counts and scans); the index of the whole batch
    must equal the two halves' indices laid end to end, bit for bit."""
    from synth import event_sizes
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    n_ev = 2 * sm + 40
    sizes, noise = event_sizes(43, n_ev, median=120, lo=0, hi=900)
    b = generate(EventSpec(seed=43, n_events=n_ev, n_tracks=sizes, noise_frac=noise), det)
    ctx = _ctx()
    L, NB = det.n_layers, ctx.cfg.n_eta_bins * ctx.cfg.n_phi_bins

    def arrays(bb):
        idx = ctx.build_hit_index(device_hits(bb))
        torch.cuda.synchronize()
        ctx.sync_status()
        v = idx.view()
        n, nbt = bb.n_hits, bb.n_events * L * NB
        out = dict(xyzi=_copy_dev(v.hit_xyzi, n * 4, torch.float32).cpu().numpy().view(np.int32),
                   var=_copy_dev(v.hit_var, n * 2, torch.float32).cpu().numpy().view(np.int32),
                   sub=_copy_dev(v.bin_sub, nbt * 4, torch.int32).cpu().numpy(),
                   off=_copy_dev(v.bin_off, nbt + 1, torch.int32).cpu().numpy(),
                   pos=_copy_dev(v.pos_of_hit, n, torch.int32).cpu().numpy(),
                   vmax=_copy_dev(v.var_max, bb.n_events * L * 2, torch.float32).cpu().numpy().view(np.int32))
        idx.free()
        return out

    full = arrays(b)
    half = n_ev // 2
    a1 = arrays(select_events(b, list(range(half))))
    a2 = arrays(select_events(b, list(range(half, n_ev))))
    n1 = int(b.hit_off[half])
    assert np.array_equal(full["xyzi"], np.concatenate([a1["xyzi"], a2["xyzi"]]))
    assert np.array_equal(full["var"], np.concatenate([a1["var"], a2["var"]]))
    assert np.array_equal(full["sub"], np.concatenate([a1["sub"], a2["sub"]]))
    assert np.array_equal(full["off"], np.concatenate([a1["off"][:-1], a2["off"] + n1]))
    assert np.array_equal(full["pos"], np.concatenate([a1["pos"], a2["pos"] + n1]))
    assert np.array_equal(full["vmax"], np.concatenate([a1["vmax"], a2["vmax"]]))


@pytest.mark.parametrize("n_events", [1, 160], ids=["multi_launch", "one_block_per_event"])
def test_event_over_the_hit_limit_is_reported(n_events):
    """Event-local hit ids are 23-bit fields: an event of 2^23 + 5 hits makes the index raise
    its error bit (both index paths: one event takes the multi-launch path, 160 events the
    one-block-per-event kernel); the ids wrap inside the event's own range, so nothing is
    accessed outside it.  630 phi bins keep ~33 hits per bin."""
    import math
    big = (1 << 23) + 5
    sizes = np.full(n_events, 10)
    sizes[0] = big
    n = int(sizes.sum())
    cfg = tkf.default_config(n_phi_bins=630)
    L = cfg.n_layers
    rng = np.random.default_rng(7)
    layer = rng.integers(0, L, n).astype(np.int32)
    R = np.array([cfg.radius[l] for l in range(L)])[layer]
    phi = rng.uniform(-math.pi, math.pi, n)
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(dev)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    hits = tkf.DeviceHits(t(R * np.cos(phi), torch.float32), t(R * np.sin(phi), torch.float32),
                          t(rng.uniform(-0.8, 0.8, n) * R, torch.float32), t(np.full(n, 1e-4), torch.float32),
                          t(np.full(n, 1e-2), torch.float32), t(layer, torch.int32), t(off, torch.int32))
    ctx = tkf.Context(cfg)
    idx = ctx.build_hit_index(hits)
    with pytest.raises(tkf.TkfError, match="8388606"):
        ctx.sync_status()
    idx.free()
    # a batch within the limit on the same context reports nothing
    ok = tkf.DeviceHits(*(getattr(hits, k)[:int(off[1]) - 6] for k in ("x", "y", "z", "var_u", "var_v", "layer")),
                        t(np.array([0, int(off[1]) - 6]), torch.int32))
    ctx.build_hit_index(ok).free()
    ctx.sync_status()
    ctx.close()


def _copy_dev(ptr, count, dtype):
    """Copies `count` elements from a raw device pointer owned by the library."""
    class _Wrap:
        __cuda_array_interface__ = {"shape": (count,), "typestr": {torch.float32: "<f4", torch.int32: "<i4"}[dtype],
                                    "data": (ptr, False), "version": 3}
    return torch.as_tensor(_Wrap(), device="cuda").clone()


# ------------------------------------------------------------------ seed estimate and fit

def _fit_inputs(det, n=1000, seed=1, **kw):
    b = generate(EventSpec(seed=seed, n_tracks=n, **kw), det)
    return b


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
def test_seed_state_parity(det, prec):
    b = _fit_inputs(det, n=1000)
    ctx = _ctx(prec)
    dh = device_hits(b)
    out = tkf.DeviceTracks.empty(b.n_tracks, det.n_layers, prec)
    sh = torch.as_tensor(np.ascontiguousarray(b.trk_hits[:, :3].T), dtype=torch.int32, device="cuda")
    ctx.seed_state(dh, sh, out)
    ctx.sync_status()
    got = host_tracks(out)
    g = O.make_geom(det)
    par, cov = O.seed_estimate(g, O.hits_of(b), b.trk_hits[:, :3])
    bad, worst = param_violations(got["par"], par)
    assert not bad.any(), worst
    assert np.allclose(got["cov"], cov, rtol=1e-6)
    assert np.all(got["nhits"] == 0) and np.all(got["chi2"] == 0)
    assert np.array_equal(got["hit_idx"][:, :3], b.trk_hits[:, :3])
    assert np.all(got["hit_idx"][:, 3:] == -1)


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
@pytest.mark.parametrize("pt_max", [10.0, 100.0])
def test_fit_parity(det, prec, pt_max):
    """Track fit of 1000 tracks (the plain-fit workload, seed 1) from the same initial states."""
    b = _fit_inputs(det, n=1000, seed=1, pt_max=pt_max)
    g = O.make_geom(det)
    hits = O.hits_of(b)
    par0, cov0 = O.seed_estimate(g, hits, b.trk_hits[:, :3])
    par0, cov0 = rounded(par0, prec), rounded(cov0, prec)
    ref = O.fit(g, hits, par0, cov0, b.trk_hits, 0, det.n_layers - 1)
    ctx = _ctx(prec)
    init = device_tracks(par0, cov0, np.zeros(b.n_tracks), np.zeros(b.n_tracks), b.trk_hits, precision=prec)
    out = tkf.DeviceTracks.empty(b.n_tracks, det.n_layers, prec)
    ctx.fit(device_hits(b), init, 0, det.n_layers - 1, out)
    ctx.sync_status()
    got = host_tracks(out)
    assert np.array_equal(got["nhits"], ref[3])
    bad, worst = param_violations(got["par"], ref[0])
    assert not bad.any(), worst
    bad, worst = chi2_violations(got["chi2"], ref[2])
    assert not bad.any(), worst
    if prec == tkf.FP64:  # same arithmetic type as the oracle: far inside the stated bound
        assert param_violations(got["par"], ref[0], rel=1e-8)[1] <= 1.0
    assert np.array_equal(got["hit_idx"], b.trk_hits)


def test_fit_pipeline_seed_then_fit_with_holes(det):
    """Seed estimate + fit on the GPU end to end, with some layers' hits removed (holes)."""
    b = _fit_inputs(det, n=777, seed=3)
    ids = b.trk_hits.copy()
    rng = np.random.default_rng(0)
    holes = rng.random(ids.shape) < 0.1
    holes[:, :3] = False
    ids[holes] = -1
    g = O.make_geom(det)
    hits = O.hits_of(b)
    par0, cov0 = O.seed_estimate(g, hits, ids[:, :3])
    ref = O.fit(g, hits, par0, cov0, ids, 0, det.n_layers - 1)
    ctx = _ctx()
    dh = device_hits(b)
    st = tkf.DeviceTracks.empty(b.n_tracks, det.n_layers)
    ctx.seed_state(dh, torch.as_tensor(np.ascontiguousarray(ids[:, :3].T), dtype=torch.int32, device="cuda"), st)
    hid = torch.as_tensor(np.ascontiguousarray(ids.T), dtype=torch.int32, device="cuda")
    out = tkf.DeviceTracks.empty(b.n_tracks, det.n_layers)
    ctx.fit(dh, st, 0, det.n_layers - 1, out, hit_idx=hid)
    ctx.sync_status()
    got = host_tracks(out)
    assert np.array_equal(got["nhits"], ref[3])
    assert not param_violations(got["par"], ref[0])[0].any()
    assert not chi2_violations(got["chi2"], ref[2])[0].any()


# ------------------------------------------------------------------ building

def _seeds_for(batch, det, prec, n_cand=6):
    """Oracle FP64 seed states (first three layers), rounded to the GPU's type, per event."""
    g = O.make_geom(det, O.Settings(n_cand=n_cand))
    L = det.n_layers
    out = []
    for e in range(batch.n_events):
        h0, h1 = batch.hit_off[e], batch.hit_off[e + 1]
        t0, t1 = batch.trk_off[e], batch.trk_off[e + 1]
        hits = O.hits_of(batch, slice(h0, h1))
        local = batch.trk_hits[t0:t1] - h0
        sp, sP, sc2, snh, sh = oracle_seeds(g, hits, local)
        out.append((hits, local, rounded(sp, prec), rounded(sP, prec), rounded(sc2, prec), snh, sh))
    return g, out


def _run_build(det, batch, prec, n_cand=6, seeds_per_block=0, want_all=False, **cfg):
    g, per_ev = _seeds_for(batch, det, prec, n_cand)
    L = det.n_layers
    par = np.concatenate([s[2] for s in per_ev])
    cov = np.concatenate([s[3] for s in per_ev])
    c2 = np.concatenate([s[4] for s in per_ev])
    nh = np.concatenate([s[5] for s in per_ev])
    hid = np.concatenate([np.where(s[6] >= 0, s[6] + batch.hit_off[e], -1) for e, s in enumerate(per_ev)])
    ev = np.repeat(np.arange(batch.n_events), np.diff(batch.trk_off))
    ctx = _ctx(prec, n_cand=n_cand, seeds_per_block=seeds_per_block, **cfg)
    dh = device_hits(batch)
    idx = ctx.build_hit_index(dh)
    seeds = device_tracks(par, cov, c2, nh, hid, event=ev, precision=prec)
    n = len(par)
    out = tkf.DeviceTracks.empty(n, L, prec)
    out_all = tkf.DeviceTracks.empty(n * n_cand, L, prec) if want_all else None
    ncand = torch.zeros(n, dtype=torch.int32, device="cuda") if want_all else None
    ctx.build_tracks(idx, seeds, out, out_all=out_all, n_cand_out=ncand)
    ctx.sync_status()
    got = host_tracks(out)
    got_all = host_tracks(out_all) if want_all else None
    ncand = ncand.cpu().numpy() if want_all else None
    # oracle on exactly the same (rounded) seeds
    refs = []
    for e, s in enumerate(per_ev):
        hits, local, sp, sP, sc2, snh, sh = s
        idx_o = O.hit_index(g, hits)
        refs.append(O.build(g, idx_o, sp, sP, sc2, snh, sh))
    return got, got_all, ncand, refs


def _check_build(batch, got, refs, n_layers, max_divergent=0.05, rel=None):
    n_div = 0
    n_all = 0
    for e, ref in enumerate(refs):
        t0, t1 = batch.trk_off[e], batch.trk_off[e + 1]
        h0 = batch.hit_off[e]
        gh = got["hit_idx"][t0:t1]
        gh = np.where(gh >= 0, gh - h0, -1)
        rh = ref.hits[:, 0, :]
        same = np.all(gh == rh, axis=1) & (ref.n_cand > 0)
        for s in np.nonzero(~same)[0]:
            if ref.n_cand[s] == 0:
                assert got["nhits"][t0 + s] == tkf.TRACK_LOST
                continue
            assert divergence_allowed(gh[s], ref, s), ("hit assignment differs before any fragile decision", e, s,
                                                       ref.fragile[s], gh[s], rh[s])
            n_div += 1
        n_all += t1 - t0
        m = np.nonzero(same)[0]
        bad, worst = param_violations(got["par"][t0 + m], ref.par[m, 0])
        assert not bad.any(), worst
        bad, worst = chi2_violations(got["chi2"][t0 + m], ref.chi2[m, 0])
        assert not bad.any(), worst
        assert np.array_equal(got["nhits"][t0 + m], ref.nhits[m, 0])
        if rel is not None:
            assert param_violations(got["par"][t0 + m], ref.par[m, 0], rel=rel)[1] <= 1.0
    assert n_div <= max_divergent * n_all, (n_div, n_all)
    return n_div / max(n_all, 1)


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
def test_build_parity_plain_workload(det, prec):
    """Two events of the plain building workload (5000 tracks, 20% noise hits, N = 6)."""
    b = generate(EventSpec(seed=1, n_events=2, n_tracks=5000, noise_frac=0.2), det)
    got, _, _, refs = _run_build(det, b, prec)
    frac = _check_build(b, got, refs, det.n_layers, rel=1e-8 if prec == tkf.FP64 else None)
    print("tie-divergent fraction", PNAME[prec], frac)


@pytest.mark.parametrize("n_cand", [1, 4, 10, 16])
def test_build_parity_every_candidate(det, n_cand):
    """All final candidates of every seed, for several candidate counts, on a ragged batch
    (seed count not a multiple of the tile) with an empty event."""
    b = generate(EventSpec(seed=43, n_events=3, n_tracks=[701, 0, 333], noise_frac=0.35), det)
    got, got_all, ncand, refs = _run_build(det, b, tkf.FP32, n_cand=n_cand, seeds_per_block=32, want_all=True)
    _check_build(b, got, refs, det.n_layers)
    for e, ref in enumerate(refs):
        t0, t1 = b.trk_off[e], b.trk_off[e + 1]
        h0 = b.hit_off[e]
        for s in range(t1 - t0):
            if ref.fragile[s] < det.n_layers:
                continue
            assert ncand[t0 + s] == ref.n_cand[s]
            for r in range(ref.n_cand[s]):
                o = (t0 + s) * n_cand + r
                gh = got_all["hit_idx"][o]
                assert np.array_equal(np.where(gh >= 0, gh - h0, -1), ref.hits[s, r]), (e, s, r)
                assert got_all["nhits"][o] == ref.nhits[s, r]
                assert abs(got_all["chi2"][o] - ref.chi2[s, r]) <= 1e-3 * max(ref.chi2[s, r], 1.0)


def test_build_multi_event_isolation(det):
    """Events packed in one launch only see their own hits: a lognormal-sized batch matches
    the oracle event by event, and a batch holding one of its events twice gives that event's
    result twice, bit for bit."""
    sizes, noise = event_sizes(7, 6, median=400, lo=50, hi=2000)
    b = generate(EventSpec(seed=44, n_events=6, n_tracks=sizes, noise_frac=noise), det)
    got, _, _, refs = _run_build(det, b, tkf.FP32)
    _check_build(b, got, refs, det.n_layers)
    twice = select_events(b, [2, 2])
    got2, _, _, _ = _run_build(det, twice, tkf.FP32)
    t0, t1 = b.trk_off[2], b.trk_off[3]
    n = t1 - t0
    for c in range(2):
        sl = slice(c * n, (c + 1) * n)
        gh = got2["hit_idx"][sl]
        assert np.array_equal(np.where(gh >= 0, gh - twice.hit_off[c], -1),
                              np.where(got["hit_idx"][t0:t1] >= 0, got["hit_idx"][t0:t1] - b.hit_off[2], -1))
        assert np.array_equal(got2["par"][sl], got["par"][t0:t1])
        assert np.array_equal(got2["chi2"][sl], got["chi2"][t0:t1])


def test_build_no_seeds_and_empty_layers(det):
    ctx = _ctx()
    b = generate(EventSpec(seed=45, n_events=1, n_tracks=50, noise_frac=0.0), det)
    # drop every hit of layer 6: candidates must take holes there
    keep = b.layer != 6
    for k in ("x", "y", "z", "var_u", "var_v", "layer", "mc"):
        setattr(b, k, getattr(b, k)[keep])
    remap = np.cumsum(keep) - 1
    b.trk_hits = np.where(b.trk_hits >= 0, remap[np.maximum(b.trk_hits, 0)], -1)
    b.trk_hits[:, 6] = -1
    b.hit_off = np.array([0, keep.sum()])
    got, _, _, refs = _run_build(det, b, tkf.FP32)
    _check_build(b, got, refs, det.n_layers)
    assert np.all(got["hit_idx"][:, 6] == -1)
    # zero seeds: nothing to do, no error
    idx = ctx.build_hit_index(device_hits(b))
    empty = tkf.DeviceTracks.empty(0, det.n_layers)
    empty.n = 0
    ctx.build_tracks(idx, empty, empty)
    ctx.sync_status()


# ------------------------------------------------------------------ hits off the cylinders (Sec. 2.2)

# modules 0.5 cm inside and outside each layer's average radius (the simplified CMS geometry):
# hit_dr = 0.5 cm, states taken to each hit's radius, building in two steps
MODULES = Detector(module_dr=1.0)


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
def test_two_step_fit_parity(prec):
    """Fit of 1000 tracks (|eta| < 2) on the module geometry from the same initial states; with
    hit_dr = 0 the same hits do not fit (the setting reaches the kernel)."""
    b = generate(EventSpec(seed=71, n_tracks=1000, eta_max=2.0), MODULES)
    g = O.make_geom(MODULES)
    hits = O.hits_of(b)
    par0, cov0 = O.seed_estimate(g, hits, b.trk_hits[:, :3])
    par0, cov0 = rounded(par0, prec), rounded(cov0, prec)
    ref = O.fit(g, hits, par0, cov0, b.trk_hits, 0, MODULES.n_layers - 1)
    assert np.all(ref[4] == 0)
    L = MODULES.n_layers
    init = device_tracks(par0, cov0, np.zeros(b.n_tracks), np.zeros(b.n_tracks), b.trk_hits, precision=prec)
    got = {}
    for dr in (0.5, 0.0):
        ctx = _ctx(prec, hit_dr=dr)
        out = tkf.DeviceTracks.empty(b.n_tracks, L, prec)
        ctx.fit(device_hits(b), init, 0, L - 1, out)
        ctx.sync_status()
        got[dr] = host_tracks(out)
        ctx.close()
    r = got[0.5]
    assert np.array_equal(r["nhits"], ref[3])
    bad, worst = param_violations(r["par"], ref[0])
    assert not bad.any(), worst
    bad, worst = chi2_violations(r["chi2"], ref[2])
    assert not bad.any(), worst
    if prec == tkf.FP64:
        assert param_violations(r["par"], ref[0], rel=1e-8)[1] <= 1.0
    assert np.median(got[0.0]["chi2"]) > 5.0 * np.median(r["chi2"])


@pytest.mark.parametrize("prec", PRECS, ids=lambda p: PNAME[p])
def test_two_step_build_parity(prec):
    """Two events (2000 and 3000 tracks, 30 % noise hits, |eta| < 2, N = 6) on the module
    geometry: window on the average radius, every candidate hit scored after its own step."""
    b = generate(EventSpec(seed=72, n_events=2, n_tracks=[2000, 3000], noise_frac=0.3, eta_max=2.0), MODULES)
    got, _, _, refs = _run_build(MODULES, b, prec, hit_dr=0.5)
    _check_build(b, got, refs, MODULES.n_layers, max_divergent=0.01, rel=1e-8 if prec == tkf.FP64 else None)
    own = np.all(got["hit_idx"] == b.trk_hits, axis=1).mean()
    assert own >= 0.97, own


@pytest.mark.parametrize("n_cand", [1, 16])
def test_two_step_build_parity_candidate_counts(n_cand):
    b = generate(EventSpec(seed=73, n_tracks=1500, noise_frac=0.3, eta_max=1.5), MODULES)
    got, _, _, refs = _run_build(MODULES, b, tkf.FP32, n_cand=n_cand, hit_dr=0.5)
    _check_build(b, got, refs, MODULES.n_layers, max_divergent=0.01)


def test_two_step_settings_are_validated():
    for dr in (-0.1, float("nan"), 2.0, 4.0):  # negative, NaN, half the 4 cm gap, the first radius
        with pytest.raises(tkf.TkfError):
            _ctx(hit_dr=dr)
    _ctx(hit_dr=1.99).close()
