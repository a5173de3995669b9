"""Parity of tkf_find_seeds (seeding from hit triplets on layers 0-2, confirmed on layer 3) with
the oracle's brute-force definition: the same pick (layer-1 and layer-2 hit) for every layer-0
hit and the same score, except where the oracle shows a decision within 1e-4 of a cut or a tie
(the kernel evaluates the cut quantities in FP32, the oracle in FP64); on small events element
by element, on the 640-event seeding workload for a seeded sample of first hits plus properties
of every seed."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
from _gpu import device_hits
from synth import Detector, EventSpec, generate

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1702_06359_gb300 import tkf  # noqa: E402

PIX = Detector(pixel_layers=4)
FRAGILE = 1e-4      # oracle margin / score gap below which FP32 may decide otherwise
SCORE_ABS = 2e-4    # |score difference| allowed for the same pick


def _cuts(oracle_side=False, **kw):
    c = tkf.default_seed_cuts(**kw)
    if oracle_side:
        return O.SeedCuts(c.pt_min, c.kappa_slack, c.z_vertex, c.d0_max, c.dz_max, c.conf_rphi, c.conf_z, c.confirm)
    return c


def _copy_dev(ptr, count, dtype):
    """Copies `count` elements from a raw device pointer owned by the library."""
    class _Wrap:
        __cuda_array_interface__ = {"shape": (count,), "typestr": {torch.float32: "<f4", torch.int32: "<i4"}[dtype],
                                    "data": (ptr, False), "version": 3}
    return torch.as_tensor(_Wrap(), device="cuda").clone()


def _gpu_seeds(b, cuts, max_seeds=None, ctx=None):
    ctx = ctx or tkf.Context()
    idx = ctx.build_hit_index(device_hits(b))
    cap = b.n_hits if max_seeds is None else max_seeds
    dev = torch.device("cuda", 0)
    sh = torch.full((3, max(cap, 1)), -7, dtype=torch.int32, device=dev)
    se = torch.full((max(cap, 1),), -7, dtype=torch.int32, device=dev)
    ss = torch.zeros(max(cap, 1), dtype=torch.float32, device=dev)
    nf = torch.zeros(1, dtype=torch.int32, device=dev)
    ctx.find_seeds(idx, cuts, cap, sh, se, nf, ss)
    ctx.sync_status()
    n = int(nf.item())
    k = min(n, cap)
    pos = _copy_dev(idx.view().pos_of_hit, b.n_hits, torch.int32).cpu().numpy()
    return dict(n=n, hits=sh[:, :k].cpu().numpy(), event=se[:k].cpu().numpy(), score=ss[:k].cpu().numpy(),
                pos_of_hit=pos, raw=(sh, se, ss))


def _oracle_picks(b, cuts_o, events=None):
    """Per event: the oracle's SEED_PICK records of its hits (event-local)."""
    g = O.make_geom(b.detector)
    out = {}
    for e in (range(b.n_events) if events is None else events):
        sl = slice(int(b.hit_off[e]), int(b.hit_off[e + 1]))
        out[e] = O.find_seeds(g, cuts_o, O.hits_of(b, sl))
    return out


def _compare(b, gpu, picks, min_seeds=1):
    """Element-by-element comparison per layer-0 hit; returns (matches, excused)."""
    by_a = {int(a): (int(h1), int(h2), float(s), int(e)) for a, h1, h2, s, e in
            zip(gpu["hits"][0], gpu["hits"][1], gpu["hits"][2], gpu["score"], gpu["event"])}
    assert len(by_a) == gpu["hits"].shape[1], "a first hit starts at most one seed"
    match = excused = 0
    for e, pk in picks.items():
        base = int(b.hit_off[e])
        l0 = np.nonzero(pk["h1"] >= -1)[0]
        l0 = l0[b.layer[base + l0] == 0]
        for a in l0:
            p = pk[a]
            got = by_a.get(base + int(a))
            fragile = p["margin"] < FRAGILE or p["gap"] < FRAGILE
            if p["h1"] < 0:
                ok = got is None
            else:
                ok = got is not None and got[0] == base + p["h1"] and got[1] == base + p["h2"] and got[3] == e and \
                    abs(got[2] - p["score"]) <= SCORE_ABS
            if ok:
                match += 1
            else:
                assert fragile, (e, int(a), p, got)
                excused += 1
    assert match >= min_seeds
    return match, excused


def _check_order(b, gpu):
    ev = gpu["event"]
    assert np.all(np.diff(ev) >= 0)
    pos = gpu["pos_of_hit"][gpu["hits"][0]]
    same = np.diff(ev) == 0
    assert np.all(np.diff(pos)[same] > 0), "seeds follow the index order of their first hits"
    assert np.all(b.layer[gpu["hits"][0]] == 0) and np.all(b.layer[gpu["hits"][1]] == 1)
    assert np.all(b.layer[gpu["hits"][2]] == 2)
    assert np.all((gpu["hits"] >= b.hit_off[ev]) & (gpu["hits"] < b.hit_off[ev + 1]))


@pytest.mark.parametrize("confirm", [1, 0])
def test_seeds_match_oracle_small_events(confirm):
    """Events of 40 to 1200 tracks with 0-50 % noise (several thread blocks, ragged tails, an
    event with no noise), every first hit compared."""
    b = generate(EventSpec(seed=81, n_events=5, n_tracks=np.array([300, 1200, 40, 700, 150]),
                           noise_frac=np.array([0.3, 0.5, 0.0, 0.2, 0.4])), PIX)
    gpu = _gpu_seeds(b, _cuts(confirm=confirm))
    assert gpu["n"] == gpu["hits"].shape[1]
    picks = _oracle_picks(b, _cuts(True, confirm=confirm))
    match, excused = _compare(b, gpu, picks, min_seeds=2000)
    assert excused <= 0.005 * (match + excused)
    _check_order(b, gpu)
    n_oracle = sum(int((pk["h1"] >= 0).sum()) for pk in picks.values())
    assert abs(gpu["n"] - n_oracle) <= excused


def test_seeds_on_the_plain_detector_and_after_index_reuse():
    """The plain barrel (1 mm in z: many more candidates per hit) and a second index over other
    hits in the same context: scratch reuse, other sizes."""
    ctx = tkf.Context()
    b = generate(EventSpec(seed=82, n_events=2, n_tracks=np.array([400, 90]), noise_frac=0.3))
    gpu = _gpu_seeds(b, _cuts(), ctx=ctx)
    match, excused = _compare(b, gpu, _oracle_picks(b, _cuts(True)), min_seeds=300)
    assert excused <= 0.01 * (match + excused)
    b2 = generate(EventSpec(seed=83, n_events=3, n_tracks=np.array([60, 500, 20]), noise_frac=0.1), PIX)
    gpu2 = _gpu_seeds(b2, _cuts(), ctx=ctx)
    _compare(b2, gpu2, _oracle_picks(b2, _cuts(True)), min_seeds=450)
    _check_order(b2, gpu2)


def test_truncation_single_track_events_and_errors():
    b = generate(EventSpec(seed=84, n_events=4, n_tracks=np.array([200, 1, 300, 1]), noise_frac=0.0), PIX)
    full = _gpu_seeds(b, _cuts())
    assert full["n"] > 400
    part = _gpu_seeds(b, _cuts(), max_seeds=100)
    assert part["n"] == full["n"] and part["hits"].shape[1] == 100
    assert np.array_equal(part["hits"], full["hits"][:, :100]) and np.array_equal(part["event"], full["event"][:100])
    assert np.array_equal(part["score"], full["score"][:100])
    # max_seeds = 0 only counts
    zero = _gpu_seeds(b, _cuts(), max_seeds=0)
    assert zero["n"] == full["n"]
    ctx = tkf.Context()
    idx = ctx.build_hit_index(device_hits(b))
    dev = torch.device("cuda", 0)
    buf = torch.zeros((3, 8), dtype=torch.int32, device=dev)
    ev = torch.zeros(8, dtype=torch.int32, device=dev)
    nf = torch.zeros(1, dtype=torch.int32, device=dev)
    for bad in (dict(d0_max=0.0), dict(pt_min=-1.0), dict(conf_z=0.0)):
        with pytest.raises(tkf.TkfError):
            ctx.find_seeds(idx, _cuts(**bad), 8, buf, ev, nf)
    with pytest.raises(tkf.TkfError):
        ctx.find_seeds(idx, _cuts(), -1, buf, ev, nf)
    # an index binned by another configuration
    other = tkf.Context(tkf.default_config(n_eta_bins=20, eta_bin_w=0.2))
    with pytest.raises(tkf.TkfError):
        other.find_seeds(idx, _cuts(), 8, buf, ev, nf)


def test_empty_events_and_empty_batch():
    """An event without hits between others starts no seed and leaves the others unchanged; a
    batch without any hit finds none."""
    b = generate(EventSpec(seed=86, n_events=3, n_tracks=np.array([150, 0, 90]), noise_frac=0.2), PIX)
    assert b.hit_off[1] == b.hit_off[2]
    gpu = _gpu_seeds(b, _cuts())
    assert gpu["n"] > 200 and not np.any(gpu["event"] == 1)
    _compare(b, gpu, _oracle_picks(b, _cuts(True), events=[0, 2]), min_seeds=250)
    _check_order(b, gpu)
    empty = generate(EventSpec(seed=87, n_events=2, n_tracks=np.array([0, 0]), noise_frac=0.0), PIX)
    assert empty.n_hits == 0
    assert _gpu_seeds(empty, _cuts(), max_seeds=4)["n"] == 0


def test_seeds_feed_the_pipeline():
    """Seeds found on the device go straight into tkf_pipeline_run (the seed rows and event
    ids it takes), and the built tracks of true seeds carry their tracks' hits."""
    b = generate(EventSpec(seed=85, n_events=3, n_tracks=np.array([500, 800, 300]), noise_frac=0.3), PIX)
    gpu = _gpu_seeds(b, _cuts())
    n = gpu["n"]
    ctx = tkf.Context(tkf.default_config(seed_order=1))
    p = tkf.DevicePipeline(ctx, b.n_hits, b.n_events, n, use_graph=False)
    sh, se = gpu["raw"][0], gpu["raw"][1]
    p.run(device_hits(b), sh[:, :n].contiguous(), se[:n].contiguous(), n)
    ctx.sync_status()
    _, _, fitted = p.outputs()
    hit_idx = tkf.tracks_tensors(fitted, b.detector.n_layers)["hit_idx"][:, :n].T.cpu().numpy()
    mc = b.mc[gpu["hits"][0]]
    true = mc >= 0
    own = true & (b.mc[gpu["hits"][1]] == mc) & (b.mc[gpu["hits"][2]] == mc)
    assert own.sum() >= 0.97 * b.n_tracks
    # built hits of own seeds on the outer layers belong to the same track
    outer = hit_idx[own][:, 3:]
    ok = outer >= 0
    same = b.mc[np.where(ok, outer, 0)] == mc[own][:, None]
    assert (same | ~ok).mean() >= 0.97


def _full_batch():
    import bench
    with mp.get_context("spawn").Pool(min(os.cpu_count() or 1, 16)) as pool:
        return bench.workload(3, 640, pool, pixel_layers=4)


def test_full_seeding_workload_sampled_parity_and_properties():
    """The bench's seeding leg: the 640-event batch (2.6 M tracks, lognormal sizes up to 20 000
    tracks, 20-50 % noise) with pixel inner layers, in the launch bench.py times."""
    b = _full_batch()
    gpu = _gpu_seeds(b, _cuts())
    n = gpu["n"]
    _check_order(b, gpu)
    th = b.trk_hits
    pick = np.full(b.n_hits, -1, dtype=np.int64)
    pick2 = np.full(b.n_hits, -1, dtype=np.int64)
    pick[gpu["hits"][0]] = gpu["hits"][1]
    pick2[gpu["hits"][0]] = gpu["hits"][2]
    own = (pick[th[:, 0]] == th[:, 1]) & (pick2[th[:, 0]] == th[:, 2])
    assert own.mean() >= 0.95, own.mean()
    assert n <= 1.3 * b.n_tracks
    # sampled first hits of 32 events (the largest included) against the oracle's definition
    rng = np.random.default_rng(5)
    sizes = np.diff(b.trk_off)
    events = list(rng.choice(b.n_events, 31, replace=False)) + [int(np.argmax(sizes))]
    g = O.make_geom(PIX)
    cuts_o = _cuts(True)
    by_a = {int(a): (int(h1), int(h2), float(s)) for a, h1, h2, s in
            zip(gpu["hits"][0], gpu["hits"][1], gpu["hits"][2], gpu["score"])}
    match = excused = 0
    for e in events:
        base, end = int(b.hit_off[e]), int(b.hit_off[e + 1])
        l0 = np.nonzero(b.layer[base:end] == 0)[0]
        first = rng.choice(l0, min(12, len(l0)), replace=False).astype(np.int32)
        pk = O.find_seeds(g, cuts_o, O.hits_of(b, slice(base, end)), first=first)
        for a, p in zip(first, pk):
            got = by_a.get(base + int(a))
            if p["h1"] < 0:
                ok = got is None
            else:
                ok = got is not None and got[:2] == (base + p["h1"], base + p["h2"]) and abs(got[2] - p["score"]) <= SCORE_ABS
            if ok:
                match += 1
            else:
                assert p["margin"] < FRAGILE or p["gap"] < FRAGILE, (e, int(a), p, got)
                excused += 1
    assert match >= 370 and excused <= 4
    # every seed passes the definition's triplet cuts (sampled 20 000 seeds)
    sel = rng.choice(n, min(n, 20000), replace=False)
    hits = O.hits_of(b)
    bad = 0
    for k in sel:
        a, bb, c = (O.make_hit(*hits[gpu["hits"][r, k]][["x", "y", "z", "var_u", "var_v"]], r) for r in range(3))
        ok, q = O.seed_eval(g, cuts_o, a, bb, c)
        if not ok:
            kmax = O.seed_kappa_max(g, cuts_o)
            ratios = [abs(q.kappa01) / kmax, abs(q.zv) / cuts_o.z_vertex, q.kappa / kmax, abs(q.d0) / cuts_o.d0_max,
                      abs(q.dz) / cuts_o.dz_max]
            assert max(ratios) <= 1 + FRAGILE, ratios
            bad += 1
    assert bad <= 2
