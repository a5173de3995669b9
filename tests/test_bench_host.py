"""Host-side logic of bench.py (no GPU): the building-efficiency measure and the seeding leg's
tracking measure, the layout of events lent to the server, the balanced dealing of oracle events
to host cores, and the sample selection."""
import ctypes as C

import numpy as np
import pytest

import bench
from synth import Detector, EventSpec, generate


@pytest.fixture(scope="module")
def small_batch():
    return generate(EventSpec(seed=5, n_events=3, n_tracks=[40, 0, 25], noise_frac=0.3), Detector())


def test_efficiency_counts_tracks_with_three_quarters_own_hits(small_batch):
    b = small_batch
    truth = b.trk_hits.T.copy()  # [L, n]: every track its own simulated hits
    assert bench.efficiency(b, truth) == 1.0
    noise = np.nonzero(b.mc < 0)[0]
    bad = truth.copy()
    bad[3:6, 0] = noise[:3]  # 3 of 10 hits of track 0 from noise: 70 % own
    bad[3:5, 1] = noise[3:5]  # 2 of 10 for track 1: 80 % own
    bad[:, 2] = -1
    bad[:3, 2] = truth[:3, 2]  # only the seed hits: 100 % own
    eff = bench.efficiency(b, bad)
    assert eff == pytest.approx((b.n_tracks - 1) / b.n_tracks)


def test_lent_events_point_into_the_batch_planes(small_batch):
    torch = pytest.importorskip("torch")
    from paper_1702_06359_gb300 import tkf
    b = small_batch
    host = {k: torch.as_tensor(np.ascontiguousarray(getattr(b, k)), dtype=torch.int32 if k == "layer" else torch.float32)
            for k in ("x", "y", "z", "var_u", "var_v", "layer")}
    lent = bench.LentEvents(tkf, b, host, 10)
    assert len(lent.events) == b.n_events and len(lent.array) == b.n_events
    for e, ev in enumerate(lent.events):
        h0, h1, t0, t1 = b.hit_off[e], b.hit_off[e + 1], b.trk_off[e], b.trk_off[e + 1]
        assert ev.n_hits == h1 - h0 and ev.n_seeds == t1 - t0 and ev.borrow == 1
        if ev.n_hits:
            z = np.ctypeslib.as_array(C.cast(ev.z, C.POINTER(C.c_float)), shape=(ev.n_hits,))
            assert np.array_equal(z, b.z[h0:h1])
        if ev.n_seeds:
            sd = np.ctypeslib.as_array(C.cast(ev.seed_hits, C.POINTER(C.c_int32)), shape=(3 * ev.n_seeds,))
            assert np.array_equal(sd.reshape(3, -1), (b.trk_hits[t0:t1, :3] - h0).T)
    assert lent.h2d == b.n_hits * 24 + b.n_tracks * 12 + b.n_events * 8


def test_oracle_events_are_dealt_largest_first_to_the_least_loaded_core():
    class _Pool:
        def map(self, fn, chunks, chunksize=1):
            self.chunks = chunks
            return [(sum(len(ev[1]) for ev in c), 0.001 * sum(len(ev[1]) for ev in c)) for c in chunks]
    sizes = [50, 10, 40, 30, 20, 5]
    sample = [(None, np.zeros((n, 10))) for n in sizes]
    pool = _Pool()
    done, comp, wall = bench.cpu_baseline(sample, pool, 2)
    assert done == sum(sizes) and wall >= 0 and abs(comp - 0.080) < 1e-12  # the slowest worker's computing
    loads = sorted(sum(len(ev[1]) for ev in c) for c in pool.chunks)
    assert loads == [75, 80]  # 50+20+5 and 40+30+10


def test_sample_events_cover_the_requested_tracks():
    ev, n = bench.sample_events(3, 20000)
    from synth import event_sizes
    sizes, _ = event_sizes(3, 640)
    assert ev == list(range(len(ev))) and n == int(sizes[:len(ev)].sum()) >= 20000
    assert int(sizes[:len(ev) - 1].sum()) < 20000


def test_backward_baseline_helpers():
    """The bench's covariance unpacking matches the test helpers' packing, and its oracle
    backward-pass worker runs the oracle's pass on every track it is given."""
    import oracle as O
    from _gpu import pack_cov
    from synth import Detector, EventSpec, generate
    rng = np.random.default_rng(5)
    a = rng.normal(size=(7, 6, 6))
    cov = a @ np.transpose(a, (0, 2, 1))
    assert np.array_equal(bench._unpack_cov(pack_cov(cov)), cov)
    det = Detector()
    b = generate(EventSpec(seed=9, n_tracks=40), det)
    g = O.make_geom(det)
    hits = O.hits_of(b)
    p0, c0 = O.seed_estimate(g, hits, b.trk_hits[:, :3])
    pf, cf, _, _, st = O.fit(g, hits, p0, c0, b.trk_hits, 0, det.n_layers - 1)
    assert np.all(st == 0)
    done, secs = bench._oracle_backward([(hits, b.trk_hits, pf, cf), (hits, b.trk_hits[:5], pf[:5], cf[:5])])
    assert done == 45 and secs > 0


def test_physics_of_a_perfect_reconstruction_and_of_planted_errors(small_batch):
    """Own hits and true states on the last layer: every track has ten own hits, the pT
    resolution is zero and no charge is wrong; a track given a hole and another with its charge
    flipped and pT 10 % high move exactly those figures."""
    b = small_batch
    L = b.detector.n_layers
    hid = b.trk_hits.T.copy()
    par = b.truth[:, -1].T.copy()  # [6, n]
    nh = np.full(b.n_tracks, L)
    ph = bench.physics(b, hid, par, nh)
    assert ph["own_ten_hits"] == 1.0 and ph["charge_misid"] == 0.0
    assert ph["fraction_by_nhits"][L] == 1.0
    assert ph["pt_resolution"]["rms"] == pytest.approx(0.0, abs=1e-12)
    hid[5, 0] = -1
    nh[0] = L - 1
    par[3, 1] = -par[3, 1] / 1.1  # flipped charge, pT 10 % high
    ph = bench.physics(b, hid, par, nh)
    n = b.n_tracks
    assert ph["own_ten_hits"] == pytest.approx((n - 1) / n)
    assert ph["fraction_by_nhits"][L - 1] == pytest.approx(1 / n)
    assert ph["charge_misid"] == pytest.approx(1 / (n - 1))
    assert ph["pt_resolution"]["rms"] == pytest.approx(0.1 / np.sqrt(n - 1), rel=1e-9)


def test_issue_roofline_arithmetic():
    r = bench.issue_roofline(2867.0, 1_000_000, 4.0)
    assert r["achieved"] == pytest.approx(2867.0 * 1e6 / 4e-3)
    assert r["peak"] == pytest.approx(152 * 4 * 2.07e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.issue_roofline(None, 1, 1.0) is None


def test_seeded_efficiency_counts_found_fake_and_duplicate(small_batch):
    """The seeding leg's tracking measure: with one seed per track on its own hits every track is
    found; a second seed of a track is a duplicate; a seed that starts on a noise hit, or whose
    built track has fewer than 75 % of one track's hits, is a fake."""
    b = small_batch
    truth = b.trk_hits.T.copy()  # [L, n]
    first = truth[0].copy()
    r = bench.seeded_efficiency(b, first, truth)
    assert r == {"track_efficiency": 1.0, "fake_rate": 0.0, "duplicate_rate": 0.0}
    # track 0 seeded twice, track 1's built track mostly noise, one seed on a noise hit
    noise = np.nonzero(b.mc < 0)[0]
    hits = np.concatenate([truth, truth[:, :1], truth[:, :1]], axis=1)
    firsts = np.concatenate([first, first[:1], [noise[0]]])
    hits[:, -1] = -1
    hits[0, -1] = noise[0]
    hits[3:6, 1] = noise[1:4]  # 7 of 10 own: below 75 %
    r = bench.seeded_efficiency(b, firsts, hits)
    n = b.n_tracks
    assert r["track_efficiency"] == pytest.approx((n - 1) / n)
    assert r["fake_rate"] == pytest.approx(2 / (n + 2))
    assert r["duplicate_rate"] == pytest.approx(1 / (n - 1))
