"""Seeded input generator: Philox known answers, determinism, and the event recipe."""
import os

import numpy as np

from synth import EventSpec, event_sizes, generate, philox4x32_10

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        out = philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_generator_is_deterministic_and_addressable(det):
    a = generate(EventSpec(seed=5, n_events=3, n_tracks=50, noise_frac=0.2), det)
    b = generate(EventSpec(seed=5, n_events=3, n_tracks=50, noise_frac=0.2), det)
    for k in ("x", "y", "z", "layer", "mc"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    # event 1 alone equals event 1 inside the batch (counter-based draws)
    c = generate(EventSpec(seed=5, n_events=3, n_tracks=[0, 50, 0], noise_frac=0.2), det)
    assert np.allclose(c.truth, a.truth[50:100])


def test_hits_lie_on_cylinders_and_truth_is_consistent(det):
    b = generate(EventSpec(seed=7, n_events=2, n_tracks=200, noise_frac=0.25), det)
    r = np.hypot(b.x.astype(np.float64), b.y.astype(np.float64))
    R = np.asarray(det.radii)[b.layer]
    assert np.all(np.abs(r - R) < 1e-5)
    for e in range(2):
        h0, h1 = b.hit_off[e], b.hit_off[e + 1]
        assert np.all(np.diff(b.layer[h0:h1]) >= 0)
        for l in range(det.n_layers):
            n_l = np.sum(b.layer[h0:h1] == l)
            assert n_l == 200 + round(0.25 * 200)
    assert np.all(b.mc[b.trk_hits] == np.arange(b.n_tracks)[:, None])
    tr = b.truth
    assert np.allclose(np.hypot(tr[..., 0], tr[..., 1]), np.asarray(det.radii)[None, :], atol=1e-9)


def test_event_sizes_recipe():
    n, f = event_sizes(11, 4000)
    assert n.min() >= 200 and n.max() <= 20000
    assert abs(np.median(n) - 3000) < 150
    assert np.all((f >= 0.2) & (f <= 0.5))
    inner = n[(n > 200) & (n < 20000)]
    assert abs(np.std(np.log(inner)) - 0.8) < 0.05


def test_events_generated_in_chunks_equal_one_batch(det):
    from synth import concat
    n = [30, 0, 45, 12, 60]
    whole = generate(EventSpec(seed=8, n_events=5, n_tracks=n, noise_frac=0.3), det)
    parts = [generate(EventSpec(seed=8, n_events=2, n_tracks=n[0:2], noise_frac=0.3), det),
             generate(EventSpec(seed=8, n_events=3, n_tracks=n[2:5], noise_frac=0.3, first_event=2), det)]
    c = concat(parts)
    for k in ("hit_off", "trk_off", "x", "y", "z", "layer", "mc", "trk_event", "trk_hits"):
        assert np.array_equal(getattr(c, k), getattr(whole, k)), k
    assert np.array_equal(c.truth, whole.truth)
