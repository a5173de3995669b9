"""Shared test helpers: event preparation for the oracle and the CUDA path."""
import math

import numpy as np

import oracle as O
from synth import Detector, EventSpec, generate


def oracle_seeds(g, hits_ev, trk_hits_local, n_seed_layers=3):
    """Seed states after the first three layers (initial estimate + Kalman fit), FP64."""
    L = g.n_layers
    n = len(trk_hits_local)
    par0, cov0 = O.seed_estimate(g, hits_ev, trk_hits_local[:, :3])
    ids = np.full((n, L), -1, dtype=np.int32)
    ids[:, :n_seed_layers] = trk_hits_local[:, :n_seed_layers]
    po, co, c2, nh, st = O.fit(g, hits_ev, par0, cov0, ids, 0, n_seed_layers - 1)
    assert np.all(st == 0)
    return po, co, c2, nh, ids


def rotate_into_jet(batch, width=0.05, seed=0):
    """Rotate every track (its hits and truth) about z so that all tracks point into a narrow
    azimuthal window around phi = 0; noise hits are rotated into the same window.  Rotations
    about the field axis leave the physics unchanged, so this only raises hit density."""
    rng = np.random.default_rng(seed)
    b = batch
    x = b.x.astype(np.float64)
    y = b.y.astype(np.float64)
    for t in range(b.n_tracks):
        a = -b.vertex_state[t, 4] + rng.uniform(-width, width)
        ids = b.trk_hits[t]
        c, s = math.cos(a), math.sin(a)
        x[ids], y[ids] = c * x[ids] - s * y[ids], s * x[ids] + c * y[ids]
    noise = b.mc < 0
    ph = np.arctan2(y[noise], x[noise])
    a = -ph + rng.uniform(-2 * width, 2 * width, size=noise.sum())
    r = np.hypot(x[noise], y[noise])
    x[noise], y[noise] = r * np.cos(ph + a), r * np.sin(ph + a)
    b.x, b.y = x.astype(np.float32), y.astype(np.float32)
    return b


def small_event(det, seed, n_tracks, noise_frac, **kw):
    return generate(EventSpec(seed=seed, n_events=1, n_tracks=n_tracks, noise_frac=noise_frac, **kw), det)


def select_events(batch, events):
    """A new batch made of the listed events of `batch` (repeats allowed), re-indexed."""
    import copy
    hs, ts = [], []
    hit_off, trk_off = [0], [0]
    for e in events:
        h0, h1 = batch.hit_off[e], batch.hit_off[e + 1]
        t0, t1 = batch.trk_off[e], batch.trk_off[e + 1]
        hs.append((h0, h1, hit_off[-1]))
        ts.append((t0, t1, trk_off[-1], hit_off[-1] - h0))
        hit_off.append(hit_off[-1] + h1 - h0)
        trk_off.append(trk_off[-1] + t1 - t0)
    out = copy.copy(batch)
    cat = lambda a: np.concatenate([a[h0:h1] for h0, h1, _ in hs])
    for k in ("x", "y", "z", "var_u", "var_v", "layer"):
        setattr(out, k, cat(getattr(batch, k)))
    out.mc = np.concatenate([np.where(batch.mc[h0:h1] >= 0, batch.mc[h0:h1] - batch.trk_off[e] + trk_off[i], -1)
                             for i, ((h0, h1, _), e) in enumerate(zip(hs, events))])
    out.trk_hits = np.concatenate([np.where(batch.trk_hits[t0:t1] >= 0, batch.trk_hits[t0:t1] + shift, -1)
                                   for t0, t1, _, shift in ts])
    out.truth = np.concatenate([batch.truth[t0:t1] for t0, t1, _, _ in ts])
    out.trk_event = np.repeat(np.arange(len(events)), [t1 - t0 for t0, t1, _, _ in ts])
    out.hit_off = np.asarray(hit_off, dtype=np.int64)
    out.trk_off = np.asarray(trk_off, dtype=np.int64)
    return out
