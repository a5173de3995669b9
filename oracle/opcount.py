"""ORACLE -- test infrastructure.  Counts the algorithmic work of combinatorial building per
seed on a seeded sample of a workload by instrumenting the oracle: candidates propagated,
hits scored, Kalman updates and kept branches (each kept branch gets the scattering noise).

    python oracle/opcount.py [--events K] [--workload batched|plain] [--module-dr D] [--forward]

--module-dr D places each layer's modules D/2 inside and outside its radius (hits off the
cylinders, the two-step building); n_steps then counts the hits taken to their own radius.
--forward takes the same events, each with a quarter of its tracks, on the endcap tracker (ten
pairs of disks, 1.7 <= |eta| <= 2.5).

The per-seed counts it prints, times the per-operation FP32 operation counts of the build
kernel's arithmetic, give the algorithmic FLOP per built track used for the roofline.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from synth import FORWARD_ETA, FORWARD_PRIOR, Detector, EventSpec, event_sizes, forward_detector, generate  # noqa: E402


def count(batch, det, settings=O.Settings()):
    g = O.make_geom(det, settings)
    tot = dict(n_prop=0, n_hits_examined=0, n_updates=0, n_kept=0, n_steps=0, seeds=0)
    L = det.n_layers
    for e in range(batch.n_events):
        h0, h1 = batch.hit_off[e], batch.hit_off[e + 1]
        t0, t1 = batch.trk_off[e], batch.trk_off[e + 1]
        if t1 == t0:
            continue
        hits = O.hits_of(batch, slice(h0, h1))
        local = batch.trk_hits[t0:t1] - h0
        p0, c0 = O.seed_estimate(g, hits, local[:, :3])
        ids = np.full((t1 - t0, L), -1, dtype=np.int32)
        ids[:, :3] = local[:, :3]
        sp, sP, sc2, snh, _ = O.fit(g, hits, p0, c0, ids, 0, 2)
        res = O.build(g, O.hit_index(g, hits), sp, sP, sc2, snh, ids)
        for k in ("n_prop", "n_hits_examined", "n_updates", "n_kept", "n_steps"):
            tot[k] += res.stats[k]
        tot["seeds"] += t1 - t0
    return {k: v / tot["seeds"] for k, v in tot.items() if k != "seeds"} | {"seeds": tot["seeds"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--events", type=int, default=16)
    ap.add_argument("--workload", choices=["batched", "plain"], default="batched")
    ap.add_argument("--module-dr", type=float, default=0.0)
    ap.add_argument("--forward", action="store_true")
    a = ap.parse_args()
    det = forward_detector() if a.forward else Detector(module_dr=a.module_dr)
    eta = dict(eta_min=FORWARD_ETA[0], eta_max=FORWARD_ETA[1]) if a.forward else {}
    st = O.Settings(eta_min=-3.0, n_eta_bins=60, prior_sigma=FORWARD_PRIOR) if a.forward else O.Settings()
    if a.workload == "batched":
        n, f = event_sizes(3, 640)
        if a.forward:  # the endcaps' share of each event: a quarter of its tracks
            n = np.maximum(1, np.rint(0.25 * n)).astype(np.int64)
        spec = EventSpec(seed=3, n_events=a.events, n_tracks=n[:a.events], noise_frac=f[:a.events], **eta)
    else:
        spec = EventSpec(seed=1, n_events=a.events, n_tracks=5000, noise_frac=0.2, **eta)
    c = count(generate(spec, det), det, st)
    print(" ".join("%s=%.4f" % kv for kv in c.items()))


if __name__ == "__main__":
    main()
