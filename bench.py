"""Benchmark of the tracking hot path on GB300: built tracks/s.

Workload (default): the batched-building configuration -- 640 synthetic barrel events with
lognormal track counts (median 3000, sigma_ln 0.8, clipped to [200, 20000]) and 20-50% noise
hits, N = 6 candidates per seed, FP32.  One step = one pass of the whole hot path over the
batch: hit index, seed estimate, seed fit (layers 0-2), combinatorial building (layers 3-9),
final fit -- everything in libtkf.so kernels, inputs resident in HBM (about 0.8 GB of hits,
larger than L2).

Reported besides the device-timed value: `e2e` (same metric through the C ABI with host
buffers, H2D of the step's inputs and D2H of its results inside the timed region),
`roofline` of the building kernel (ALU-bound: FP32 operations vs the FP32 FMA peak),
`plain` (the same events launched one event at a time: tracks/s and per-event latency
p50/p99), `cpu_baseline` (the FP64 oracle on the host cores on a bounded sample) and the
SM clocks seen during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tkf|reference]
"""
from __future__ import annotations

import argparse
import collections
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "built tracks/s per GB300 at high occupancy; p50/p99 event latency vs plain"
UNIT = "tracks/s"

# FP32 operations of the building kernel's arithmetic (kf_math.cuh, minimal sparse forms;
# an FMA counts 2, divisions, square roots and transcendental functions are not counted):
FLOP_PROPAGATE = 593   # helix/cylinder Newton solve, transport Jacobian, J P J^T
FLOP_WINDOW = 40       # chi2 bounding box -> eta/phi bin ranges
FLOP_CHI2 = 39         # one hit: tangent-plane residual, 2x2 S, chi2, half-cylinder test
FLOP_UPDATE = 335      # Kalman gain, state update, Joseph-form covariance
FLOP_SCATTER = 30      # Highland width and the four covariance terms
# FP64 operations of one MIXED Kalman update (kalman_update<double, float>): B = H P (18), S and
# its determinant (11), the inverse's three terms (3), chi2 (9), gain (36), D = B^T - K S (48),
# Joseph form (168); conversions and the division are not counted
FLOP_UPDATE_FP64 = 290
# Work per seed on the batched workload, counted with the oracle's instrumentation
# (python oracle/opcount.py --events 16 --workload batched, 53756 seeds):
PER_SEED = dict(n_prop=19.2502, n_hits_examined=189.7167, n_updates=18.0985, n_kept=21.7897)
FLOP_PER_SEED = (PER_SEED["n_prop"] * (FLOP_PROPAGATE + FLOP_WINDOW) + PER_SEED["n_hits_examined"] * FLOP_CHI2
                 + PER_SEED["n_updates"] * FLOP_UPDATE + PER_SEED["n_kept"] * 6.0 / 7.0 * FLOP_SCATTER)
# Hits off the layers' cylinders (modules 0.5 cm inside and outside each radius, the two-step
# building): per examined hit only the residual and window test (14) before the step; per hit
# inside the window the short step to its radius with the two measured rows of the transported
# covariance and chi2 (step_chi2, 405); per candidate window the widening by the radial offset
# (15); per update a second propagation (FLOP_PROPAGATE) to the hit's radius.  Work per seed
# from the oracle (python oracle/opcount.py --events 16 --module-dr 1.0, 53756 seeds):
FLOP_RESIDUAL, FLOP_STEP_CHI2, FLOP_WIDEN = 14, 405, 15
PER_SEED_TWO_STEP = dict(n_prop=19.5538, n_hits_examined=213.4334, n_updates=18.2336, n_kept=22.1408,
                         n_steps=25.6186)
FLOP_PER_SEED_TWO_STEP = (PER_SEED_TWO_STEP["n_prop"] * (FLOP_PROPAGATE + FLOP_WINDOW + FLOP_WIDEN)
                          + PER_SEED_TWO_STEP["n_hits_examined"] * FLOP_RESIDUAL
                          + PER_SEED_TWO_STEP["n_steps"] * FLOP_STEP_CHI2
                          + PER_SEED_TWO_STEP["n_updates"] * (FLOP_UPDATE + FLOP_PROPAGATE)
                          + PER_SEED_TWO_STEP["n_kept"] * 6.0 / 7.0 * FLOP_SCATTER)
MODULE_DR = 1.0  # cm between the inner and outer module rows of a layer (hit_dr = 0.5 cm)
# Endcap disks (the forward tracker): per propagation to a plane 296 (closed-form path, one
# helix evaluation, the plane's J P J^T from plane_cov); per window 57 (r-phi and r extents, the
# eta bins of the radii); per examined hit 57 (r-phi and r residuals, the disk's 2x2 S, chi2,
# half-disk and endcap-side tests); per update 359 (the radial row of H adds 24); per kept
# branch's scattering 23.  Work per seed from the oracle on the forward workload (a quarter of
# each event's tracks; python oracle/opcount.py --events 64 --forward, 69674 seeds):
FLOP_PROPAGATE_PLANE, FLOP_WINDOW_DISK, FLOP_CHI2_DISK, FLOP_UPDATE_DISK, FLOP_SCATTER_DISK = 296, 57, 57, 359, 23
PER_SEED_DISK = dict(n_prop=25.7421, n_hits_examined=218.2409, n_updates=26.9508, n_kept=29.2005)
# DRAM bytes (read + write) per seed of the FP32 endcap building (k_first_scan + k_build; one ncu
# capture of its 640-event launches: 130.8 + 480.2 MB for 649 624 seeds; summary in profiles/);
# None when a kernel changes
BUILD3_DRAM_BYTES_PER_SEED = 940.6
FLOP_PER_SEED_DISK = (PER_SEED_DISK["n_prop"] * (FLOP_PROPAGATE_PLANE + FLOP_WINDOW_DISK)
                      + PER_SEED_DISK["n_hits_examined"] * FLOP_CHI2_DISK
                      + PER_SEED_DISK["n_updates"] * FLOP_UPDATE_DISK
                      + PER_SEED_DISK["n_kept"] * 6.0 / 7.0 * FLOP_SCATTER_DISK)
# DRAM bytes (read + write) per seed of the two-step FP32 building (k_first_scan + k_build), from
# one ncu capture of the kernels as built now (160-event case: 124.2 + 434.8 MB for 701 095
# seeds; summary in profiles/); None whenever a kernel changes until it is captured again
BUILD2_DRAM_BYTES_PER_SEED = 797.3
# Warp instructions per seed of the building kernels (ncu smsp__inst_executed.sum of the same
# captures: 47.3 M + 1.675 G one-step, 170.9 M + 3.516 G two-step, for 701 095 seeds), for the
# instruction-issue roofline beside the FP32 one: an SM sub-partition issues at most one warp
# instruction per cycle, 4 per SM; None whenever a kernel changes until it is captured again
BUILD_WARP_INST_PER_SEED, BUILD2_WARP_INST_PER_SEED = 2455.9, 5259.1
# FP32 FMA peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (maximum SM clock)
SM_COUNT, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.07
# libtkf.so kernels per step: hit index (event order, per-event count/scan/place, bin sort),
# seed estimate with seed fit, seed ordering (key, segment totals, segment scan, bin scan,
# place), first-layer scan, build, final fit
KERNELS_PER_STEP = 12
# DRAM bytes (read + write) per seed of the FP32 building (k_first_scan + k_build), from one ncu
# capture of the kernels as built now (160-event case: 124.1 + 433.3 MB for 701 095 seeds;
# summary in profiles/); None whenever a kernel changes until it is captured again
BUILD_DRAM_BYTES_PER_SEED = 795.1
# warp instructions of k_seed_find per layer-0 hit and active lanes per instruction, from one ncu
# capture of the 160-event seeding case (3.185 G instructions for 932 025 first hits; summary in
# profiles/); None whenever the kernel changes until it is captured again
SEED_WARP_INST_PER_FIRST_HIT, SEED_LANES_ACTIVE = 3417.5, 19.01
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1e3
ISSUE_PEAK_WARP_INST_PER_S = SM_COUNT * 4 * SM_MAX_GHZ * 1e9


def _gen_chunk(args):
    from synth import FORWARD_ETA, Detector, EventSpec, event_sizes, forward_detector, generate
    seed, e0, e1, module_dr, forward = args[:5]
    pixel = args[5] if len(args) > 5 else 0
    n, f = event_sizes(seed, 640)
    eta = dict(eta_min=FORWARD_ETA[0], eta_max=FORWARD_ETA[1]) if forward else {}
    if forward:  # the endcaps' share: a quarter of each event's tracks
        n = np.maximum(1, np.rint(0.25 * n)).astype(np.int64)
    return generate(EventSpec(seed=seed, n_events=e1 - e0, n_tracks=n[e0:e1], noise_frac=f[e0:e1], first_event=e0,
                              **eta), forward_detector() if forward else Detector(module_dr=module_dr, pixel_layers=pixel))


def workload(seed: int, n_events: int, pool=None, module_dr=0.0, forward=False, pixel_layers=0):
    """The first n_events events of the 640-event batched workload (generated in parallel
    chunks when a process pool is given; the result does not depend on the chunking);
    module_dr > 0: the same events on modules off the layers' cylinders; forward: a quarter of each
    event's tracks on the endcap tracker (ten pairs of disks), with 1.7 <= |eta| <= 2.5;
    pixel_layers: the same events with that many inner layers of pixel resolution (the seeding
    workload)."""
    from synth import concat
    if pool is None or n_events < 32:
        return _gen_chunk((seed, 0, n_events, module_dr, forward, pixel_layers))
    step = max(1, n_events // 64)
    chunks = [(seed, e, min(e + step, n_events), module_dr, forward, pixel_layers) for e in range(0, n_events, step)]
    return concat(pool.map(_gen_chunk, chunks, chunksize=1))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def issue_roofline(inst_per_seed, seeds, launch_ms):
    """The build launch against the instruction-issue limit: warp instructions (ncu count per
    seed x seeds) per second of the CUDA-event launch time, over 152 SMs x 4 x 2.07 GHz."""
    if inst_per_seed is None:
        return None
    a = inst_per_seed * seeds / (launch_ms / 1e3)
    return {"achieved": a, "peak": ISSUE_PEAK_WARP_INST_PER_S, "unit": "warp instructions/s",
            "frac": a / ISSUE_PEAK_WARP_INST_PER_S, "inst_per_seed": inst_per_seed,
            "source": "ncu smsp__inst_executed.sum per seed of the 160-event capture"}


def physics(b, hit_idx, par, nhits):
    """Physics performance of the built and fitted tracks, the quantities of the paper's figure on
    track-building physics: the fraction of seeds whose track has k hits (k = 0..10, the track
    building's own count), the fraction carrying all ten of their own hits, the transverse
    momentum resolution (pT_fit - pT_true) / pT_true against the generator's truth on the last
    layer for those tracks (half-width of the central 68 % and RMS, in bins of true pT), and the
    fraction with the wrong charge.  hit_idx: [L, n] batch hit ids; par: [6, n]; nhits: [n]."""
    h = np.asarray(hit_idx)
    L, n = h.shape
    nh = np.asarray(nhits)
    frac = {int(k): float(np.mean(nh == k)) for k in range(0, L + 1)}
    own = np.all(h.T == b.trk_hits, axis=1)
    w_fit, w_true = np.asarray(par)[3], b.truth[:, -1, 3]
    pt_fit, pt_true = 1.0 / np.abs(w_fit), 1.0 / np.abs(w_true)
    res = (pt_fit - pt_true) / pt_true
    bins = [(0.5, 1.0), (1.0, 2.0), (2.0, 5.0), (5.0, 10.0)]
    by_pt = []
    for lo, hi in bins:
        m = own & (pt_true >= lo) & (pt_true < hi)
        r = res[m]
        q16, q84 = np.percentile(r, [16, 84]) if len(r) else (np.nan, np.nan)
        by_pt.append({"pt_gev": [lo, hi], "tracks": int(m.sum()), "sigma68": float(0.5 * (q84 - q16)),
                      "rms": float(np.sqrt(np.mean(r * r))) if len(r) else None,
                      "mean": float(np.mean(r)) if len(r) else None})
    r = res[own]
    return {"fraction_by_nhits": frac, "own_ten_hits": float(own.mean()),
            "pt_resolution": {"sigma68": float(0.5 * np.subtract(*np.percentile(r, [84, 16]))),
                              "rms": float(np.sqrt(np.mean(r * r))), "by_pt": by_pt},
            "charge_misid": float(np.mean(np.sign(w_fit[own]) != np.sign(w_true[own])))}


def efficiency(b, hit_idx):
    """Fraction of seeds whose built track has >= 75 % of its hits from the seed's own simulated
    track (hit_idx: [L, n_tracks] batch hit ids, -1 = hole)."""
    h = np.asarray(hit_idx)
    own = (h >= 0) & (b.mc[np.maximum(h, 0)] == np.arange(h.shape[1])[None, :])
    nh = (h >= 0).sum(0)
    return float(np.mean(own.sum(0) >= 0.75 * np.maximum(nh, 1)))


def seeded_efficiency(b, first_hits, hit_idx):
    """Tracking with found seeds: a built track matches simulated track t when >= 75 % of its hits
    are t's; returns the fraction of simulated tracks matched by some seed, the fraction of seeds
    that match none (fakes) and matched seeds per matched track minus one (duplicates).
    first_hits: [n] layer-0 hit of each seed; hit_idx: [L, n] built hit ids (-1 = hole)."""
    h = np.asarray(hit_idx)
    t = b.mc[np.asarray(first_hits)]
    own = (h >= 0) & (b.mc[np.maximum(h, 0)] == t[None, :])
    nh = (h >= 0).sum(0)
    match = (t >= 0) & (own.sum(0) >= 0.75 * np.maximum(nh, 1))
    found = np.unique(t[match])
    return {"track_efficiency": float(len(found) / b.n_tracks), "fake_rate": float(1.0 - match.mean()),
            "duplicate_rate": float(match.sum() / max(len(found), 1) - 1.0)}


# ----------------------------------------------------------------------------- replicas
def job_rate(units, ms, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: the units of every rank summed, over the
    slowest rank's time (ms).  Returns (units, ms_max, units per second)."""
    import torch
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    m = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
    units, ms = float(u.item()), float(m.item())
    return units, ms, units / (ms / 1e3)


# ----------------------------------------------------------------------------- CPU baseline (oracle)
def _oracle_events(chunk, module_dr=0.0, forward=False):
    """Runs the oracle's whole path (index, seed, seed fit, build, final fit) on a few events,
    each given as (oracle hit records, track hit ids [n, L]); returns (tracks, seconds spent
    computing in this process)."""
    import oracle as O
    from synth import FORWARD_PRIOR, Detector, forward_detector
    det = forward_detector() if forward else Detector(module_dr=module_dr)
    g = O.make_geom(det, O.Settings(eta_min=-3.0, n_eta_bins=60, prior_sigma=FORWARD_PRIOR) if forward
                    else O.Settings())
    L = det.n_layers
    done = 0
    t0 = time.perf_counter()
    for hits, local in chunk:
        p0, c0 = O.seed_estimate(g, hits, local[:, :3])
        ids = np.full((len(local), L), -1, dtype=np.int32)
        ids[:, :3] = local[:, :3]
        sp, sP, sc2, snh, _ = O.fit(g, hits, p0, c0, ids, 0, 2)
        res = O.build(g, O.hit_index(g, hits), sp, sP, sc2, snh, ids)
        O.fit(g, hits, p0, c0, res.hits[:, 0, :], 0, L - 1)
        done += len(local)
    return done, time.perf_counter() - t0


def _oracle_fit(chunk):
    """The oracle's plain fit on a few events, each (hit records, track hit ids [n, L]): the
    three-hit estimate and the Kalman fit over every layer with the known hits; returns
    (tracks, seconds computing)."""
    import oracle as O
    from synth import Detector
    det = Detector()
    g = O.make_geom(det)
    done = 0
    t0 = time.perf_counter()
    for hits, local in chunk:
        p0, c0 = O.seed_estimate(g, hits, local[:, :3])
        O.fit(g, hits, p0, c0, local, 0, det.n_layers - 1)
        done += len(local)
    return done, time.perf_counter() - t0


def _oracle_events_modules(chunk):
    """_oracle_events on the module geometry (hits off the layers' cylinders)."""
    return _oracle_events(chunk, MODULE_DR)


def _oracle_events_forward(chunk):
    """_oracle_events on the endcap tracker."""
    return _oracle_events(chunk, forward=True)


def forward_config(tkf, **kw):
    """The library configuration of the endcap tracker (ten pairs of disks at z = +-8..80 cm)."""
    from synth import FORWARD_PRIOR, forward_detector
    det = forward_detector()
    return tkf.default_config(radius=det.radii, x_over_x0=det.x_over_x0, disk_z=det.disk_z, eta_min=-3.0,
                              n_eta_bins=60, prior_sigma=FORWARD_PRIOR, **kw)


def _oracle_backward(chunk):
    """The oracle's backward pass on a few events, each (hit records, hit ids [n, L], states on
    the outermost layer [n, 6], covariances [n, 6, 6]); returns (tracks, seconds computing)."""
    import oracle as O
    from synth import Detector
    det = Detector()
    g = O.make_geom(det)
    done = 0
    t0 = time.perf_counter()
    for hits, ids, par, cov in chunk:
        O.fit_backward(g, hits, par, cov, ids, det.n_layers - 1, 0, 1e4)
        done += len(ids)
    return done, time.perf_counter() - t0


def _unpack_cov(c21):
    """[21, n] packed lower triangle (row order) -> [n, 6, 6]"""
    out = np.zeros((c21.shape[1], 6, 6))
    k = 0
    for i in range(6):
        for j in range(i + 1):
            out[:, i, j] = out[:, j, i] = c21[k]
            k += 1
    return out


def oracle_sample(batch, events):
    """Per-event oracle inputs for the listed events of a generated batch."""
    import oracle as O
    out = []
    for e in events:
        h0, h1 = batch.hit_off[e], batch.hit_off[e + 1]
        t0, t1 = batch.trk_off[e], batch.trk_off[e + 1]
        out.append((O.hits_of(batch, slice(h0, h1)), batch.trk_hits[t0:t1] - h0))
    return out


def cpu_baseline(sample, pool, cores, fn=_oracle_events):
    """The oracle on the sample's items (events), one worker process per core, items dealt
    largest first to the least-loaded worker; (tracks, seconds of the slowest worker's
    computing, wall seconds including the transfer of the inputs to the workers)."""
    chunks, load = [[] for _ in range(cores)], [0] * cores
    for ev in sorted(sample, key=lambda e: -len(e[1])):
        k = load.index(min(load))
        chunks[k].append(ev)
        load[k] += len(ev[1])
    chunks = [c for c in chunks if c]
    t0 = time.perf_counter()
    res = pool.map(fn, chunks, chunksize=1)
    wall = time.perf_counter() - t0
    return sum(r[0] for r in res), max(r[1] for r in res), wall


def sample_events(seed, target_tracks):
    """First events of the batch holding at least `target_tracks` tracks."""
    from synth import event_sizes
    n, _ = event_sizes(seed, 640)
    ev, tot = [], 0
    for e in range(640):
        if tot >= target_tracks:
            break
        ev.append(e)
        tot += int(n[e])
    return ev, tot


def run_reference(a):
    """The oracle (plain FP64 C, one process per host core) timed on bounded samples of the
    same workload: each step builds and fits the tracks of the first events of the batch."""
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    ev, ntr = sample_events(a.seed, a.ref_tracks)
    with ctx.Pool(cores) as pool:
        sample = oracle_sample(workload(a.seed, ev[-1] + 1, pool), ev)
        for _ in range(a.warmup):
            cpu_baseline(sample, pool, cores)
        times, walls = [], []
        for _ in range(a.steps):
            tracks, comp, wall = cpu_baseline(sample, pool, cores)
            times.append(comp)
            walls.append(wall)
    value = ntr / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched building sample: events %d..%d of the 640-event lognormal batch "
                                   "(%d tracks), oracle FP64 on host cores" % (ev[0], ev[-1], ntr),
                       "events": len(ev), "tracks": ntr},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d events, %d tracks per step; time = the slowest worker's computing "
                                       "(mean %.2f s; %.2f s wall with the transfer of the inputs)"
                                       % (len(ev), ntr, statistics.mean(times), statistics.mean(walls))},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- served stream
class LentEvents:
    """Every event of a batch as a tkf_event lent to the server (borrow = 1): hit planes are
    slices of the batch's pinned host planes, seed ids event-local [3][n] blocks of one pinned
    array."""

    def __init__(self, tkf, b, host, n_layers):
        import torch
        self._seeds_t = torch.empty(3 * b.n_tracks, dtype=torch.int32)
        if torch.cuda.is_available():
            self._seeds_t = self._seeds_t.pin_memory()  # pinned like the hit planes
        self.seeds = self._seeds_t.numpy()
        self.events = []
        base = {k: host[k].data_ptr() for k in ("x", "y", "z", "var_u", "var_v", "layer")}
        for e in range(b.n_events):
            h0, h1 = int(b.hit_off[e]), int(b.hit_off[e + 1])
            t0, t1 = int(b.trk_off[e]), int(b.trk_off[e + 1])
            blk = self.seeds[3 * t0:3 * t1].reshape(3, t1 - t0)
            blk[:] = (b.trk_hits[t0:t1, :3] - h0).T
            ev = tkf.Event(*[base[k] + 4 * h0 for k in ("x", "y", "z", "var_u", "var_v", "layer")], h1 - h0,
                           blk.ctypes.data, t1 - t0, 1)
            self.events.append(ev)
        self.array = (tkf.Event * len(self.events))(*self.events)
        self.n_tracks = b.n_tracks
        # bytes the server moves per pass: hit planes, seed ids and two offsets per event in;
        # final parameters, covariance, chi2, nhits and hit ids out
        self.h2d = b.n_hits * 24 + b.n_tracks * 12 + b.n_events * 8
        self.d2h = b.n_tracks * (6 + 21 + 1 + 1 + n_layers) * 4


def device_breakdown(res):
    """Device side of one server pass, from the CUDA-event times each result carries (ms on the
    server's clock, per batch): [span from the first batch's first copy to the last batch's last
    copy, time with at least one batch in flight, input copies, kernels and result copies summed
    over batches, batches]."""
    batches = sorted({(r.gpu_start_ms, r.gpu_inputs_ms, r.gpu_results_ms, r.gpu_done_ms) for r in res})
    busy, end = 0.0, -1e30
    for b in batches:
        busy += max(0.0, b[3] - max(b[0], end))
        end = max(end, b[3])
    span = max(b[3] for b in batches) - batches[0][0] if batches else 0.0
    return [round(x, 3) for x in (span, busy, sum(b[1] - b[0] for b in batches), sum(b[2] - b[1] for b in batches),
                                  sum(b[3] - b[2] for b in batches))] + [len(batches)]


def server_pass(sv, lent):
    """Submits every event of the batch, waits for all results and releases them (one call
    each); returns (seconds, tracks)."""
    t0 = time.perf_counter()
    code, tickets = sv.submit_many(lent.array)
    if code != 0 or len(tickets) != len(lent.events):
        raise RuntimeError("server pass: submission returned %d" % code)
    code, res = sv.wait_all(tickets)
    if code != 0:
        raise RuntimeError("server pass: wait returned %d" % code)
    tracks = sum(r.n_tracks for r in res)
    server_pass.device = device_breakdown(res)
    sv.release_many(tickets)
    return time.perf_counter() - t0, tracks


def served_stream(tkf, lent, rates, seconds, max_events, seed, cfg=None, pool_events=200, **server_opts):
    """Poisson arrivals of the batch's first events (cycled) into a tkf_server; latency is the
    server's completion time minus submission time of each event."""
    n_pool = min(pool_events, len(lent.events))
    pool = lent.events[:n_pool]
    out = []
    for rate in rates:
        sv = tkf.Server(cfg, **server_opts)
        for k in range(5):  # warm-up
            t = sv.submit_struct(pool[k % n_pool])
            sv.poll(t, timeout_us=30_000_000, copy=False)
            sv.release(t)
        rng = np.random.default_rng(seed + int(rate))
        n_ev = int(min(max_events, rate * seconds))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_ev))
        outstanding = collections.deque()
        retries = 0
        lat, first, last, tracks = [], None, None, 0

        def reap(timeout_us):
            # the client side: results are read and released in submission order as they finish
            nonlocal first, last, tracks
            code, r = sv.poll(outstanding[0], timeout_us=timeout_us, copy=False)
            if code != tkf.OK:
                return False
            lat.append((r.t_done_ns - r.t_submit_ns) / 1e6)
            first = r.t_submit_ns if first is None else min(first, r.t_submit_ns)
            last = r.t_done_ns if last is None else max(last, r.t_done_ns)
            tracks += r.n_tracks
            sv.release(outstanding.popleft())
            return True
        t0 = time.perf_counter_ns()
        for k in range(n_ev):
            target = t0 + int(arrivals[k] * 1e9)
            while time.perf_counter_ns() < target:
                if outstanding:
                    reap(0)
            while True:
                code, t = sv.try_submit(pool[k % n_pool])
                if code == tkf.OK:
                    break
                retries += 1
                if outstanding:
                    reap(0)
            outstanding.append(t)
            reap(0)
        while outstanding:
            if not reap(60_000_000):
                raise RuntimeError("served stream: an event did not finish")
        st = sv.stats()
        sv.close()
        lat = np.asarray(lat)
        out.append({"rate_hz": rate, "events": n_ev, "tracks_per_s": tracks / ((last - first) / 1e9),
                    "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
                    "batches": st["batches"], "mean_batch_events": (st["events_done"] - 5) / max(st["batches"] - 5, 1),
                    "retries_queue_full": retries})
    return out


# ----------------------------------------------------------------------------- GPU benchmark
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["tkf", "reference"], default="tkf")
    ap.add_argument("--events", type=int, default=640)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--plain-events", type=int, default=640, help="events timed one at a time")
    ap.add_argument("--cpu-tracks", type=int, default=600000, help="oracle CPU-baseline sample (tracks)")
    ap.add_argument("--ref-tracks", type=int, default=600000,
                    help="reference-arm sample per step (tracks; the same first events as the CPU baseline)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--serve", type=int, default=1, help="1: also measure the served stream")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="arrival window per rate; each rate runs for this long or 20000 events, whichever is fewer")
    ap.add_argument("--mixed", type=int, default=1, help="1: also time the batched step in MIXED precision")
    ap.add_argument("--backward", type=int, default=1,
                    help="1: also time the backward pass of the final fit over the batch's fitted tracks")
    ap.add_argument("--fit", type=int, default=1,
                    help="1: also time the plain fit (known hits, all layers) over every track of the batch")
    ap.add_argument("--probe", type=int, default=1, help="1: measure the SMs' FP32/FP64/SFU throughput")
    ap.add_argument("--batch-scan", type=str, default="10,40,160",
                    help="also time the step on the batch's first K events for each K (comma list; empty: skip)")
    ap.add_argument("--two-step", type=int, default=160,
                    help="events of the batch also timed on modules off the layers' cylinders (two-step building); "
                         "0: skip")
    ap.add_argument("--disks", type=int, default=640,
                    help="events of the batch also timed on the endcap tracker, each with a quarter of its tracks "
                         "(forward tracks on disks); 0: skip")
    ap.add_argument("--seeding", type=int, default=640,
                    help="events of the seeding leg (hit triplets on pixel inner layers; 0: off)")
    ap.add_argument("--tile", type=int, default=0, help="seeds per warp work tile (0: autotuned)")
    ap.add_argument("--e2e-batch", type=int, default=160, help="events per server batch in the e2e measurement")
    ap.add_argument("--e2e-slots", type=int, default=4, help="server slots in the e2e measurement")
    ap.add_argument("--seed-order", type=int, default=1,
                    help="batched form: 1 = build seeds grouped by detector region (the per-event form keeps input order)")
    a = ap.parse_args()
    if a.impl == "reference":
        run_reference(a)
        return

    import multiprocessing as mp
    cores = os.cpu_count() or 1
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    pool = mp.get_context("spawn").Pool(cores)  # before the first CUDA call

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1702_06359_gb300 import tkf

    # weak scaling: every rank builds its own 640-event batch (seed offset by rank)
    b = workload(a.seed + 1000 * rank, a.events, pool)
    n_tr, n_hits = b.n_tracks, b.n_hits
    dev = torch.device("cuda", local)
    pin = lambda arr, dt: torch.as_tensor(np.ascontiguousarray(arr), dtype=dt).pin_memory()
    host = {
        "x": pin(b.x, torch.float32), "y": pin(b.y, torch.float32), "z": pin(b.z, torch.float32),
        "var_u": pin(b.var_u, torch.float32), "var_v": pin(b.var_v, torch.float32),
        "layer": pin(b.layer, torch.int32), "event_off": pin(b.hit_off, torch.int32),
        "seed_hits": pin(b.trk_hits[:, :3].T, torch.int32), "seed_event": pin(b.trk_event, torch.int32),
    }
    d = {k: v.to(dev, non_blocking=False) for k, v in host.items()}
    hits = tkf.DeviceHits(d["x"], d["y"], d["z"], d["var_u"], d["var_v"], d["layer"], d["event_off"])
    ctx = tkf.Context(tkf.default_config(seed_order=a.seed_order, seeds_per_block=max(a.tile, 0)))
    L = ctx.cfg.n_layers
    pipe = tkf.DevicePipeline(ctx, n_hits, b.n_events, n_tr, use_graph=True)
    stream = torch.cuda.current_stream()

    def step():
        pipe.run(hits, d["seed_hits"], d["seed_event"], n_tr, stream=stream)

    # work-tile autotuner of the building kernel (seeds pulled per warp), then warm-up
    step()
    seeds_t, built_t, fitted_t = pipe.outputs()
    spw = 32 // ctx.cfg.n_cand
    tiles = [spw, 2 * spw, 4 * spw, 32, 64, 128]

    class _T:
        def __init__(self, t):
            self.t = t

        def struct(self):
            return self.t
    scratch_out = tkf.DeviceTracks.empty(n_tr, L, device=dev)
    n_grid = {}
    if a.tile > 0:  # fixed work tile (no search), e.g. for profiling a given configuration
        best_tile, tile_ms, tiles = a.tile, [], [a.tile]
    else:
        best_tile, tile_ms = ctx.autotune_build(pipe.index(), _T(seeds_t), scratch_out, tiles, repeats=2,
                                                stream=stream)
    # the same search at N = 4 and 10 candidates per seed (reported; the accuracy claim and the
    # headline stay at N = 6)
    for n_cand in ((4, 10) if a.tile <= 0 else ()):
        cn = tkf.Context(tkf.default_config(seed_order=a.seed_order, n_cand=n_cand))
        spw_n = 32 // n_cand
        tl = sorted({spw_n, 2 * spw_n, 4 * spw_n, 32, 64, 128})
        bt, tms = cn.autotune_build(pipe.index(), _T(seeds_t), scratch_out, tl, repeats=2, stream=stream)
        n_grid[n_cand] = {"tiles": tl, "build_ms": [round(x, 4) for x in tms], "best": bt}
        cn.close()
    n_grid[6] = {"tiles": tiles, "build_ms": [round(x, 4) for x in tile_ms], "best": best_tile}
    del scratch_out
    # building efficiency at each N on this workload (the physics side of the N choice)
    for n_cand in sorted(n_grid):
        if n_cand == 6:
            hid = tkf.tracks_tensors(pipe.outputs()[1], L)["hit_idx"][:, :n_tr]
            n_grid[6]["efficiency"] = efficiency(b, hid.cpu().numpy())
            continue
        cn = tkf.Context(tkf.default_config(seed_order=a.seed_order, n_cand=n_cand,
                                            seeds_per_block=n_grid[n_cand]["best"]))
        pn = tkf.DevicePipeline(cn, n_hits, b.n_events, n_tr, use_graph=False)
        pn.run(hits, d["seed_hits"], d["seed_event"], n_tr, stream=stream)
        cn.sync_status(stream)
        hid = tkf.tracks_tensors(pn.outputs()[1], L)["hit_idx"][:, :n_tr]
        n_grid[n_cand]["efficiency"] = efficiency(b, hid.cpu().numpy())
        pn.close()
        cn.close()
    # the clock sampler starts before the warm-up: nvidia-smi's start-up must not fall in the
    # timed region
    clocks = ClockSampler(local).__enter__()
    time.sleep(0.5)
    for _ in range(a.warmup):
        step()
    ctx.sync_status(stream)

    # ---------------- device-resident throughput (one graph replay per step)
    ev_start = torch.cuda.Event(enable_timing=True)
    ev_stop = torch.cuda.Event(enable_timing=True)
    build_ms = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n_before = len(clocks.lines)
    ev_start.record(stream)
    for k in range(a.steps):
        step()
        build_ms.append(pipe.build_ms())  # waits for the build kernel of this step only
    ev_stop.record(stream)
    torch.cuda.synchronize()
    time.sleep(0.25)
    clocks.__exit__(None, None, None)
    clocks.lines = clocks.lines[n_before:] or clocks.lines[-2:]
    ctx.sync_status(stream)
    ms = ev_start.elapsed_time(ev_stop) / a.steps
    build_ms = statistics.mean(build_ms)
    if dist:
        dist.barrier()
    total_tracks, ms_max, value = job_rate(n_tr, ms, dist, dev)

    # ---------------- physics performance of the step's tracks
    _, built_t, fitted_t = pipe.outputs()
    fv_ph = tkf.tracks_tensors(fitted_t, L)
    phys = physics(b, tkf.tracks_tensors(built_t, L)["hit_idx"][:, :n_tr].cpu().numpy(),
                   fv_ph["par"][:, :n_tr].double().cpu().numpy(), fv_ph["nhits"][:n_tr].cpu().numpy())
    del fv_ph

    # ---------------- the backward pass of the final fit over every fitted track of the batch
    backward = None
    if a.backward:
        _, built_t, fitted_t = pipe.outputs()
        bhid = tkf.tracks_tensors(built_t, L)["hit_idx"]
        back = tkf.DeviceTracks.empty(n_tr, L, device=dev)

        def run_backward():
            ctx.fit_backward(hits, _T(fitted_t), L - 1, 0, back, cov_scale=1e4, hit_idx=bhid, stream=stream)
        for _ in range(max(3, a.warmup)):
            run_backward()
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(a.steps):
            run_backward()
        b1.record(stream)
        torch.cuda.synchronize()
        ctx.sync_status(stream)
        bw_ms = b0.elapsed_time(b1) / a.steps
        nh = back.nhits[:n_tr]
        live = int((nh >= 0).sum())
        bw_flop = (float(nh.clamp(min=0).sum()) * FLOP_UPDATE
                   + live * ((L - 1) * FLOP_PROPAGATE + L * FLOP_SCATTER))
        backward = {"ms": bw_ms, "tracks_per_s": n_tr / bw_ms * 1e3, "achieved_tflops": bw_flop / bw_ms / 1e9,
                    "frac_fp32_peak": bw_flop / bw_ms / 1e9 / FP32_PEAK_TFLOPS, "kernel": "k_fit_backward<float,float>",
                    "flop_per_track": bw_flop / max(live, 1),
                    "form": "tkf_fit_backward over the pipeline's %d fitted tracks, layer 10 to layer 1, covariance "
                            "scale 1e4, FP32; one launch per pass, CUDA events; inputs larger than L2" % n_tr}
        del back

    # ---------------- the plain fit: three-hit estimate and KF fit over all layers with the
    # known hit assignment, every track of the batch (the fit configuration at 2.6 M tracks)
    fit_leg = None
    if a.fit:
        true_ids = torch.as_tensor(np.ascontiguousarray(b.trk_hits.T), dtype=torch.int32).to(dev)
        f_init = tkf.DeviceTracks.empty(n_tr, L, device=dev)
        f_out = tkf.DeviceTracks.empty(n_tr, L, device=dev)

        def run_seed():
            ctx.seed_state(hits, d["seed_hits"], f_init, stream=stream)

        def run_fit():
            ctx.fit(hits, f_init, 0, L - 1, f_out, hit_idx=true_ids, stream=stream)

        def timed(fn):
            for _ in range(max(3, a.warmup)):
                fn()
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(a.steps):
                fn()
            f1.record(stream)
            torch.cuda.synchronize()
            return f0.elapsed_time(f1) / a.steps
        s_ms = timed(run_seed)
        k_ms = timed(run_fit)
        ctx.sync_status(stream)
        f_ms = s_ms + k_ms
        n_full = int((f_out.nhits[:n_tr] == L).sum())  # tracks fitted through every layer's hit
        f_flop = n_tr * ((L - 1) * FLOP_PROPAGATE + L * FLOP_UPDATE + (L - 1) * FLOP_SCATTER)
        fit_leg = {"ms": f_ms, "tracks_per_s": n_tr / f_ms * 1e3,
                   "fit_kernel_ms": k_ms, "seed_kernel_ms": s_ms,
                   "achieved_tflops": f_flop / k_ms / 1e9,
                   "frac_fp32_peak": f_flop / k_ms / 1e9 / FP32_PEAK_TFLOPS,
                   "frac_fp32_peak_with_seed": f_flop / f_ms / 1e9 / FP32_PEAK_TFLOPS,
                   "flop_per_track": f_flop / n_tr,
                   "kernels": "k_seed<float> (the three-hit estimate, memory-bound), k_fit<float,float> (the KF "
                              "over ten layers, every counted FLOP)",
                   "tracks_with_all_hits": n_full,
                   "form": "tkf_seed_state, then tkf_fit (layers 1..10, the known hit lists), over the batch's %d "
                           "tracks, FP32; each timed alone with CUDA events over %d passes (frac_fp32_peak: the fit "
                           "kernel; ms and tracks_per_s: both); inputs larger than L2" % (n_tr, a.steps)}
        del f_init, f_out, true_ids

    # ---------------- the SMs' arithmetic throughput (measured roofline denominators)
    alu = tkf.probe_alu(stream) if a.probe else None

    # ---------------- throughput against batch size: the step on the batch's first K events
    batch_scan = None
    if a.batch_scan:
        batch_scan = []
        for k in sorted({int(x) for x in a.batch_scan.split(",") if x.strip()}):
            if not 0 < k < b.n_events:
                continue
            nh_k, nt_k = int(b.hit_off[k]), int(b.trk_off[k])
            hk = tkf.DeviceHits(d["x"][:nh_k], d["y"][:nh_k], d["z"][:nh_k], d["var_u"][:nh_k], d["var_v"][:nh_k],
                                d["layer"][:nh_k], d["event_off"][:k + 1])
            sk = d["seed_hits"][:, :nt_k].contiguous()  # [3][K's tracks]: rows strided by the pipeline's capacity
            pk = tkf.DevicePipeline(ctx, nh_k, k, nt_k, use_graph=True)
            for _ in range(max(3, a.warmup)):
                pk.run(hk, sk, d["seed_event"], nt_k, stream=stream)
            torch.cuda.synchronize()
            k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            for _ in range(a.steps):
                pk.run(hk, sk, d["seed_event"], nt_k, stream=stream)
            k1.record(stream)
            torch.cuda.synchronize()
            ctx.sync_status(stream)
            kms = k0.elapsed_time(k1) / a.steps
            batch_scan.append({"events": k, "tracks": nt_k, "ms_per_step": kms, "tracks_per_s": nt_k / (kms / 1e3)})
            pk.close()
        batch_scan.append({"events": b.n_events, "tracks": n_tr, "ms_per_step": ms, "tracks_per_s": n_tr / (ms / 1e3)})

    # ---------------- the same events on modules off the layers' cylinders (two-step building)
    two_step = None
    b2 = None
    if a.two_step > 0:
        n2 = min(a.two_step, a.events)
        b2 = workload(a.seed + 1000 * rank, n2, pool, module_dr=MODULE_DR)
        t2 = lambda arr, dt: torch.as_tensor(np.ascontiguousarray(arr), dtype=dt).to(dev)
        d2 = {"x": t2(b2.x, torch.float32), "y": t2(b2.y, torch.float32), "z": t2(b2.z, torch.float32),
              "var_u": t2(b2.var_u, torch.float32), "var_v": t2(b2.var_v, torch.float32),
              "layer": t2(b2.layer, torch.int32), "event_off": t2(b2.hit_off, torch.int32),
              "seed_hits": t2(b2.trk_hits[:, :3].T, torch.int32), "seed_event": t2(b2.trk_event, torch.int32)}
        hits2 = tkf.DeviceHits(d2["x"], d2["y"], d2["z"], d2["var_u"], d2["var_v"], d2["layer"], d2["event_off"])
        c2 = tkf.Context(tkf.default_config(seed_order=a.seed_order, hit_dr=0.5 * MODULE_DR,
                                            seeds_per_block=max(a.tile, 0)))
        n2t = b2.n_tracks
        p2 = tkf.DevicePipeline(c2, b2.n_hits, b2.n_events, n2t, use_graph=True)
        step2 = lambda: p2.run(hits2, d2["seed_hits"], d2["seed_event"], n2t, stream=stream)
        step2()
        s2t = p2.outputs()[0]
        if a.tile > 0:
            tile2, t2ms = a.tile, []
        else:
            sc2 = tkf.DeviceTracks.empty(n2t, L, device=dev)
            tile2, t2ms = c2.autotune_build(p2.index(), _T(s2t), sc2, tiles, repeats=2, stream=stream)
            del sc2
            c2.close()
            p2.close()
            c2 = tkf.Context(tkf.default_config(seed_order=a.seed_order, hit_dr=0.5 * MODULE_DR,
                                                seeds_per_block=tile2))
            p2 = tkf.DevicePipeline(c2, b2.n_hits, b2.n_events, n2t, use_graph=True)
            step2 = lambda: p2.run(hits2, d2["seed_hits"], d2["seed_event"], n2t, stream=stream)
        for _ in range(max(3, a.warmup)):
            step2()
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        qb = []
        q0.record(stream)
        for _ in range(a.steps):
            step2()
            qb.append(p2.build_ms())
        q1.record(stream)
        torch.cuda.synchronize()
        c2.sync_status(stream)
        q_ms = q0.elapsed_time(q1) / a.steps
        q_build = statistics.mean(qb)
        hid2 = tkf.tracks_tensors(p2.outputs()[1], L)["hit_idx"][:, :n2t].cpu().numpy()
        ach2 = FLOP_PER_SEED_TWO_STEP * n2t / (q_build / 1e3) / 1e12
        two_step = {
            "value": n2t / (q_ms / 1e3), "unit": UNIT, "ms_per_step": q_ms, "build_ms": q_build,
            "events": b2.n_events, "tracks": n2t, "hits": b2.n_hits, "efficiency": efficiency(b2, hid2),
            "own_hit_lists": float(np.mean(np.all(hid2.T == b2.trk_hits, axis=1))),
            "seeds_per_warp_tile": tile2, "autotune_build_ms": [round(x, 4) for x in t2ms],
            "roofline": {"kernel": "k_first_scan + k_build<6,float,float,two-step>", "bound": "alu", "achieved": ach2,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach2 / FP32_PEAK_TFLOPS,
                         "traffic": None if BUILD2_DRAM_BYTES_PER_SEED is None else BUILD2_DRAM_BYTES_PER_SEED * n2t,
                         "traffic_unit": "bytes per launch pair (ncu DRAM read + write of the 160-event case, per seed)",
                         "launch_ms": q_build, "flop_per_seed": FLOP_PER_SEED_TWO_STEP,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                         "issue": issue_roofline(BUILD2_WARP_INST_PER_SEED, n2t, q_build)},
            "form": "events 0..%d of the batched workload with each layer's modules 0.5 cm inside and outside "
                    "its radius (hit_dr = 0.5 cm): window on the average radius, a second propagation to each "
                    "candidate hit's radius; fits to each hit's radius; FP32, N = 6, whole step replayed from a "
                    "CUDA graph; inputs larger than L2" % (b2.n_events - 1)}
        p2.close()
        c2.close()
        del d2, hits2

    # ---------------- forward tracks on the endcap disks (the "endcap z" geometry)
    disks = None
    b3 = None
    if a.disks > 0:
        n3 = min(a.disks, 640)
        b3 = workload(a.seed + 1000 * rank, n3, pool, forward=True)
        t3 = lambda arr, dt: torch.as_tensor(np.ascontiguousarray(arr), dtype=dt).to(dev)
        d3 = {"x": t3(b3.x, torch.float32), "y": t3(b3.y, torch.float32), "z": t3(b3.z, torch.float32),
              "var_u": t3(b3.var_u, torch.float32), "var_v": t3(b3.var_v, torch.float32),
              "layer": t3(b3.layer, torch.int32), "event_off": t3(b3.hit_off, torch.int32),
              "seed_hits": t3(b3.trk_hits[:, :3].T, torch.int32), "seed_event": t3(b3.trk_event, torch.int32)}
        hits3 = tkf.DeviceHits(d3["x"], d3["y"], d3["z"], d3["var_u"], d3["var_v"], d3["layer"], d3["event_off"])
        n3t = b3.n_tracks
        c3 = tkf.Context(forward_config(tkf, seed_order=a.seed_order, seeds_per_block=max(a.tile, 0)))
        p3 = tkf.DevicePipeline(c3, b3.n_hits, b3.n_events, n3t, use_graph=True)
        p3.run(hits3, d3["seed_hits"], d3["seed_event"], n3t, stream=stream)
        if a.tile > 0:
            tile3, t3ms = a.tile, []
        else:
            sc3 = tkf.DeviceTracks.empty(n3t, L, device=dev)
            tile3, t3ms = c3.autotune_build(p3.index(), _T(p3.outputs()[0]), sc3, tiles, repeats=2, stream=stream)
            del sc3
            p3.close()
            c3.close()
            c3 = tkf.Context(forward_config(tkf, seed_order=a.seed_order, seeds_per_block=tile3))
            p3 = tkf.DevicePipeline(c3, b3.n_hits, b3.n_events, n3t, use_graph=True)
        step3 = lambda: p3.run(hits3, d3["seed_hits"], d3["seed_event"], n3t, stream=stream)
        for _ in range(max(3, a.warmup)):
            step3()
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        qb = []
        q0.record(stream)
        for _ in range(a.steps):
            step3()
            qb.append(p3.build_ms())
        q1.record(stream)
        torch.cuda.synchronize()
        c3.sync_status(stream)
        d_ms = q0.elapsed_time(q1) / a.steps
        d_build = statistics.mean(qb)
        hid3 = tkf.tracks_tensors(p3.outputs()[1], L)["hit_idx"][:, :n3t].cpu().numpy()
        own3 = (hid3.T == b3.trk_hits).sum(axis=1)
        ach3 = FLOP_PER_SEED_DISK * n3t / (d_build / 1e3) / 1e12
        disks = {
            "value": n3t / (d_ms / 1e3), "unit": UNIT, "ms_per_step": d_ms, "build_ms": d_build,
            "events": b3.n_events, "tracks": n3t, "hits": b3.n_hits, "efficiency": efficiency(b3, hid3),
            "own_hit_lists": float(np.mean(own3 == L)), "seeds_per_warp_tile": tile3,
            "autotune_build_ms": [round(x, 4) for x in t3ms],
            "roofline": {"kernel": "k_first_scan + k_build<6,float,float,disks>", "bound": "alu", "achieved": ach3,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach3 / FP32_PEAK_TFLOPS,
                         "traffic": BUILD3_DRAM_BYTES_PER_SEED * n3t if BUILD3_DRAM_BYTES_PER_SEED else None,
                         "traffic_unit": "bytes per launch pair (ncu DRAM read + write of the 640-event endcap launches, "
                                         "per seed)",
                         "launch_ms": d_build, "flop_per_seed": FLOP_PER_SEED_DISK,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
            "form": "events 0..%d of the batched workload, each with a quarter of its tracks (the endcaps' "
                    "share) and its noise fraction, on the endcap tracker (ten pairs of disks at z = +-8..80 cm, "
                    "tracks with 1.7 <= |eta| <= 2.5, hits in r-phi and r); FP32, N = 6, whole step replayed from "
                    "a CUDA graph" % (b3.n_events - 1)}
        p3.close()
        c3.close()
        del d3, hits3

    # ---------------- seeding from hit triplets, then the whole chain with the found seeds
    seeding = None
    if a.seeding > 0:
        n4 = min(a.seeding, 640)
        b4 = workload(a.seed + 1000 * rank, n4, pool, pixel_layers=4)
        t4 = lambda arr, dt: torch.as_tensor(np.ascontiguousarray(arr), dtype=dt).to(dev)
        hits4 = tkf.DeviceHits(t4(b4.x, torch.float32), t4(b4.y, torch.float32), t4(b4.z, torch.float32),
                               t4(b4.var_u, torch.float32), t4(b4.var_v, torch.float32), t4(b4.layer, torch.int32),
                               t4(b4.hit_off, torch.int32))
        c4 = tkf.Context(tkf.default_config(seed_order=a.seed_order, seeds_per_block=best_tile))
        idx4 = c4.build_hit_index(hits4, stream=stream)
        cuts4 = tkf.default_seed_cuts()
        n_first = int((b4.layer == 0).sum())
        sh4 = torch.empty((3, n_first), dtype=torch.int32, device=dev)
        se4 = torch.empty(n_first, dtype=torch.int32, device=dev)
        nf4 = torch.zeros(1, dtype=torch.int32, device=dev)
        find4 = lambda: c4.find_seeds(idx4, cuts4, n_first, sh4, se4, nf4, stream=stream)
        for _ in range(max(3, a.warmup)):
            find4()
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(a.steps):
            find4()
        s1.record(stream)
        torch.cuda.synchronize()
        c4.sync_status(stream)
        seed_ms = s0.elapsed_time(s1) / a.steps
        n_found = int(nf4.item())
        seeds_np = sh4[:, :n_found].cpu().numpy()
        th4 = b4.trk_hits
        pick1 = np.full(b4.n_hits, -1, dtype=np.int64)
        pick2 = np.full(b4.n_hits, -1, dtype=np.int64)
        pick1[seeds_np[0]], pick2[seeds_np[0]] = seeds_np[1], seeds_np[2]
        own_trip = float(np.mean((pick1[th4[:, 0]] == th4[:, 1]) & (pick2[th4[:, 0]] == th4[:, 2])))
        # the chain: index, seeding into the pipeline's seed rows, seed fit, building, final fit
        shc = torch.empty((3, n_found), dtype=torch.int32, device=dev)
        sec = torch.empty(n_found, dtype=torch.int32, device=dev)
        p4 = tkf.DevicePipeline(c4, b4.n_hits, b4.n_events, n_found, use_graph=True)

        def chain():
            c4.build_hit_index(hits4, reuse=idx4, stream=stream)
            c4.find_seeds(idx4, cuts4, n_found, shc, sec, nf4, stream=stream)
            p4.run(hits4, shc, sec, n_found, stream=stream)

        for _ in range(max(3, a.warmup)):
            chain()
        torch.cuda.synchronize()
        s0.record(stream)
        for _ in range(a.steps):
            chain()
        s1.record(stream)
        torch.cuda.synchronize()
        c4.sync_status(stream)
        chain_ms = s0.elapsed_time(s1) / a.steps
        hid4 = tkf.tracks_tensors(p4.outputs()[2], L)["hit_idx"][:, :n_found].cpu().numpy()
        seeding = {
            "value": b4.n_tracks / (chain_ms / 1e3), "unit": UNIT, "ms_per_step": chain_ms,
            "seeding_ms": seed_ms, "first_hits_per_s": n_first / (seed_ms / 1e3), "events": b4.n_events,
            "tracks": b4.n_tracks, "hits": b4.n_hits, "first_layer_hits": n_first, "seeds": n_found,
            "seeds_per_track": n_found / b4.n_tracks, "own_triplet": own_trip,
            "roofline": None if SEED_WARP_INST_PER_FIRST_HIT is None else {
                "kernel": "k_seed_find (+ k_seed_count, k_seed_scan, k_seed_scatter in seeding_ms)", "bound": "issue",
                "achieved": SEED_WARP_INST_PER_FIRST_HIT * n_first / (seed_ms / 1e3),
                "peak": ISSUE_PEAK_WARP_INST_PER_S, "unit": "warp instructions/s",
                "frac": SEED_WARP_INST_PER_FIRST_HIT * n_first / (seed_ms / 1e3) / ISSUE_PEAK_WARP_INST_PER_S,
                "inst_per_first_hit": SEED_WARP_INST_PER_FIRST_HIT, "lanes_active": SEED_LANES_ACTIVE,
                "source": "ncu smsp__inst_executed.sum per layer-0 hit and thread instructions per warp instruction "
                          "of the 160-event capture; 152 SMs x 4 x 2.07 GHz"},
            **seeded_efficiency(b4, seeds_np[0], hid4),
            "cuts": {k: getattr(cuts4, k) for k in ("pt_min", "kappa_slack", "z_vertex", "d0_max", "dz_max",
                                                    "conf_rphi", "conf_z", "confirm")},
            "form": "the batched workload's events 0..%d with pixel resolution (20 um r-phi, 50 um z) on layers "
                    "0-3: tkf_find_seeds over the hit index (k_seed_find, one thread per layer-0 hit, then "
                    "count, scan and scatter) timed alone (seeding_ms); value = simulated tracks per second "
                    "of the chain hit index + seeding + pipeline (its own index, seed fit, building, final "
                    "fit) with the found seeds; FP32, N = 6" % (b4.n_events - 1)}
        p4.close()
        c4.close()
        del hits4, sh4, se4, shc, sec

    # ---------------- end to end through host buffers
    _, built_t, fitted_t = pipe.outputs()
    fv = tkf.tracks_tensors(fitted_t, L)
    outs = [fv["par"][:, :n_tr], fv["chi2"][:n_tr], fv["nhits"][:n_tr], fv["hit_idx"][:, :n_tr]]
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    res_host = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
    d2h = sum(r.numel() * r.element_size() for r in res_host)
    e2e_start = torch.cuda.Event(enable_timing=True)
    e2e_stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e2e_start.record(stream)
    for _ in range(a.steps):
        for k, v in host.items():
            d[k].copy_(v, non_blocking=True)
        step()
        for r, o in zip(res_host, outs):
            r.copy_(o, non_blocking=True)
    e2e_stop.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e2e_start.elapsed_time(e2e_stop) / a.steps

    e2e_pipe = {"value": job_rate(n_tr, e2e_ms, dist, dev)[2], "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "form": "graph-replayed pipeline with torch copies of pinned host planes on the same stream"}

    # ---------------- end to end through the public serving API (host buffers lent to tkf_server)
    lent = LentEvents(tkf, b, host, L)
    # pinned result memory for about 25 full-size batches (a pass holds the results of all its 10-16
    # batches until it waits for them): after the warm-up passes every batch finds a free result
    # buffer and nothing is allocated or freed while timing
    e2e_opts = dict(n_slots=a.e2e_slots, max_batch_events=a.e2e_batch, max_batch_hits=1 << 24,
                    max_batch_tracks=1 << 20, result_bytes=4 << 30)
    sv = tkf.Server(ctx.cfg, **e2e_opts)
    for _ in range(max(1, a.warmup)):
        server_pass(sv, lent)
    e2e_s = []
    allocs0 = sv.stats()["result_allocs"]
    gc.collect()
    gc.disable()  # a serving host does not collect garbage between a batch's submission and its results
    devices = []
    try:
        for _ in range(a.steps):
            dt, nt = server_pass(sv, lent)
            assert nt == n_tr
            e2e_s.append(dt)
            devices.append(server_pass.device)
    finally:
        gc.enable()
    e2e_allocs = sv.stats()["result_allocs"] - allocs0
    sv.close()
    e2e = {"value": job_rate(n_tr, 1e3 * statistics.mean(e2e_s), dist, dev)[2], "unit": UNIT,
           "h2d_bytes_per_step": lent.h2d,
           "d2h_bytes_per_step": lent.d2h, "ms_per_step": 1e3 * statistics.mean(e2e_s),
           "ms_per_step_median": 1e3 * statistics.median(e2e_s), "ms_per_step_max": 1e3 * max(e2e_s),
           "ms_per_step_p99": 1e3 * float(np.percentile(e2e_s, 99)),
           "passes_ms": [round(1e3 * x, 3) for x in e2e_s],
           "result_buffer_allocations_while_timed": e2e_allocs,
           "device_ms": devices,
           "form": "tkf_submit_events of all %d events (hit planes lent from pinned host memory), tkf_wait_all, "
                   "tkf_release_many; %d slots, batches of up to %d events; host wall clock, mean over the "
                   "timed passes (Python garbage collection off during them); device_ms: per pass, the device "
                   "span from the first batch's first copy to the last batch's last copy, the time with a batch "
                   "in flight, the input copies, kernels and result copies summed over batches, and the "
                   "batches"
                   % (b.n_events, a.e2e_slots, a.e2e_batch)}

    # ---------------- the same batched step in MIXED precision (FP64 inverse + Joseph update)
    mixed = None
    if a.mixed:
        mctx = tkf.Context(tkf.default_config(seed_order=a.seed_order, precision=tkf.MIXED,
                                              seeds_per_block=best_tile))
        mpipe = tkf.DevicePipeline(mctx, n_hits, b.n_events, n_tr, use_graph=True)
        mstep = lambda: mpipe.run(hits, d["seed_hits"], d["seed_event"], n_tr, stream=stream)
        for _ in range(max(3, a.warmup)):
            mstep()
        torch.cuda.synchronize()
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        mb = []
        m0.record(stream)
        for _ in range(a.steps):
            mstep()
            mb.append(mpipe.build_ms())
        m1.record(stream)
        torch.cuda.synchronize()
        mctx.sync_status(stream)
        mms = m0.elapsed_time(m1) / a.steps
        mb_ms = statistics.mean(mb)
        m_fp64 = PER_SEED["n_updates"] * FLOP_UPDATE_FP64 * n_tr / (mb_ms / 1e3) / 1e12
        mixed = {"value": n_tr / (mms / 1e3), "unit": UNIT, "ms_per_step": mms, "build_ms": mb_ms,
                 "roofline": {"kernel": "k_first_scan + k_build<6,float,double>", "bound": "fp64", "achieved": m_fp64,
                              "peak": None, "unit": "TFLOP/s", "frac": None,
                              "flop_per_seed_fp64": PER_SEED["n_updates"] * FLOP_UPDATE_FP64,
                              "note": "FP64 arithmetic of the updates against the measured FP64 multiply-add "
                                      "rate (alu_peaks); each block's updates run packed into full warps; ncu "
                                      "shows the FP64 pipe 77 % busy at 19 of 32 active lanes, the rest of its "
                                      "work the update's other double operations (reciprocal, negations, "
                                      "compares)"},
                 "precision": "mixed: FP32 propagation, window and chi2; FP64 innovation inverse and Joseph update",
                 "seeds_per_warp_tile": best_tile}
        mpipe.close()
        mctx.close()
        if alu is not None:
            mixed["roofline"]["peak"] = alu["fp64_tflops"]
            mixed["roofline"]["frac"] = m_fp64 / alu["fp64_tflops"]

    # ---------------- plain form: one event per pass (direct launches), per-event latency
    plain = None
    if a.plain_events > 0:
        n_pe = min(a.plain_events, b.n_events)
        views = []
        hit_off, trk_off = b.hit_off, b.trk_off
        stride = int(np.max(np.diff(trk_off[:n_pe + 1])))
        max_h = int(np.max(np.diff(hit_off[:n_pe + 1])))
        for e in range(n_pe):
            h0, h1, t0_, t1_ = int(hit_off[e]), int(hit_off[e + 1]), int(trk_off[e]), int(trk_off[e + 1])
            off = torch.tensor([0, h1 - h0], dtype=torch.int32, device=dev)
            sh = torch.full((3, stride), -1, dtype=torch.int32, device=dev)
            sh[:, :t1_ - t0_] = d["seed_hits"][:, t0_:t1_] - h0
            views.append((tkf.DeviceHits(d["x"][h0:h1], d["y"][h0:h1], d["z"][h0:h1], d["var_u"][h0:h1],
                                         d["var_v"][h0:h1], d["layer"][h0:h1], off), sh,
                          torch.zeros(stride, dtype=torch.int32, device=dev), t1_ - t0_))
        pctx = tkf.Context(tkf.default_config())
        ppipe = tkf.DevicePipeline(pctx, max_h, 1, stride, use_graph=False)
        for hv, sh, se, nt in views[:3]:
            ppipe.run(hv, sh, se, nt, stream=stream)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in views]
        p_start = torch.cuda.Event(enable_timing=True)
        p_stop = torch.cuda.Event(enable_timing=True)
        p_start.record(stream)
        for (hv, sh, se, nt), (e0, e1) in zip(views, evs):
            e0.record(stream)
            ppipe.run(hv, sh, se, nt, stream=stream)
            e1.record(stream)
        p_stop.record(stream)
        torch.cuda.synchronize()
        pctx.sync_status(stream)
        lat = np.array([e0.elapsed_time(e1) for e0, e1 in evs])
        pe_tracks = int(trk_off[n_pe])
        plain = {"value": pe_tracks / (p_start.elapsed_time(p_stop) / 1e3), "unit": UNIT, "events": n_pe,
                 "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
                 "form": "one event per pipeline pass, direct launches, same kernels and stream"}
        ppipe.close()

    # ---------------- served stream: Poisson arrivals, continuous batching vs one event at a time
    serve = None
    if a.serve and rank == 0:
        torch.cuda.synchronize()
        rates = [1000.0, 5000.0, 20000.0]
        hmax = int(np.max(np.diff(b.hit_off[:201])))
        opts = dict(n_slots=3, max_batch_events=64, max_batch_hits=max(1 << 22, hmax), max_batch_tracks=1 << 18)
        mcfg = tkf.default_config(precision=tkf.MIXED)
        serve = {"batched": served_stream(tkf, lent, rates, a.serve_seconds, 20000, a.seed, cfg=mcfg, **opts),
                 "batched_fp32": served_stream(tkf, lent, rates, a.serve_seconds, 20000, a.seed, **opts),
                 "plain": served_stream(tkf, lent, rates, a.serve_seconds, 20000, a.seed, n_slots=1,
                                        max_batch_events=1, max_batch_hits=max(hmax, 1), max_batch_tracks=1 << 16),
                 "batched_form": "MIXED precision, continuous batching over 3 slots, up to 64 events per batch "
                                 "(batched_fp32: the same in FP32)",
                 "plain_form": "FP32, one event per batch, one slot",
                 "arrivals": "Poisson (seeded exponential gaps), events cycled from the batch's first 200, "
                             "hit planes lent from pinned host memory",
                 "latency": "server completion time minus submission time"}

    # ---------------- CPU baseline
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        ev, ntr = sample_events(a.seed, a.cpu_tracks)
        sample = oracle_sample(b, ev)
        tracks, comp, wall = cpu_baseline(sample, pool, cores)
        # one core: the same oracle in this process on the sample's first events (>= 100 000 tracks)
        ev1 = ev[:max(1, next((k + 1 for k in range(len(ev)) if int(b.trk_off[ev[k] + 1] - b.trk_off[ev[0]]) >= 100000),
                              len(ev)))]
        n1, comp1 = _oracle_events(sample[:len(ev1)])
        cpu = {"value": tracks / comp, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "events %d..%d of the same batch (%d tracks): index, seed, seed fit, build, final fit, "
                         "FP64, one process per core, events dealt largest first; time = the slowest worker's "
                         "computing (%.2f s; %.2f s wall with the transfer of the inputs to the workers)"
                         % (ev[0], ev[-1], tracks, comp, wall),
               "wall_value": tracks / wall,
               "single_core": {"value": n1 / comp1, "unit": UNIT, "cores": 1,
                               "sample": "events %d..%d (%d tracks), one process" % (ev1[0], ev1[-1], n1)}}
        if backward is not None:
            # the oracle's backward pass beside the GPU's, from the GPU's fitted states of the
            # same sample events
            _, built_t, fitted_t = pipe.outputs()
            t_hi = int(b.trk_off[ev[-1] + 1])
            hid = tkf.tracks_tensors(built_t, L)["hit_idx"][:, :t_hi].T.cpu().numpy()
            fv = tkf.tracks_tensors(fitted_t, L)
            fpar = fv["par"][:, :t_hi].double().T.cpu().numpy()
            fcov = _unpack_cov(fv["cov"][:, :t_hi].double().cpu().numpy())
            fnh = fv["nhits"][:t_hi].cpu().numpy()
            bsample = []
            for (hits_e, _), e in zip(sample, ev):
                t0, t1, h0 = int(b.trk_off[e]), int(b.trk_off[e + 1]), int(b.hit_off[e])
                live = np.nonzero(fnh[t0:t1] >= 0)[0] + t0
                ids = np.where(hid[live] >= 0, hid[live] - h0, -1).astype(np.int32)
                bsample.append((hits_e, ids, fpar[live], fcov[live]))
            nb, compb, wallb = cpu_baseline(bsample, pool, cores, fn=_oracle_backward)
            backward["cpu_baseline"] = {
                "value": nb / compb, "unit": "tracks/s", "cores": cores, "kind": "oracle",
                "sample": "the backward pass of events %d..%d (%d tracks) from the GPU's fitted states, FP64, one "
                          "process per core; time = the slowest worker's computing (%.2f s; %.2f s wall with the "
                          "transfer of the inputs)" % (ev[0], ev[-1], nb, compb, wallb)}
        if fit_leg is not None:
            nf, compf, wallf = cpu_baseline(sample, pool, cores, fn=_oracle_fit)
            fit_leg["cpu_baseline"] = {
                "value": nf / compf, "unit": "tracks/s", "cores": cores, "kind": "oracle",
                "sample": "the plain fit of events %d..%d (%d tracks), FP64, one process per core; time = the "
                          "slowest worker's computing (%.2f s; %.2f s wall)" % (ev[0], ev[-1], nf, compf, wallf)}
        if two_step is not None:
            # the oracle on the first events of the module-geometry batch (its share of the sample)
            n2s = next((k + 1 for k in range(b2.n_events) if int(b2.trk_off[k + 1]) >= a.cpu_tracks // 4), b2.n_events)
            tracks2, comp2, wall2 = cpu_baseline(oracle_sample(b2, range(n2s)), pool, cores, fn=_oracle_events_modules)
            two_step["cpu_baseline"] = {
                "value": tracks2 / comp2, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": "events 0..%d of the module-geometry batch (%d tracks): index, seed, seed fit, two-step "
                          "build, final fit, FP64, one process per core; time = the slowest worker's computing "
                          "(%.2f s; %.2f s wall)" % (n2s - 1, tracks2, comp2, wall2)}
        if disks is not None:
            n3s = next((k + 1 for k in range(b3.n_events) if int(b3.trk_off[k + 1]) >= a.cpu_tracks // 4), b3.n_events)
            tracks3, comp3, wall3 = cpu_baseline(oracle_sample(b3, range(n3s)), pool, cores, fn=_oracle_events_forward)
            disks["cpu_baseline"] = {
                "value": tracks3 / comp3, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": "events 0..%d of the endcap batch (%d tracks): index, seed, seed fit, build, final fit, "
                          "FP64, one process per core; time = the slowest worker's computing (%.2f s; %.2f s wall)"
                          % (n3s - 1, tracks3, comp3, wall3)}
    pool.close()

    achieved = FLOP_PER_SEED * n_tr / (build_ms / 1e3) / 1e12
    line = {
        "impl": "tkf", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched building: %d events, lognormal tracks (median 3000, sigma_ln 0.8, "
                               "200..20000), noise 20-50%%, N=6, fp32, one persistent build launch per step, "
                               "whole step replayed from a CUDA graph"
                               % b.n_events,
                   "events": b.n_events, "tracks": n_tr, "hits": n_hits, "n_cand": 6, "precision": "fp32",
                   "seeds_per_warp_tile": best_tile, "cuda_graph": True,
                   "l2": "inputs larger than L2 (%.0f MB of hit planes)" % (n_hits * 24 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"kernel": "k_first_scan + k_build<6,float,float>", "bound": "alu", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": None if BUILD_DRAM_BYTES_PER_SEED is None else BUILD_DRAM_BYTES_PER_SEED * n_tr,
                     "traffic_unit": "bytes per launch pair (ncu DRAM read + write, scaled by seeds from the 160-event case)",
                     "launch_note": "launch_ms: CUDA events around tkf_build_tracks inside the graph (seed ordering, "
                                    "k_first_scan, k_build)",
                     "launch_ms": build_ms, "flop_per_seed": FLOP_PER_SEED,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                     "issue": issue_roofline(BUILD_WARP_INST_PER_SEED, n_tr, build_ms),
                     "measured_peak": None if alu is None else alu["fp32_tflops"],
                     "frac_of_measured": None if alu is None else achieved / alu["fp32_tflops"]},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "e2e_pipeline": e2e_pipe,
        "mixed": mixed,
        "backward_pass": backward,
        "two_step": two_step,
        "disks": disks,
        "seeding": seeding,
        "batch_scan": batch_scan,
        "physics": phys,
        "fit": fit_leg,
        "alu_peaks": None if alu is None else dict(alu, source="tkf_probe_alu: independent FMA / __sinf chains, "
                                                               "2048 threads per SM, best of 3 launches"),
        "plain": plain,
        "serve": serve,
        "autotune": {"grid": "seeds per warp tile x candidates per seed N (build launch ms)",
                     "by_n_cand": n_grid, "best": best_tile, "n_cand": 6,
                     "hit_tile": None,
                     "hit_tile_note": "no hit-tile axis: the build kernel stages no hit tiles in shared memory; each "
                                      "candidate's window is a few short index ranges (about 3 hits) read through "
                                      "L1/L2, so there is no tile size to tune"},
        "gpu_launches": KERNELS_PER_STEP * a.steps,
        "clocks": clocks.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
