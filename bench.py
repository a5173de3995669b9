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
# Work per seed on the batched workload, counted with the oracle's instrumentation
# (python oracle/opcount.py --events 16 --workload batched, 53756 seeds):
PER_SEED = dict(n_prop=19.2502, n_hits_examined=189.7167, n_updates=18.0985, n_kept=21.7897)
FLOP_PER_SEED = (PER_SEED["n_prop"] * (FLOP_PROPAGATE + FLOP_WINDOW) + PER_SEED["n_hits_examined"] * FLOP_CHI2
                 + PER_SEED["n_updates"] * FLOP_UPDATE + PER_SEED["n_kept"] * 6.0 / 7.0 * FLOP_SCATTER)
# FP32 FMA peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (maximum SM clock)
SM_COUNT, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.07
# libtkf.so kernels per step: hit index (count, segment totals, segment scan, bin scan,
# scatter, bin sort), seed estimate, seed fit, seed ordering (key, segment totals, segment
# scan, bin scan, place), build, final fit
KERNELS_PER_STEP = 15
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1e3


def _gen_chunk(args):
    from synth import EventSpec, event_sizes, generate
    seed, e0, e1 = args
    n, f = event_sizes(seed, 640)
    return generate(EventSpec(seed=seed, n_events=e1 - e0, n_tracks=n[e0:e1], noise_frac=f[e0:e1], first_event=e0))


def workload(seed: int, n_events: int, pool=None):
    """The first n_events events of the 640-event batched workload (generated in parallel
    chunks when a process pool is given; the result does not depend on the chunking)."""
    from synth import concat
    if pool is None or n_events < 32:
        return _gen_chunk((seed, 0, n_events))
    step = max(1, n_events // 64)
    chunks = [(seed, e, min(e + step, n_events)) for e in range(0, n_events, step)]
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


# ----------------------------------------------------------------------------- CPU baseline (oracle)
def _oracle_events(chunk):
    """Runs the oracle's whole path (index, seed, seed fit, build, final fit) on a few events,
    each given as (oracle hit records, track hit ids [n, L])."""
    import oracle as O
    from synth import Detector
    det = Detector()
    g = O.make_geom(det)
    L = det.n_layers
    done = 0
    for hits, local in chunk:
        p0, c0 = O.seed_estimate(g, hits, local[:, :3])
        ids = np.full((len(local), L), -1, dtype=np.int32)
        ids[:, :3] = local[:, :3]
        sp, sP, sc2, snh, _ = O.fit(g, hits, p0, c0, ids, 0, 2)
        res = O.build(g, O.hit_index(g, hits), sp, sP, sc2, snh, ids)
        O.fit(g, hits, p0, c0, res.hits[:, 0, :], 0, L - 1)
        done += len(local)
    return done


def oracle_sample(batch, events):
    """Per-event oracle inputs for the listed events of a generated batch."""
    import oracle as O
    out = []
    for e in events:
        h0, h1 = batch.hit_off[e], batch.hit_off[e + 1]
        t0, t1 = batch.trk_off[e], batch.trk_off[e + 1]
        out.append((O.hits_of(batch, slice(h0, h1)), batch.trk_hits[t0:t1] - h0))
    return out


def cpu_baseline(sample, pool, cores):
    """The oracle on the sample's events, one worker process per core; (tracks, wall s)."""
    chunks = [sample[i::cores] for i in range(cores)]
    chunks = [c for c in chunks if c]
    t0 = time.perf_counter()
    done = sum(pool.map(_oracle_events, chunks, chunksize=1))
    return done, time.perf_counter() - t0


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
        times = []
        for _ in range(a.steps):
            tracks, wall = cpu_baseline(sample, pool, cores)
            times.append(wall)
    value = ntr / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched building sample: events %d..%d of the 640-event lognormal batch "
                                   "(%d tracks), oracle FP64 on host cores" % (ev[0], ev[-1], ntr),
                       "events": len(ev), "tracks": ntr},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d events, %d tracks per step" % (len(ev), ntr)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    ap.add_argument("--cpu-tracks", type=int, default=200000, help="oracle CPU-baseline sample (tracks)")
    ap.add_argument("--ref-tracks", type=int, default=60000, help="reference-arm sample per step (tracks)")
    ap.add_argument("--no-cpu", action="store_true")
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
    ctx = tkf.Context(tkf.default_config(seed_order=a.seed_order))
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
    best_tile, tile_ms = ctx.autotune_build(pipe.index(), _T(seeds_t), scratch_out, tiles, repeats=2, stream=stream)
    del scratch_out
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
    t = torch.tensor([ms], device=dev)
    if dist:
        dist.barrier()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    total_tracks = n_tr * world
    value = total_tracks / (ms_max / 1e3)

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

    # ---------------- CPU baseline
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        ev, ntr = sample_events(a.seed, a.cpu_tracks)
        tracks, wall = cpu_baseline(oracle_sample(b, ev), pool, cores)
        cpu = {"value": ntr / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "events %d..%d of the same batch (%d tracks): index, seed, seed fit, build, final fit, "
                         "FP64, one process per core; inputs pickled to the workers inside the timed region"
                         % (ev[0], ev[-1], ntr)}
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
        "roofline": {"kernel": "k_build<6,float,float>", "bound": "alu", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": None, "launch_ms": build_ms, "flop_per_seed": FLOP_PER_SEED,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
        "cpu_baseline": cpu,
        "e2e": {"value": total_tracks / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "plain": plain,
        "autotune": {"tiles": tiles, "build_ms": [round(x, 4) for x in tile_ms], "best": best_tile},
        "gpu_launches": KERNELS_PER_STEP * a.steps,
        "clocks": clocks.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
