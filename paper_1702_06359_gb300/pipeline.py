"""The tracking hot path as one call sequence over a batch of events (Sec. 2: seeding,
building, final fit), on device buffers allocated once for the batch's capacity.

Every step is a call into libtkf.so; this module only owns the buffers and issues the calls
in order on one stream:
  hit index -> three-hit seed estimate -> KF fit of layers 0..2 (the seed) ->
  combinatorial building of layers 3..L-1 -> KF fit of the built hit list from layer 0.
"""
from __future__ import annotations

from . import tkf


class Pipeline:
    def __init__(self, ctx: tkf.Context, n_tracks: int, device="cuda"):
        import torch
        cfg = ctx.cfg
        self.ctx = ctx
        self.L = cfg.n_layers
        self.first = cfg.first_build_layer
        self.prec = cfg.precision
        self.n = n_tracks
        self.init = tkf.DeviceTracks.empty(n_tracks, self.L, self.prec, device)
        self.seeds = tkf.DeviceTracks.empty(n_tracks, self.L, self.prec, device)
        self.built = tkf.DeviceTracks.empty(n_tracks, self.L, self.prec, device)
        self.final = tkf.DeviceTracks.empty(n_tracks, self.L, self.prec, device)
        self.index = None
        self._torch = torch

    def run(self, hits: tkf.DeviceHits, seed_hits, seed_event, stream=None, n_tracks=None, build_events=None):
        """seed_hits: int32 [3, stride] hit ids of each seed on layers 0, 1, 2; seed_event: int32
        [stride] event of each seed.  `build_events` (optional pair of CUDA events) brackets
        the building kernel."""
        n = self.n if n_tracks is None else n_tracks
        for t in (self.init, self.seeds, self.built, self.final):
            t.n = n
        self.seeds.event = seed_event
        ctx = self.ctx
        self.index = ctx.build_hit_index(hits, reuse=self.index, stream=stream)
        ctx.seed_state(hits, seed_hits, self.init, stream=stream)
        ctx.fit(hits, self.init, 0, self.first - 1, self.seeds, stream=stream)
        if build_events is not None:
            build_events[0].record(stream)
        ctx.build_tracks(self.index, self.seeds, self.built, stream=stream)
        if build_events is not None:
            build_events[1].record(stream)
        ctx.fit(hits, self.init, 0, self.L - 1, self.final, hit_idx=self.built.hit_idx, stream=stream)
        return self.final

    # kernels of libtkf.so launched by one run(): hit index (count, layer scan, bin scan,
    # scatter, bin sort), seed estimate, seed fit, build, final fit
    KERNELS_PER_RUN = 9
