"""tkf_build_hit_index_noalloc: the hit index for callers that cannot allocate device memory
(code running inside another framework's memory pool, with all device memory reserved up
front, or on a time-critical path where an allocation could block or fail).  It must give
exactly what tkf_build_hit_index gives, call after call, while using only the library's
fixed scratch array; inputs beyond that array's capacity are refused up front.

This file is collected last on purpose, so a run that stops at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_1702_06359_gb300 import tkf


def test_noalloc_rejects_inputs_beyond_its_capacity():
    from paper_1702_06359_gb300 import build
    build.build()
    cfg = tkf.default_config()
    fake = 256  # never dereferenced: the size check comes before any device work
    h = tkf.Hits(fake, fake, fake, fake, fake, fake, fake, tkf.NOALLOC_MAX_HITS + 1, 1)
    o = tkf.HitIndexOut(fake, fake, fake, fake, fake, fake, fake)
    L = tkf.lib()
    assert L.tkf_build_hit_index_noalloc(C.byref(cfg), C.byref(h), C.byref(o), None) == tkf.ERR_TOO_LARGE
    # 11 events x 10 layers x 2520 bins = 277 200 bins > 262 144
    h.n, h.n_events = 1000, 11
    assert L.tkf_build_hit_index_noalloc(C.byref(cfg), C.byref(h), C.byref(o), None) == tkf.ERR_TOO_LARGE
    assert L.tkf_build_hit_index_noalloc(None, C.byref(h), C.byref(o), None) == tkf.ERR_INVALID
    assert L.tkf_status_string(tkf.ERR_TOO_LARGE).startswith(b"input exceeds")


@pytest.mark.gpu
@pytest.mark.parametrize("branch", ["multi_launch", "block_per_event"])
def test_noalloc_index_equals_allocating_index_on_consecutive_calls(branch):
    """Two calls in a row against tkf_build_hit_index, bit for bit.  "multi_launch": a few
    events on the ten-layer barrel (fewer events than twice the SMs: the index is built by
    kernels that spread one event over the GPU).  "block_per_event": 320 events (more than twice
    the SMs) on a four-layer barrel with 8 x 8 bins (1 280 segments, 81 920 bins, inside the fixed
    capacity), which takes the one-block-per-event kernels."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from _gpu import device_hits
    from synth import Detector, EventSpec, generate

    if branch == "multi_launch":
        det = Detector()
        cfg = tkf.default_config()
        batches = [generate(EventSpec(seed=51, n_events=3, n_tracks=[2000, 0, 1500], noise_frac=0.3), det),
                   generate(EventSpec(seed=52, n_events=2, n_tracks=[800, 3000], noise_frac=0.5), det)]
    else:
        det = Detector(radii=(4.0, 8.0, 12.0, 16.0), x_over_x0=(0.03,) * 4)
        cfg = tkf.default_config(n_layers=4, radius=det.radii, x_over_x0=det.x_over_x0, n_eta_bins=8,
                                 n_phi_bins=8, eta_min=-1.6, eta_bin_w=0.4)
        rng = np.random.default_rng(53)
        batches = [generate(EventSpec(seed=53, n_events=320, n_tracks=rng.integers(0, 400, 320).tolist(),
                                      noise_frac=0.3), det),
                   generate(EventSpec(seed=54, n_events=320, n_tracks=rng.integers(0, 300, 320).tolist(),
                                      noise_frac=0.5), det)]
        props = torch.cuda.get_device_properties(0)
        assert all(b.n_events >= 2 * props.multi_processor_count for b in batches)
        assert 320 * 4 <= tkf.NOALLOC_MAX_SEGMENTS and 320 * 4 * 64 <= tkf.NOALLOC_MAX_BINS
    ctx = tkf.Context(cfg)
    L, NB = cfg.n_layers, cfg.n_eta_bins * cfg.n_phi_bins

    def raw(ptr, count, dtype):
        class _Wrap:
            __cuda_array_interface__ = {"shape": (count,), "typestr": {torch.float32: "<f4", torch.int32: "<i4"}[dtype],
                                        "data": (ptr, False), "version": 3}
        return torch.as_tensor(_Wrap(), device="cuda").clone()

    for call, b in enumerate(batches):
        dh = device_hits(b)
        n, E = b.n_hits, b.n_events
        out = {"hit_xyzi": torch.full((n, 4), -7.0, device="cuda"), "hit_var": torch.full((n, 2), -7.0, device="cuda"),
               "bin_sub": torch.full((E * L * NB, 4), -7, dtype=torch.int32, device="cuda"),
               "pos_of_hit": torch.full((n,), -7, dtype=torch.int32, device="cuda"),
               "bin_off": torch.full((E * L * NB + 1,), -7, dtype=torch.int32, device="cuda"),
               "var_max": torch.full((E * L, 2), -7.0, device="cuda"),
               "event_off": torch.full((E + 1,), -7, dtype=torch.int32, device="cuda")}
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        assert tkf.build_hit_index_noalloc(cfg, dh, out) == tkf.OK
        torch.cuda.synchronize()
        if call > 0:  # the first call may load the library's device code; later calls take nothing
            assert torch.cuda.mem_get_info()[0] >= free_before
        ref = ctx.build_hit_index(dh)
        torch.cuda.synchronize()
        ctx.sync_status()
        v = ref.view()
        assert torch.equal(out["hit_xyzi"].view(-1), raw(v.hit_xyzi, n * 4, torch.float32))
        assert torch.equal(out["hit_var"].view(-1), raw(v.hit_var, n * 2, torch.float32))
        assert torch.equal(out["bin_sub"].view(-1), raw(v.bin_sub, E * L * NB * 4, torch.int32))
        assert torch.equal(out["pos_of_hit"], raw(v.pos_of_hit, n, torch.int32))
        assert torch.equal(out["bin_off"], raw(v.bin_off, E * L * NB + 1, torch.int32))
        assert torch.equal(out["var_max"].view(-1), raw(v.var_max, E * L * 2, torch.float32))
        assert torch.equal(out["event_off"], raw(v.event_off, E + 1, torch.int32))
        assert int(out["bin_off"][-1]) == n
        ref.free()
    ctx.close()
