"""Python binding of libtkf.so (include/tkf.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module only turns torch
tensors into the C structs of the ABI and checks status codes.  It raises if the library
has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from dataclasses import dataclass

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtkf.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "tkf.h")

MAX_LAYERS = 16
MAX_CAND = 16
FP32, MIXED, FP64 = 0, 1, 2
OK, ERR_INVALID, ERR_CUDA, ERR_NOMEM, ERR_AGAIN, ERR_TIMEOUT, ERR_NOTREADY, ERR_KERNEL, ERR_TOO_LARGE = range(9)
NOALLOC_MAX_HITS, NOALLOC_MAX_BINS, NOALLOC_MAX_SEGMENTS = 1 << 20, 1 << 18, 4096
TRACK_NOREACH, TRACK_SINGULAR, TRACK_LOST = -1, -2, -3


class Config(C.Structure):
    _fields_ = [
        ("n_layers", C.c_int32),
        ("radius", C.c_double * MAX_LAYERS),
        ("x_over_x0", C.c_double * MAX_LAYERS),
        ("bz", C.c_double),
        ("mass", C.c_double),
        ("prior_sigma", C.c_double * 6),
        ("eta_min", C.c_double),
        ("eta_bin_w", C.c_double),
        ("n_eta_bins", C.c_int32),
        ("n_phi_bins", C.c_int32),
        ("chi2_cut", C.c_double),
        ("window_margin", C.c_double),
        ("n_cand", C.c_int32),
        ("first_build_layer", C.c_int32),
        ("precision", C.c_int32),
        ("seeds_per_block", C.c_int32),
        ("seed_order", C.c_int32),
        ("hit_dr", C.c_double),
        ("disk_z", C.c_double * MAX_LAYERS),
    ]


class Hits(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("var_u", C.c_void_p),
                ("var_v", C.c_void_p), ("layer", C.c_void_p), ("event_off", C.c_void_p),
                ("n", C.c_int32), ("n_events", C.c_int32)]


class Tracks(C.Structure):
    _fields_ = [("par", C.c_void_p), ("cov", C.c_void_p), ("chi2", C.c_void_p), ("nhits", C.c_void_p),
                ("hit_idx", C.c_void_p), ("event", C.c_void_p), ("n", C.c_int32), ("stride", C.c_int32)]


class SeedCuts(C.Structure):
    """tkf_seed_cuts: cuts of the seeding from hit triplets (lengths in cm, pt_min in GeV)."""

    _fields_ = [("pt_min", C.c_double), ("kappa_slack", C.c_double), ("z_vertex", C.c_double),
                ("d0_max", C.c_double), ("dz_max", C.c_double), ("conf_rphi", C.c_double), ("conf_z", C.c_double),
                ("confirm", C.c_int32), ("reserved", C.c_int32)]


def default_seed_cuts(**kw) -> SeedCuts:
    c = SeedCuts()
    lib().tkf_default_seed_cuts(C.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(k)
        setattr(c, k, v)
    return c


class HitIndexOut(C.Structure):
    _fields_ = [("hit_xyzi", C.c_void_p), ("hit_var", C.c_void_p), ("bin_sub", C.c_void_p), ("pos_of_hit", C.c_void_p),
                ("bin_off", C.c_void_p), ("var_max", C.c_void_p), ("event_off", C.c_void_p)]


class HitIndexView(C.Structure):
    _fields_ = [("hit_xyzi", C.c_void_p), ("hit_var", C.c_void_p), ("bin_sub", C.c_void_p), ("pos_of_hit", C.c_void_p),
                ("bin_off", C.c_void_p), ("var_max", C.c_void_p), ("event_off", C.c_void_p),
                ("n", C.c_int32), ("n_events", C.c_int32), ("n_layers", C.c_int32), ("n_bins", C.c_int32)]


class ServerOptions(C.Structure):
    _fields_ = [("n_slots", C.c_int32), ("max_batch_events", C.c_int32), ("max_batch_hits", C.c_int32),
                ("max_batch_tracks", C.c_int32), ("queue_bytes", C.c_size_t), ("result_bytes", C.c_size_t)]


class Event(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("var_u", C.c_void_p),
                ("var_v", C.c_void_p), ("layer", C.c_void_p), ("n_hits", C.c_int32), ("seed_hits", C.c_void_p),
                ("n_seeds", C.c_int32), ("borrow", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_tracks", C.c_int32), ("stride", C.c_int32), ("par", C.c_void_p), ("cov", C.c_void_p),
                ("chi2", C.c_void_p), ("nhits", C.c_void_p), ("hit_idx", C.c_void_p), ("t_submit_ns", C.c_int64),
                ("t_start_ns", C.c_int64), ("t_done_ns", C.c_int64), ("gpu_start_ms", C.c_float),
                ("gpu_done_ms", C.c_float), ("gpu_inputs_ms", C.c_float), ("gpu_results_ms", C.c_float)]


class ServerStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("submitted", "rejected", "events_done", "tracks_done", "batches",
                                         "max_batch_events", "result_allocs")]


_lib = None


def declared_functions() -> list[str]:
    """Names of every function declared in include/tkf.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tkf_\w+)\s*\(", text, flags=re.M)))


def lib():
    """Loads libtkf.so (built by paper_1702_06359_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtkf.so is not built (%s); run `python -c 'import __graft_entry__ as g; "
                               "g.build()'` -- there is no CPU fallback" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, i32 = C.c_void_p, C.c_int32
        L.tkf_default_config.argtypes = [C.POINTER(Config)]
        L.tkf_default_config.restype = None
        L.tkf_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
        L.tkf_destroy.argtypes = [vp]
        L.tkf_last_error.argtypes = [vp]
        L.tkf_last_error.restype = C.c_char_p
        L.tkf_status_string.argtypes = [C.c_int]
        L.tkf_status_string.restype = C.c_char_p
        L.tkf_get_config.argtypes = [vp, C.POINTER(Config)]
        L.tkf_build_hit_index.argtypes = [vp, C.POINTER(Hits), C.POINTER(vp), vp]
        L.tkf_hit_index_free.argtypes = [vp]
        L.tkf_hit_index_get_view.argtypes = [vp, C.POINTER(HitIndexView)]
        L.tkf_seed_state.argtypes = [vp, C.POINTER(Hits), vp, C.POINTER(Tracks), vp]
        L.tkf_fit.argtypes = [vp, C.POINTER(Hits), C.POINTER(Tracks), vp, i32, i32, C.POINTER(Tracks), vp]
        L.tkf_fit_continue.argtypes = [vp, C.POINTER(Hits), C.POINTER(Tracks), vp, i32, i32, C.POINTER(Tracks), vp]
        L.tkf_seed_fit.argtypes = [vp, C.POINTER(Hits), vp, i32, C.POINTER(Tracks), vp]
        L.tkf_fit_backward.argtypes = [vp, C.POINTER(Hits), C.POINTER(Tracks), vp, i32, i32, C.c_double,
                                       C.POINTER(Tracks), vp]
        L.tkf_build_tracks.argtypes = [vp, vp, C.POINTER(Tracks), C.POINTER(Tracks), C.POINTER(Tracks), vp, vp]
        L.tkf_sync_status.argtypes = [vp, vp]
        L.tkf_pipeline_create.argtypes = [vp, i32, i32, i32, i32, C.POINTER(vp)]
        L.tkf_pipeline_destroy.argtypes = [vp]
        L.tkf_pipeline_run.argtypes = [vp, C.POINTER(Hits), vp, vp, i32, vp]
        L.tkf_pipeline_outputs.argtypes = [vp, C.POINTER(Tracks), C.POINTER(Tracks), C.POINTER(Tracks)]
        L.tkf_pipeline_captures.argtypes = [vp]
        L.tkf_pipeline_set_backward.argtypes = [vp, C.c_double]
        L.tkf_pipeline_backward_outputs.argtypes = [vp, C.POINTER(Tracks)]
        L.tkf_probe_alu.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.tkf_pipeline_index.argtypes = [vp]
        L.tkf_pipeline_build_ms.argtypes = [vp, C.POINTER(C.c_float)]
        L.tkf_autotune_build.argtypes = [vp, vp, C.POINTER(Tracks), C.POINTER(Tracks), vp, i32, i32, vp, vp, vp]
        L.tkf_server_default_options.argtypes = [C.POINTER(ServerOptions)]
        L.tkf_server_create.argtypes = [C.POINTER(Config), C.POINTER(ServerOptions), C.POINTER(vp)]
        L.tkf_server_destroy.argtypes = [vp]
        L.tkf_submit_event.argtypes = [vp, C.POINTER(Event), C.POINTER(C.c_uint64)]
        L.tkf_poll.argtypes = [vp, C.c_uint64, C.POINTER(Result), C.c_int64]
        L.tkf_release.argtypes = [vp, C.c_uint64]
        L.tkf_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.tkf_submit_events.argtypes = [vp, C.POINTER(Event), i32, C.POINTER(C.c_uint64), C.POINTER(i32)]
        L.tkf_wait_all.argtypes = [vp, C.POINTER(C.c_uint64), i32, C.POINTER(Result), C.c_int64]
        L.tkf_release_many.argtypes = [vp, C.POINTER(C.c_uint64), i32]
        L.tkf_default_seed_cuts.argtypes = [C.POINTER(SeedCuts)]
        L.tkf_default_seed_cuts.restype = None
        L.tkf_find_seeds.argtypes = [vp, vp, C.POINTER(SeedCuts), i32, vp, vp, vp, vp, vp]
        L.tkf_build_hit_index_noalloc.argtypes = [C.POINTER(Config), C.POINTER(Hits), C.POINTER(HitIndexOut), vp]
        for name in declared_functions():
            if name not in ("tkf_last_error", "tkf_status_string", "tkf_default_config", "tkf_pipeline_index",
                            "tkf_server_default_options", "tkf_default_seed_cuts"):
                getattr(L, name).restype = C.c_int
        L.tkf_pipeline_index.restype = vp
        L.tkf_server_default_options.restype = None
        _lib = L
    return _lib


class TkfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (lib().tkf_status_string(code).decode(), code, msg))
        self.code = code


def default_config(**kw) -> Config:
    cfg = Config()
    lib().tkf_default_config(C.byref(cfg))
    for k, v in kw.items():
        if k in ("radius", "x_over_x0", "prior_sigma", "disk_z"):
            arr = getattr(cfg, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(cfg, k, v)
    return cfg


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


@dataclass
class DeviceHits:
    """Hits of a batch of events as torch CUDA tensors (float32 x, y, z, var_u, var_v; int32
    layer; int32 event_off with n_events + 1 entries)."""

    x: object
    y: object
    z: object
    var_u: object
    var_v: object
    layer: object
    event_off: object

    def struct(self) -> Hits:
        h = Hits()
        h.x, h.y, h.z = self.x.data_ptr(), self.y.data_ptr(), self.z.data_ptr()
        h.var_u, h.var_v = self.var_u.data_ptr(), self.var_v.data_ptr()
        h.layer, h.event_off = self.layer.data_ptr(), self.event_off.data_ptr()
        h.n = self.x.numel()
        h.n_events = self.event_off.numel() - 1
        return h


@dataclass
class DeviceTracks:
    """Track SoA planes as torch tensors: par [6, stride], cov [21, stride], chi2 [stride],
    nhits [stride] int32, hit_idx [n_layers, stride] int32, event [stride] int32."""

    par: object
    cov: object
    chi2: object
    nhits: object
    hit_idx: object = None
    event: object = None
    n: int = -1

    @staticmethod
    def empty(n, n_layers, precision=FP32, device="cuda", stride=None):
        import torch
        stride = n if stride is None else stride
        dt = torch.float64 if precision == FP64 else torch.float32
        return DeviceTracks(
            par=torch.zeros((6, stride), dtype=dt, device=device),
            cov=torch.zeros((21, stride), dtype=dt, device=device),
            chi2=torch.zeros(stride, dtype=dt, device=device),
            nhits=torch.zeros(stride, dtype=torch.int32, device=device),
            hit_idx=torch.full((n_layers, stride), -1, dtype=torch.int32, device=device),
            event=torch.zeros(stride, dtype=torch.int32, device=device),
            n=n,
        )

    @property
    def stride(self):
        return self.par.shape[1]

    def struct(self) -> Tracks:
        t = Tracks()
        t.par, t.cov, t.chi2 = self.par.data_ptr(), self.cov.data_ptr(), self.chi2.data_ptr()
        t.nhits = self.nhits.data_ptr()
        t.hit_idx = self.hit_idx.data_ptr() if self.hit_idx is not None else None
        t.event = self.event.data_ptr() if self.event is not None else None
        t.stride = self.stride
        t.n = self.stride if self.n < 0 else self.n
        return t


class HitIndex:
    def __init__(self, ctx, handle):
        self.ctx, self.handle = ctx, handle

    def view(self) -> HitIndexView:
        v = HitIndexView()
        self.ctx._check(lib().tkf_hit_index_get_view(self.handle, C.byref(v)))
        return v

    def free(self):
        if self.handle:
            lib().tkf_hit_index_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """A tkf_ctx on the current CUDA device."""

    def __init__(self, cfg: Config | None = None, **kw):
        self.cfg = cfg if cfg is not None else default_config(**kw)
        h = C.c_void_p()
        code = lib().tkf_create(C.byref(self.cfg), C.byref(h))
        if code != OK:
            raise TkfError(code, "tkf_create")
        self.handle = h

    def _check(self, code):
        if code != OK:
            raise TkfError(code, lib().tkf_last_error(self.handle).decode())

    def config(self) -> Config:
        c = Config()
        self._check(lib().tkf_get_config(self.handle, C.byref(c)))
        return c

    def build_hit_index(self, hits: DeviceHits, reuse: HitIndex | None = None, stream=None) -> HitIndex:
        hs = hits.struct()
        h = C.c_void_p(reuse.handle if reuse is not None else None)
        self._check(lib().tkf_build_hit_index(self.handle, C.byref(hs), C.byref(h), _stream(stream)))
        if reuse is not None:
            reuse.handle = h.value
            return reuse
        return HitIndex(self, h.value)

    def seed_state(self, hits: DeviceHits, seed_hits, out: DeviceTracks, stream=None):
        hs, ts = hits.struct(), out.struct()
        self._check(lib().tkf_seed_state(self.handle, C.byref(hs), _ptr(seed_hits), C.byref(ts), _stream(stream)))

    def fit(self, hits: DeviceHits, init: DeviceTracks, first, last, out: DeviceTracks, hit_idx=None, stream=None,
            continue_fit=False):
        """tkf_fit; continue_fit: tkf_fit_continue (init lies on layer first - 1)."""
        hs, ti, to = hits.struct(), init.struct(), out.struct()
        fn = lib().tkf_fit_continue if continue_fit else lib().tkf_fit
        self._check(fn(self.handle, C.byref(hs), C.byref(ti), _ptr(hit_idx), int(first), int(last), C.byref(to),
                       _stream(stream)))

    def fit_backward(self, hits: DeviceHits, init: DeviceTracks, last, first, out: DeviceTracks, cov_scale=1e4,
                     hit_idx=None, stream=None):
        """tkf_fit_backward: the inward pass from layer `last` down to `first`."""
        hs, ti, to = hits.struct(), init.struct(), out.struct()
        self._check(lib().tkf_fit_backward(self.handle, C.byref(hs), C.byref(ti), _ptr(hit_idx), int(last), int(first),
                                           float(cov_scale), C.byref(to), _stream(stream)))

    def seed_fit(self, hits: DeviceHits, seed_hits, last, out: DeviceTracks, stream=None):
        hs, to = hits.struct(), out.struct()
        self._check(lib().tkf_seed_fit(self.handle, C.byref(hs), _ptr(seed_hits), int(last), C.byref(to),
                                       _stream(stream)))

    def find_seeds(self, index: HitIndex, cuts: SeedCuts, max_seeds, seed_hits, seed_event, n_found, seed_score=None,
                   stream=None):
        """tkf_find_seeds into caller-owned device tensors: seed_hits int32 [3][max_seeds],
        seed_event int32 [max_seeds], n_found int32 [1], seed_score float [max_seeds] or None."""
        self._check(lib().tkf_find_seeds(self.handle, index.handle, C.byref(cuts), int(max_seeds), _ptr(seed_hits),
                                         _ptr(seed_event), _ptr(seed_score), _ptr(n_found), _stream(stream)))

    def build_tracks(self, index: HitIndex, seeds: DeviceTracks, out: DeviceTracks, out_all: DeviceTracks = None,
                     n_cand_out=None, stream=None):
        ss, so = seeds.struct(), out.struct()
        sa = C.byref(out_all.struct()) if out_all is not None else None
        self._check(lib().tkf_build_tracks(self.handle, index.handle, C.byref(ss), C.byref(so), sa, _ptr(n_cand_out),
                                           _stream(stream)))

    def autotune_build(self, index: HitIndex, seeds: DeviceTracks, out: DeviceTracks, tiles, repeats=3, stream=None):
        """Times the building kernel for each work-tile size; keeps and returns the fastest and
        the per-size milliseconds."""
        arr = (C.c_int32 * len(tiles))(*tiles)
        ms = (C.c_float * len(tiles))()
        best = C.c_int32()
        ss, so = seeds.struct(), out.struct()
        self._check(lib().tkf_autotune_build(self.handle, index.handle, C.byref(ss), C.byref(so), arr, len(tiles),
                                             int(repeats), ms, C.byref(best), _stream(stream)))
        return best.value, list(ms)

    def sync_status(self, stream=None):
        self._check(lib().tkf_sync_status(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            lib().tkf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_alu(stream=None) -> dict:
    """tkf_probe_alu: measured FP32 / FP64 multiply-add throughput (TFLOP/s) and special-function
    throughput (tera-ops/s) of the current device."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    rc = lib().tkf_probe_alu(_stream(stream), C.byref(a), C.byref(b), C.byref(c))
    if rc:
        raise TkfError(rc, "tkf_probe_alu failed")
    return {"fp32_tflops": a.value, "fp64_tflops": b.value, "sfu_tops": c.value}


def build_hit_index_noalloc(cfg: Config, hits: DeviceHits, out: dict, stream=None):
    """tkf_build_hit_index_noalloc into caller-owned tensors `out` (keys hit_xyzi [n, 4] f32,
    hit_var [n, 2] f32, bin_sub [E*L*bins, 4] i32, pos_of_hit [n] i32, bin_off [E*L*bins + 1] i32, var_max [E*L, 2] f32,
    event_off [E + 1] i32); returns the status code."""
    o = HitIndexOut()
    for k in ("hit_xyzi", "hit_var", "bin_sub", "pos_of_hit", "bin_off", "var_max", "event_off"):
        setattr(o, k, out[k].data_ptr())
    hs = hits.struct()
    return lib().tkf_build_hit_index_noalloc(C.byref(cfg), C.byref(hs), C.byref(o), _stream(stream))


class DevicePipeline:
    """tkf_pipeline: buffers for batches up to the given sizes; run() issues the whole hot path
    (replayed from a CUDA graph when use_graph)."""

    def __init__(self, ctx: Context, max_hits, max_events, max_tracks, use_graph=True):
        self.ctx = ctx
        h = C.c_void_p()
        ctx._check(lib().tkf_pipeline_create(ctx.handle, int(max_hits), int(max_events), int(max_tracks),
                                             int(bool(use_graph)), C.byref(h)))
        self.handle = h
        self.max_tracks = int(max_tracks)

    def run(self, hits: DeviceHits, seed_hits, seed_event, n_tracks, stream=None):
        hs = hits.struct()
        self.ctx._check(lib().tkf_pipeline_run(self.handle, C.byref(hs), _ptr(seed_hits), _ptr(seed_event),
                                               int(n_tracks), _stream(stream)))

    def outputs(self):
        """(seeds, built, fitted) as tkf_tracks structs (device pointers owned by the pipeline)."""
        sd, b, f = Tracks(), Tracks(), Tracks()
        self.ctx._check(lib().tkf_pipeline_outputs(self.handle, C.byref(sd), C.byref(b), C.byref(f)))
        return sd, b, f

    def set_backward(self, cov_scale=1e4):
        """tkf_pipeline_set_backward: every following run ends with the backward pass (0: off)."""
        self.ctx._check(lib().tkf_pipeline_set_backward(self.handle, float(cov_scale)))

    def backward_outputs(self):
        """The backward pass's states on layer 0 of the last run, as a tkf_tracks struct."""
        t = Tracks()
        self.ctx._check(lib().tkf_pipeline_backward_outputs(self.handle, C.byref(t)))
        return t

    def captures(self):
        return lib().tkf_pipeline_captures(self.handle)

    def build_ms(self):
        """Duration of the building kernel in the last run (CUDA events inside the graph)."""
        ms = C.c_float()
        self.ctx._check(lib().tkf_pipeline_build_ms(self.handle, C.byref(ms)))
        return ms.value

    def index(self) -> "HitIndex":
        """The pipeline's hit index (not owned: do not free)."""
        h = HitIndex(self.ctx, lib().tkf_pipeline_index(self.handle))
        h.free = lambda: None
        return h

    def close(self):
        if getattr(self, "handle", None):
            lib().tkf_pipeline_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tracks_tensors(t: Tracks, n_layers, precision=FP32):
    """torch views (no copy) of a tkf_tracks struct's planes: par [6, stride], cov [21, stride],
    chi2, nhits, hit_idx [n_layers, stride]."""
    import torch
    dt = torch.float64 if precision == FP64 else torch.float32
    code = {torch.float32: "<f4", torch.float64: "<f8", torch.int32: "<i4"}

    def wrap(ptr, shape, dtype):
        class _W:
            __cuda_array_interface__ = {"shape": shape, "typestr": code[dtype], "data": (ptr, False), "version": 3}
        return torch.as_tensor(_W(), device="cuda")
    s = t.stride
    return dict(par=wrap(t.par, (6, s), dt), cov=wrap(t.cov, (21, s), dt), chi2=wrap(t.chi2, (s,), dt),
                nhits=wrap(t.nhits, (s,), torch.int32), hit_idx=wrap(t.hit_idx, (n_layers, s), torch.int32))


def server_options(**kw) -> ServerOptions:
    o = ServerOptions()
    lib().tkf_server_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class HostEvent:
    """One event's host arrays, kept alive while its tkf_event struct is used: float32 x, y, z,
    var_u, var_v; int32 layer; int32 seed_hits [3, n_seeds] (event-local).  borrow=True lends
    them to the server (held in pinned memory here) instead of having them copied."""

    def __init__(self, x, y, z, var_u, var_v, layer, seed_hits, borrow=False):
        import numpy as np
        c = lambda a, dt: np.ascontiguousarray(a, dtype=dt)
        self.arrays = [c(x, np.float32), c(y, np.float32), c(z, np.float32), c(var_u, np.float32),
                       c(var_v, np.float32), c(layer, np.int32), c(seed_hits, np.int32)]
        ptrs = [a.ctypes.data for a in self.arrays]
        if borrow:
            import torch
            self.pinned = [torch.from_numpy(a).pin_memory() for a in self.arrays]
            ptrs = [t.data_ptr() for t in self.pinned]
        a = self.arrays
        self.struct = Event(ptrs[0], ptrs[1], ptrs[2], ptrs[3], ptrs[4], ptrs[5], len(a[0]), ptrs[6], a[6].shape[1],
                            int(bool(borrow)))


class Server:
    """tkf_server: submit(event) -> ticket; poll(ticket) -> dict of numpy copies; release."""

    def __init__(self, cfg: Config = None, **opts):
        self.cfg = cfg if cfg is not None else default_config()
        self.opt = server_options(**opts)
        h = C.c_void_p()
        code = lib().tkf_server_create(C.byref(self.cfg), C.byref(self.opt), C.byref(h))
        if code != OK:
            raise TkfError(code, "tkf_server_create")
        self.handle = h

    def submit(self, ev):
        """Submits a HostEvent or a raw Event struct; returns (status, ticket), status ERR_AGAIN
        when the queue is full."""
        t = C.c_uint64()
        code = lib().tkf_submit_event(self.handle, C.byref(ev.struct if isinstance(ev, HostEvent) else ev),
                                      C.byref(t))
        return code, t.value

    try_submit = submit

    def submit_many(self, events):
        """Submits a ctypes array of Event structs; returns (status, tickets accepted)."""
        n = len(events)
        tickets = (C.c_uint64 * n)()
        acc = C.c_int32()
        code = lib().tkf_submit_events(self.handle, events, n, tickets, C.byref(acc))
        return code, list(tickets[:acc.value])

    def wait_all(self, tickets, timeout_us=60_000_000):
        """Waits for every ticket; returns (status, ctypes array of Result structs)."""
        n = len(tickets)
        t = (C.c_uint64 * n)(*tickets)
        res = (Result * n)()
        code = lib().tkf_wait_all(self.handle, t, n, res, int(timeout_us))
        return code, res

    def release_many(self, tickets):
        n = len(tickets)
        return lib().tkf_release_many(self.handle, (C.c_uint64 * n)(*tickets), n)

    def submit_struct(self, ev, retry_us=20):
        """Submits, waiting while the queue is full; returns the ticket, raises on errors."""
        import time
        while True:
            code, t = self.submit(ev)
            if code == OK:
                return t
            if code != ERR_AGAIN:
                raise TkfError(code, "tkf_submit_event")
            time.sleep(retry_us * 1e-6)

    def poll(self, ticket, timeout_us=0, copy=True):
        """(status, result): result holds numpy copies (copy=True) or the raw Result struct."""
        import numpy as np
        r = Result()
        code = lib().tkf_poll(self.handle, int(ticket), C.byref(r), int(timeout_us))
        if code != OK or not copy:
            return code, r
        n, L, st = r.n_tracks, self.cfg.n_layers, r.stride

        def arr(ptr, rows, ct):
            if not n:
                return np.zeros((rows, 0) if rows else (0,), dtype=np.float32 if ct is C.c_float else np.int32)
            full = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ct)), shape=((rows - 1) * st + n,) if rows else (n,))
            if not rows:
                return full.copy()
            return np.stack([full[k * st:k * st + n] for k in range(rows)])
        return code, dict(status=r.status, n_tracks=n, par=arr(r.par, 6, C.c_float),
                          cov=arr(r.cov, 21, C.c_float), chi2=arr(r.chi2, 0, C.c_float),
                          nhits=arr(r.nhits, 0, C.c_int32), hit_idx=arr(r.hit_idx, L, C.c_int32),
                          t_submit_ns=r.t_submit_ns, t_start_ns=r.t_start_ns, t_done_ns=r.t_done_ns,
                          gpu_start_ms=r.gpu_start_ms, gpu_done_ms=r.gpu_done_ms)

    def release(self, ticket):
        return lib().tkf_release(self.handle, int(ticket))

    def stats(self) -> dict:
        st = ServerStats()
        lib().tkf_server_get_stats(self.handle, C.byref(st))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().tkf_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
