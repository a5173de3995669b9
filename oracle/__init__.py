"""ORACLE -- test infrastructure only.

ctypes front end of the plain FP64 C oracle in `tkf_oracle.c` (Kalman-filter track fit and
combinatorial track building, restated from the paper in textbook form).  Only the test
suite, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may import this
package; the CUDA library and its binding never do.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tkf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")
MAX_LAYERS = 16


def compile_library(force: bool = False) -> str:
    """Compile the C oracle with gcc (seconds).  Returns the library path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "tkf_oracle.h")))
    if force or stale:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Geom(C.Structure):
    _fields_ = [
        ("n_layers", C.c_int),
        ("radius", C.c_double * MAX_LAYERS),
        ("bz", C.c_double),
        ("x_over_x0", C.c_double * MAX_LAYERS),
        ("mass", C.c_double),
        ("prior_sigma", C.c_double * 6),
        ("eta_min", C.c_double),
        ("eta_bin_w", C.c_double),
        ("n_eta_bins", C.c_int),
        ("n_phi_bins", C.c_int),
        ("chi2_cut", C.c_double),
        ("window_margin", C.c_double),
        ("tie_tol", C.c_double),
        ("n_cand", C.c_int),
        ("brute_force", C.c_int),
        ("first_build_layer", C.c_int),
        ("hit_dr", C.c_double),
        ("disk_z", C.c_double * MAX_LAYERS),
    ]


HIT_DTYPE = np.dtype([("x", "f8"), ("y", "f8"), ("z", "f8"), ("var_u", "f8"), ("var_v", "f8"),
                      ("layer", "i4"), ("disk", "i4")], align=True)


class Hit(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z", C.c_double), ("var_u", C.c_double),
                ("var_v", C.c_double), ("layer", C.c_int), ("disk", C.c_int)]


assert C.sizeof(Hit) == HIT_DTYPE.itemsize


class Event(C.Structure):
    _fields_ = [("n_hits", C.c_int), ("hits", C.c_void_p), ("order", C.c_void_p), ("bin_off", C.c_void_p),
                ("var_u_max", C.c_double * MAX_LAYERS), ("var_v_max", C.c_double * MAX_LAYERS)]


class Stats(C.Structure):
    _fields_ = [("n_prop", C.c_longlong), ("n_hits_examined", C.c_longlong), ("n_updates", C.c_longlong),
                ("n_kept", C.c_longlong), ("n_steps", C.c_longlong)]


@dataclass
class Settings:
    """Method parameters; defaults are the plain-building workload (20 x 5000 tracks)."""

    eta_min: float = -2.0
    eta_bin_w: float = 0.1
    n_eta_bins: int = 40
    n_phi_bins: int = 63
    chi2_cut: float = 30.0
    window_margin: float = 1e-3
    tie_tol: float = 1e-3
    n_cand: int = 6
    brute_force: int = 0  # 1: every hit of the layer; 2: also no residual window (hit_dr > 0)
    first_build_layer: int = 3
    prior_sigma: tuple = (0.1, 0.1, 1.0, 0.5, 0.05, 0.05)


_lib = None


def lib():
    """The committed oracle, compiled on first use; ORC_LIBRARY names another compiled copy
    instead (the planted-mistake tests run the pins against copies with a mistake)."""
    global _lib
    if _lib is None:
        _lib = load_library(os.environ.get("ORC_LIBRARY") or compile_library())
    return _lib


def load_library(path: str):
    """The oracle's functions from a compiled library at `path` (lib() loads the committed one;
    the tests also load copies with planted mistakes)."""
    L = C.CDLL(path)
    dp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p
    L.orc_propagate.argtypes = [C.POINTER(Geom), dp, C.c_double, dp, dp]
    L.orc_propagate_plane.argtypes = [C.POINTER(Geom), dp, C.c_double, dp, dp]
    L.orc_hit_eta_bin.argtypes = [C.POINTER(Geom), C.POINTER(Hit)]
    L.orc_scatter.argtypes = [C.POINTER(Geom), C.c_int, dp, dp]
    L.orc_scatter.restype = None
    L.orc_chi2.argtypes = [dp, dp, C.POINTER(Hit)]
    L.orc_chi2.restype = C.c_double
    L.orc_update.argtypes = [dp, dp, C.POINTER(Hit), dp]
    L.orc_seed_batch.argtypes = [C.POINTER(Geom), vp, C.c_int, ip, dp, dp]
    L.orc_fit_batch.argtypes = [C.POINTER(Geom), vp, C.c_int, dp, dp, ip, C.c_int, C.c_int, dp, dp, dp, ip, ip]
    L.orc_fit_backward_batch.argtypes = [C.POINTER(Geom), vp, C.c_int, dp, dp, C.c_double, ip, C.c_int, C.c_int,
                                         dp, dp, dp, ip, ip]
    L.orc_eta_bin.argtypes = [C.POINTER(Geom), C.c_int, C.c_double]
    L.orc_phi_bin.argtypes = [C.POINTER(Geom), C.c_double]
    L.orc_hit_index.argtypes = [C.POINTER(Geom), C.c_int, vp, ip, ip, ip]
    L.orc_build_batch.argtypes = [C.POINTER(Geom), C.POINTER(Event), C.c_int, dp, dp, dp, ip, ip, C.c_int,
                                  ip, dp, dp, dp, ip, ip, ip, C.POINTER(Stats)]
    L.orc_seed_kappa_max.argtypes = [C.POINTER(Geom), C.POINTER(SeedCuts)]
    L.orc_seed_kappa_max.restype = C.c_double
    L.orc_seed_eval.argtypes = [C.POINTER(Geom), C.POINTER(SeedCuts), C.POINTER(Hit), C.POINTER(Hit),
                                C.POINTER(Hit), C.POINTER(Hit), C.POINTER(SeedQuant)]
    L.orc_find_seeds.argtypes = [C.POINTER(Geom), C.POINTER(SeedCuts), C.c_int, vp, vp]
    L.orc_find_seeds_of.argtypes = [C.POINTER(Geom), C.POINTER(SeedCuts), C.c_int, vp, C.c_int, ip, vp]
    return L


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def make_geom(det, st: Settings = Settings()) -> Geom:
    g = Geom()
    g.n_layers = det.n_layers
    for l in range(det.n_layers):
        g.radius[l] = det.radii[l]
        g.x_over_x0[l] = det.x_over_x0[l]
    g.bz = det.bz
    g.mass = det.mass
    for i in range(6):
        g.prior_sigma[i] = st.prior_sigma[i]
    g.eta_min, g.eta_bin_w = st.eta_min, st.eta_bin_w
    g.n_eta_bins, g.n_phi_bins = st.n_eta_bins, st.n_phi_bins
    g.chi2_cut, g.window_margin, g.tie_tol = st.chi2_cut, st.window_margin, st.tie_tol
    g.n_cand = st.n_cand
    g.brute_force = int(st.brute_force)
    g.first_build_layer = st.first_build_layer
    g.hit_dr = 0.5 * getattr(det, "module_dr", 0.0)
    for l in range(det.n_layers):
        g.disk_z[l] = det.disk_z[l] if getattr(det, "disk_z", ()) else 0.0
    return g


def hits_of(batch, sl=slice(None), exact=False) -> np.ndarray:
    """Oracle hit records for a slice of the batch's hits: FP64 copies of the FP32 inputs, or
    (exact=True) the generator's unrounded FP64 positions."""
    h = np.zeros(len(batch.x[sl]), dtype=HIT_DTYPE)
    if exact:
        xyz = batch.extras["xyz64"][sl]
        h["x"], h["y"], h["z"] = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    else:
        h["x"], h["y"], h["z"] = batch.x[sl], batch.y[sl], batch.z[sl]
    h["var_u"], h["var_v"] = batch.var_u[sl], batch.var_v[sl]
    h["layer"] = batch.layer[sl]
    dz = getattr(batch.detector, "disk_z", ())
    if dz:
        h["disk"] = (np.asarray(dz) > 0.0)[h["layer"]].astype(np.int32)
    return h


def make_hit(x, y, z, var_u, var_v, layer=0, disk=0) -> Hit:
    return Hit(float(x), float(y), float(z), float(var_u), float(var_v), int(layer), int(disk))


def propagate_plane(g: Geom, p, Zp):
    """Propagation to the plane z = Zp (an endcap disk): (status, state, Jacobian)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(6)
    J = np.zeros(36)
    st = lib().orc_propagate_plane(C.byref(g), _d(p), float(Zp), _d(out), _d(J))
    return st, out, J.reshape(6, 6)


def propagate(g: Geom, p, R):
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(6)
    J = np.zeros(36)
    st = lib().orc_propagate(C.byref(g), _d(p), float(R), _d(out), _d(J))
    return st, out, J.reshape(6, 6)


def scatter(g: Geom, layer, p, P):
    p = np.ascontiguousarray(p, dtype=np.float64)
    P = np.array(P, dtype=np.float64).reshape(36)
    lib().orc_scatter(C.byref(g), int(layer), _d(p), _d(P))
    return P.reshape(6, 6)


def chi2(p, P, hit: Hit):
    p = np.ascontiguousarray(p, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(36)
    return lib().orc_chi2(_d(p), _d(P), C.byref(hit))


def update(p, P, hit: Hit):
    p = np.array(p, dtype=np.float64)
    P = np.array(P, dtype=np.float64).reshape(36)
    c2 = C.c_double(0.0)
    st = lib().orc_update(_d(p), _d(P), C.byref(hit), C.byref(c2))
    return st, p, P.reshape(6, 6), c2.value


def seed_estimate(g: Geom, hits: np.ndarray, seed_hits: np.ndarray):
    seed_hits = np.ascontiguousarray(seed_hits, dtype=np.int32)
    n = len(seed_hits)
    par = np.zeros((n, 6))
    cov = np.zeros((n, 36))
    st = lib().orc_seed_batch(C.byref(g), hits.ctypes.data, n, _i(seed_hits), _d(par), _d(cov))
    assert st == 0
    return par, cov.reshape(n, 6, 6)


def fit(g: Geom, hits: np.ndarray, par, cov, hit_ids, first, last):
    par = np.ascontiguousarray(par, dtype=np.float64)
    n = len(par)
    cov = np.ascontiguousarray(cov, dtype=np.float64).reshape(n, 36)
    hit_ids = np.ascontiguousarray(hit_ids, dtype=np.int32)
    assert hit_ids.shape == (n, g.n_layers)
    po, co = np.zeros((n, 6)), np.zeros((n, 36))
    c2 = np.zeros(n)
    nh = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    lib().orc_fit_batch(C.byref(g), hits.ctypes.data, n, _d(par), _d(cov), _i(hit_ids), int(first), int(last),
                        _d(po), _d(co), _d(c2), _i(nh), _i(status))
    return po, co.reshape(n, 6, 6), c2, nh, status


def fit_backward(g: Geom, hits: np.ndarray, par, cov, hit_ids, last, first, cov_scale):
    """Inward pass from layer `last` down to `first` (orc_fit_backward): par/cov are the states
    on layer `last`; returns (par, cov, chi2, nhits, status) on layer `first`."""
    par = np.ascontiguousarray(par, dtype=np.float64)
    n = len(par)
    cov = np.ascontiguousarray(cov, dtype=np.float64).reshape(n, 36)
    hit_ids = np.ascontiguousarray(hit_ids, dtype=np.int32)
    assert hit_ids.shape == (n, g.n_layers)
    po, co = np.zeros((n, 6)), np.zeros((n, 36))
    c2 = np.zeros(n)
    nh = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    lib().orc_fit_backward_batch(C.byref(g), hits.ctypes.data, n, _d(par), _d(cov), float(cov_scale), _i(hit_ids),
                                 int(last), int(first), _d(po), _d(co), _d(c2), _i(nh), _i(status))
    return po, co.reshape(n, 6, 6), c2, nh, status


class SeedCuts(C.Structure):
    """Cuts of the seeding from hit triplets (orc_seed_cuts); defaults: pT >= 0.5 GeV with 15 %
    curvature slack, |z_vertex| <= 4 cm, |d0| <= 0.8 mm, |dz| <= 0.8 mm, confirmation within 1 mm."""

    _fields_ = [("pt_min", C.c_double), ("kappa_slack", C.c_double), ("z_vertex", C.c_double),
                ("d0_max", C.c_double), ("dz_max", C.c_double), ("conf_rphi", C.c_double), ("conf_z", C.c_double),
                ("confirm", C.c_int)]

    def __init__(self, pt_min=0.5, kappa_slack=0.15, z_vertex=4.0, d0_max=0.08, dz_max=0.08, conf_rphi=0.1,
                 conf_z=0.1, confirm=1):
        super().__init__(pt_min, kappa_slack, z_vertex, d0_max, dz_max, conf_rphi, conf_z, confirm)


class SeedQuant(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("chord01", "kappa01", "zv", "chord12", "kappa", "d0", "dz", "chord23",
                                          "f3", "dz3")] + [("collinear", C.c_int)]


SEED_PICK_DTYPE = np.dtype([("h1", "i4"), ("h2", "i4"), ("h3", "i4"), ("n_pass", "i4"), ("score", "f8"),
                            ("margin", "f8"), ("gap", "f8")], align=True)


def seed_kappa_max(g: Geom, cuts: SeedCuts) -> float:
    return lib().orc_seed_kappa_max(C.byref(g), C.byref(cuts))


def seed_eval(g: Geom, cuts: SeedCuts, a: Hit, b: Hit, c: Hit | None = None, e: Hit | None = None):
    """Quantities of one pair / triplet / confirmed triplet: (passes, SeedQuant)."""
    q = SeedQuant()
    ref = lambda h: C.byref(h) if h is not None else None
    ok = lib().orc_seed_eval(C.byref(g), C.byref(cuts), C.byref(a), C.byref(b), ref(c), ref(e), C.byref(q))
    return bool(ok), q


def find_seeds(g: Geom, cuts: SeedCuts, hits: np.ndarray, first=None) -> np.ndarray:
    """Best triplet of every first-layer hit of one event (brute force over all hits): a
    SEED_PICK_DTYPE record per hit (h1 = -1: none, or not a first-layer hit), or per entry of
    `first` (event-local ids of first-layer hits) when given."""
    hits = np.ascontiguousarray(hits)
    n = len(hits)
    if first is None:
        out = np.zeros(n, dtype=SEED_PICK_DTYPE)
        st = lib().orc_find_seeds(C.byref(g), C.byref(cuts), n, hits.ctypes.data, out.ctypes.data)
    else:
        first = np.ascontiguousarray(first, dtype=np.int32)
        out = np.zeros(len(first), dtype=SEED_PICK_DTYPE)
        st = lib().orc_find_seeds_of(C.byref(g), C.byref(cuts), n, hits.ctypes.data, len(first), _i(first),
                                     out.ctypes.data)
    assert st == 0, st
    return out


@dataclass
class EventIndex:
    hits: np.ndarray
    bin_of_hit: np.ndarray
    order: np.ndarray
    bin_off: np.ndarray
    struct: Event


def hit_index(g: Geom, hits: np.ndarray) -> EventIndex:
    n = len(hits)
    nb = g.n_eta_bins * g.n_phi_bins
    bin_of_hit = np.zeros(n, dtype=np.int32)
    order = np.zeros(n, dtype=np.int32)
    bin_off = np.zeros(g.n_layers * (nb + 1), dtype=np.int32)
    st = lib().orc_hit_index(C.byref(g), n, hits.ctypes.data, _i(bin_of_hit), _i(order), _i(bin_off))
    assert st == 0
    ev = Event()
    ev.n_hits = n
    ev.hits = hits.ctypes.data
    ev.order = order.ctypes.data
    ev.bin_off = bin_off.ctypes.data
    for l in range(g.n_layers):
        m = hits["layer"] == l
        ev.var_u_max[l] = float(hits["var_u"][m].max()) if m.any() else 0.0
        ev.var_v_max[l] = float(hits["var_v"][m].max()) if m.any() else 0.0
    return EventIndex(hits, bin_of_hit, order, bin_off.reshape(g.n_layers, nb + 1), ev)


@dataclass
class BuildResult:
    n_cand: np.ndarray
    par: np.ndarray     # [n, cap, 6]
    cov: np.ndarray     # [n, cap, 6, 6]
    chi2: np.ndarray    # [n, cap]
    nhits: np.ndarray   # [n, cap]
    hits: np.ndarray    # [n, cap, n_layers], event-local hit ids
    fragile: np.ndarray  # [n] first layer with a fragile decision (n_layers if none)
    stats: dict


def build(g: Geom, idx: EventIndex, seed_par, seed_cov, seed_chi2, seed_nhits, seed_hits, cap=None) -> BuildResult:
    seed_par = np.ascontiguousarray(seed_par, dtype=np.float64)
    n = len(seed_par)
    seed_cov = np.ascontiguousarray(seed_cov, dtype=np.float64).reshape(n, 36)
    seed_chi2 = np.ascontiguousarray(seed_chi2, dtype=np.float64)
    seed_nhits = np.ascontiguousarray(seed_nhits, dtype=np.int32)
    seed_hits = np.ascontiguousarray(seed_hits, dtype=np.int32)
    assert seed_hits.shape == (n, g.n_layers)
    if cap is None:
        cap = max(g.n_cand, 1)
    L = g.n_layers
    nc = np.zeros(n, dtype=np.int32)
    par = np.zeros((n, cap, 6))
    cov = np.zeros((n, cap, 36))
    c2 = np.zeros((n, cap))
    nh = np.zeros((n, cap), dtype=np.int32)
    hh = np.full((n, cap, L), -1, dtype=np.int32)
    fr = np.zeros(n, dtype=np.int32)
    stats = Stats()
    st = lib().orc_build_batch(C.byref(g), C.byref(idx.struct), n, _d(seed_par), _d(seed_cov), _d(seed_chi2),
                               _i(seed_nhits), _i(seed_hits), int(cap), _i(nc), _d(par), _d(cov), _d(c2),
                               _i(nh), _i(hh), _i(fr), C.byref(stats))
    assert st == 0
    s = {k: getattr(stats, k) for k, _ in Stats._fields_}
    return BuildResult(nc, par, cov.reshape(n, cap, 6, 6), c2, nh, hh, fr, s)
