"""Seeded synthetic barrel events: the toy test scenario of the paper's Sec. 2.2.

A particle gun (flat pT, flat eta, flat phi, random charge, Gaussian vertex) is simulated
through an ideal barrel of thin cylinders in a uniform solenoid field Bz.  At each cylinder
the exact helix crossing is found, a hit is made by Gaussian smearing along the cylinder
(r-phi and z), and the direction is then deflected by a thin-scatterer multiple-scattering
kick (two Gaussian angles of Highland width, |p| conserved).  Uniform random noise hits are
added per layer.  The paper's own toy had no material; the thin scatterers follow the
build's workload definition and can be switched off.

This is an input producer, not an implementation of the method: it finds helix/cylinder
crossings by Newton iteration on the exact helix (the reconstruction side uses other
algorithms), and it draws every random number from Philox4x32-10 keyed by
(run seed, event) with counter (object, stream, block, kind), so results are identical on
every machine and any event can be regenerated alone.

Units: cm, GeV, T, rad.  Track state convention: (x, y, z, q/pT, phi, theta) with phi the
azimuth and theta the polar angle of the momentum.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .philox import normals, uniforms

K_B = 0.00299792458  # GeV / (T cm): curvature constant, 1/rho = K_B * Bz / pT


@dataclass(frozen=True)
class Detector:
    """Ideal barrel: n thin cylinders at radius[l], uniform Bz, thickness x/X0 per layer.

    module_dr > 0 gives the layers modules off the average cylinder (the simplified CMS
    geometry of the paper's Sec. 2.2): layer l is tiled in phi by an even number of modules,
    each about module_width long, alternately at radius[l] - module_dr/2 (even index, from
    phi = -pi) and radius[l] + module_dr/2 (odd index).  A track's module is the one where it
    crosses radius[l]; its hit and truth lie where it crosses that module's radius."""

    radii: tuple = tuple(4.0 * (l + 1) for l in range(10))
    bz: float = 3.8
    x_over_x0: tuple = tuple(0.03 for _ in range(10))
    mass: float = 0.13957  # scattering mass hypothesis (charged pion)
    sigma_rphi: float = 0.01
    sigma_z: float = 0.1    # second measured coordinate: z on a cylinder, r on a disk
    module_dr: float = 0.0
    module_width: float = 2.0
    # Endcap disks (the "endcap z" of the paper's Sec. 2.2): disk_z[l] > 0 makes layer l a pair
    # of disks at z = +-disk_z[l] (a track crosses the one on its side), radii[l] its outer
    # radius; () or 0 keeps the layer a cylinder of radius radii[l].
    disk_z: tuple = ()
    disk_rmin: float = 1.0
    # Pixel seeding layers: layers 0 .. pixel_layers - 1 measure (r-phi, z) with pixel_sigma
    # instead of (sigma_rphi, sigma_z), the fine inner layers a seeding from hit triplets needs
    # (with 1 mm in z three hits 4 cm apart do not single out a track in a dense event).
    pixel_layers: int = 0
    pixel_sigma: tuple = (0.002, 0.005)

    @property
    def n_layers(self) -> int:
        return len(self.radii)

    def sigma(self, l: int):
        """(r-phi, second coordinate) resolution of layer l in cm."""
        return tuple(self.pixel_sigma) if l < self.pixel_layers else (self.sigma_rphi, self.sigma_z)

    def is_disk(self, l: int) -> bool:
        return bool(self.disk_z) and self.disk_z[l] > 0.0

    def n_modules(self, l: int) -> int:
        return 2 * max(2, int(np.ceil(np.pi * self.radii[l] / self.module_width)))

    def module_radius(self, l: int, phi):
        """Radius of the module of layer l at azimuth phi (radius[l] when module_dr == 0)."""
        phi = np.asarray(phi, dtype=np.float64)
        if self.module_dr == 0.0:
            return np.full(phi.shape, float(self.radii[l]))
        n = self.n_modules(l)
        k = np.clip(np.floor((phi + np.pi) / (2.0 * np.pi) * n).astype(np.int64), 0, n - 1)
        return self.radii[l] + np.where(k % 2 == 0, -0.5, 0.5) * self.module_dr


@dataclass
class EventSpec:
    """What to generate.  `n_tracks` and `noise_frac` are scalars or per-event arrays."""

    seed: int = 1
    n_events: int = 1
    n_tracks: object = 1000
    pt_min: float = 0.5
    pt_max: float = 10.0
    eta_max: float = 1.0
    eta_min: float = 0.0  # > 0: |eta| uniform in [eta_min, eta_max], either sign (forward tracks)
    noise_frac: object = 0.0
    vertex_sigma: tuple = (0.01, 0.01, 1.0)
    scatter: bool = True
    smear: bool = True
    shuffle_hits: bool = True
    keep_f64: bool = False  # also keep the unrounded FP64 hit positions in extras["xyz64"]
    first_event: int = 0    # events first_event .. first_event + n_events - 1 of the run


@dataclass
class EventBatch:
    """Hits and truth of several events, concatenated event by event.

    Hits of event e occupy [hit_off[e], hit_off[e+1]); within an event they are ordered by
    layer and, inside a layer, in a seeded random order.  Tracks of event e occupy
    [trk_off[e], trk_off[e+1]).  `trk_hits[t, l]` is the global index of track t's hit on
    layer l.  `truth[t, l]` is the exact state where track t crosses layer l, before that
    layer's scattering kick; `truth_after[t, l]` is the same state right after the kick.
    """

    detector: Detector
    spec: EventSpec
    hit_off: np.ndarray
    trk_off: np.ndarray
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    var_u: np.ndarray
    var_v: np.ndarray
    layer: np.ndarray
    mc: np.ndarray
    trk_event: np.ndarray
    trk_hits: np.ndarray
    truth: np.ndarray
    truth_after: np.ndarray
    vertex_state: np.ndarray
    extras: dict = field(default_factory=dict)

    @property
    def n_events(self) -> int:
        return len(self.hit_off) - 1

    @property
    def n_hits(self) -> int:
        return len(self.x)

    @property
    def n_tracks(self) -> int:
        return len(self.trk_event)


# Philox stream ids (second counter word); documented so that both sides could regenerate.
_KIN, _LAYER0, _NOISE0, _SHUF0, _EVT = 0, 1, 40, 80, 120


def event_sizes(seed: int, n_events: int, median=3000.0, sigma_ln=0.8, lo=200, hi=20000,
                noise_lo=0.2, noise_hi=0.5):
    """Per-event track counts (lognormal, clipped) and noise fractions (uniform)."""
    ev = np.arange(n_events, dtype=np.uint64)
    key = (np.uint64(seed), np.uint64(0xFFFFFFFF))
    g0, _ = normals(key, (ev, _EVT, 0, 2))
    u0, _ = uniforms(key, (ev, _EVT, 1, 2))
    n = np.clip(np.rint(median * np.exp(sigma_ln * g0)), lo, hi).astype(np.int64)
    f = noise_lo + (noise_hi - noise_lo) * u0
    return n, f


def _helix_to_cylinder(x, y, z, w, phi, theta, radius, kb):
    """Exact helix crossing of r = radius by Newton iteration on the transverse path s."""
    kappa = -kb * w
    cphi, sphi = np.cos(phi), np.sin(phi)
    a = x * cphi + y * sphi
    s = -a + np.sqrt(np.maximum(a * a + radius * radius - (x * x + y * y), 0.0))
    # a fixed number of iterations (quadratic convergence from the straight-line start needs
    # about four) keeps every track's result independent of which tracks share the array
    for _ in range(8):
        ang = phi + kappa * s
        xs = x + (np.sin(ang) - sphi) / kappa
        ys = y - (np.cos(ang) - cphi) / kappa
        g = xs * xs + ys * ys - radius * radius
        dg = 2.0 * (xs * np.cos(ang) + ys * np.sin(ang))
        s = s - g / dg
    ang = phi + kappa * s
    xs = x + (np.sin(ang) - sphi) / kappa
    ys = y - (np.cos(ang) - cphi) / kappa
    zs = z + s * np.cos(theta) / np.sin(theta)
    if not np.all(np.abs(np.hypot(xs, ys) - radius) < 1e-9):
        raise RuntimeError("helix/cylinder Newton iteration did not converge")
    if not np.all(s > 0):
        raise RuntimeError("a generated track does not move outward")
    phi_new = np.arctan2(np.sin(ang), np.cos(ang))
    return xs, ys, zs, phi_new


def _helix_to_plane(x, y, z, w, phi, theta, zplane, kb):
    """Exact helix crossing of the plane z = zplane: the transverse path is (zplane - z) tan(theta)."""
    kappa = -kb * w
    s = (zplane - z) * np.tan(theta)
    if not np.all(s > 0):
        raise RuntimeError("a generated track does not move towards its disk")
    ang = phi + kappa * s
    xs = x + (np.sin(ang) - np.sin(phi)) / kappa
    ys = y - (np.cos(ang) - np.cos(phi)) / kappa
    return xs, ys, np.full_like(x, 0.0) + zplane, np.arctan2(np.sin(ang), np.cos(ang))


def _scatter(key, tl, l, q, w, phi, theta, cos_inc, det):
    """Thin-scatterer kick on layer l: two Gaussian angles of Highland width for the path
    x/X0 / cos_inc, orthogonal to the direction, |p| kept.  Returns (theta, phi, q/pT)."""
    a1, a2 = normals(key, (tl, _LAYER0 + l, 1, 0))
    p = 1.0 / (np.abs(w) * np.sin(theta))
    d = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)
    th0 = highland_theta0(p, det.mass, det.x_over_x0[l] / cos_inc)
    e_th = np.stack([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)], axis=1)
    e_ph = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=1)
    dn = d + (th0 * a1)[:, None] * e_th + (th0 * a2)[:, None] * e_ph
    dn /= np.linalg.norm(dn, axis=1)[:, None]
    theta = np.arccos(np.clip(dn[:, 2], -1.0, 1.0))
    phi = np.arctan2(dn[:, 1], dn[:, 0])
    return theta, phi, q / (p * np.sin(theta))


def highland_theta0(p, mass, thickness):
    """Highland width of the projected scattering angle for unit charge (PDG form)."""
    beta = p / np.sqrt(p * p + mass * mass)
    return 0.0136 / (beta * p) * np.sqrt(thickness) * (1.0 + 0.038 * np.log(thickness / (beta * beta)))


def generate(spec: EventSpec, det: Detector = Detector()) -> EventBatch:
    n_ev = spec.n_events
    n_trk = np.broadcast_to(np.asarray(spec.n_tracks, dtype=np.int64), (n_ev,)).copy()
    noise_frac = np.broadcast_to(np.asarray(spec.noise_frac, dtype=np.float64), (n_ev,)).copy()
    L = det.n_layers
    kb = K_B * det.bz

    trk_off = np.zeros(n_ev + 1, dtype=np.int64)
    trk_off[1:] = np.cumsum(n_trk)
    T = int(trk_off[-1])
    trk_event = np.repeat(np.arange(n_ev, dtype=np.int64), n_trk)
    trk_local = np.arange(T, dtype=np.int64) - trk_off[trk_event]
    key = (np.uint64(spec.seed), (trk_event + spec.first_event).astype(np.uint64))
    tl = trk_local.astype(np.uint64)

    # --- kinematics at the vertex
    u_pt, u_eta = uniforms(key, (tl, _KIN, 0, 0))
    u_phi, u_q = uniforms(key, (tl, _KIN, 1, 0))
    gvx, gvy = normals(key, (tl, _KIN, 2, 0))
    gvz, _ = normals(key, (tl, _KIN, 3, 0))
    pt = spec.pt_min + (spec.pt_max - spec.pt_min) * u_pt
    if spec.eta_min > 0.0:
        a = 2.0 * np.abs(u_eta - 0.5)
        eta = np.where(u_eta < 0.5, -1.0, 1.0) * (spec.eta_min + (spec.eta_max - spec.eta_min) * a)
    else:
        eta = -spec.eta_max + 2.0 * spec.eta_max * u_eta
    theta = 2.0 * np.arctan(np.exp(-eta))
    phi = -np.pi + 2.0 * np.pi * u_phi
    q = np.where(u_q < 0.5, 1.0, -1.0)
    x = spec.vertex_sigma[0] * gvx
    y = spec.vertex_sigma[1] * gvy
    z = spec.vertex_sigma[2] * gvz
    w = q / pt
    vertex_state = np.stack([x, y, z, w, phi, theta], axis=1)

    truth = np.zeros((T, L, 6))
    truth_after = np.zeros((T, L, 6))
    sig_hit = np.zeros((T, L, 3))  # x, y, z of the signal hit
    for l in range(L):
        R = det.radii[l]
        if det.is_disk(l):
            x, y, z, phi = _helix_to_plane(x, y, z, w, phi, theta, np.where(np.cos(theta) > 0, 1.0, -1.0) * det.disk_z[l], kb)
            truth[:, l] = np.stack([x, y, z, w, phi, theta], axis=1)
            g_rphi, g_r = normals(key, (tl, _LAYER0 + l, 0, 0))
            phi_pos = np.arctan2(y, x)
            r_pos = np.hypot(x, y)
            if spec.smear:
                sr, sz = det.sigma(l)
                phi_h = phi_pos + sr * g_rphi / r_pos
                r_h = r_pos + sz * g_r
            else:
                phi_h, r_h = phi_pos, r_pos
            sig_hit[:, l] = np.stack([r_h * np.cos(phi_h), r_h * np.sin(phi_h), z], axis=1)
            if spec.scatter and det.x_over_x0[l] > 0.0:
                theta, phi, w = _scatter(key, tl, l, q, w, phi, theta, np.abs(np.cos(theta)), det)
            truth_after[:, l] = np.stack([x, y, z, w, phi, theta], axis=1)
            continue
        if det.module_dr != 0.0:
            # the module is the one crossed on the average cylinder; the track then goes from
            # its previous point straight to that module's radius
            xa, ya, _, _ = _helix_to_cylinder(x, y, z, w, phi, theta, R, kb)
            R = det.module_radius(l, np.arctan2(ya, xa))
        x, y, z, phi = _helix_to_cylinder(x, y, z, w, phi, theta, R, kb)
        truth[:, l] = np.stack([x, y, z, w, phi, theta], axis=1)
        g_rphi, g_z = normals(key, (tl, _LAYER0 + l, 0, 0))
        phi_pos = np.arctan2(y, x)
        if spec.smear:
            sr, sz = det.sigma(l)
            phi_h = phi_pos + sr * g_rphi / R
            z_h = z + sz * g_z
        else:
            phi_h, z_h = phi_pos, z.copy()
        sig_hit[:, l] = np.stack([R * np.cos(phi_h), R * np.sin(phi_h), z_h], axis=1)
        if spec.scatter and det.x_over_x0[l] > 0.0:
            d = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)
            radial = np.stack([np.cos(phi_pos), np.sin(phi_pos), np.zeros_like(phi_pos)], axis=1)
            cos_inc = np.abs(np.sum(d * radial, axis=1))
            theta, phi, w = _scatter(key, tl, l, q, w, phi, theta, cos_inc, det)
        truth_after[:, l] = np.stack([x, y, z, w, phi, theta], axis=1)

    # --- assemble hits event by event: layer-major, signal then noise, then shuffled
    xs, ys, zs, lays, mcs = [], [], [], [], []
    hit_off = np.zeros(n_ev + 1, dtype=np.int64)
    trk_hits = np.full((T, L), -1, dtype=np.int64)
    for e in range(n_ev):
        t0, t1 = int(trk_off[e]), int(trk_off[e + 1])
        nt = t1 - t0
        base = int(hit_off[e])
        ekey = (np.uint64(spec.seed), np.uint64(e + spec.first_event))
        for l in range(L):
            R = det.radii[l]
            n_noise = int(np.rint(noise_frac[e] * nt))
            nid = np.arange(n_noise, dtype=np.uint64)
            u_a, u_b = uniforms(ekey, (nid, _NOISE0 + l, 0, 1))
            nphi = -np.pi + 2.0 * np.pi * u_a
            if det.is_disk(l):
                # uniform in phi and in |eta| over the acceptance widened by 0.2, either disk
                u_c, _ = uniforms(ekey, (nid, _NOISE0 + l, 1, 1))
                e_lo, e_hi = max(spec.eta_min - 0.2, 0.05), spec.eta_max + 0.2
                nr = det.disk_z[l] / np.sinh(e_lo + (e_hi - e_lo) * u_b)
                nz = np.where(u_c < 0.5, -1.0, 1.0) * det.disk_z[l]
            else:
                zl = R * np.sinh(spec.eta_max) + 3.0 * spec.vertex_sigma[2]
                nr = det.module_radius(l, nphi) if det.module_dr != 0.0 else R
                nz = -zl + 2.0 * zl * u_b
            hx = np.concatenate([sig_hit[t0:t1, l, 0], nr * np.cos(nphi)])
            hy = np.concatenate([sig_hit[t0:t1, l, 1], nr * np.sin(nphi)])
            hz = np.concatenate([sig_hit[t0:t1, l, 2], nz])
            mc = np.concatenate([np.arange(t0, t1, dtype=np.int64), np.full(n_noise, -1, dtype=np.int64)])
            n_l = nt + n_noise
            if spec.shuffle_hits:
                h_idx = np.arange(n_l, dtype=np.uint64)
                k0, _ = uniforms(ekey, (h_idx, _SHUF0 + l, 0, 3))
                perm = np.argsort(k0, kind="stable")
            else:
                perm = np.arange(n_l)
            hx, hy, hz, mc = hx[perm], hy[perm], hz[perm], mc[perm]
            pos = base + np.arange(n_l, dtype=np.int64)
            sig = mc >= 0
            trk_hits[mc[sig], l] = pos[sig]
            xs.append(hx); ys.append(hy); zs.append(hz); mcs.append(mc)
            lays.append(np.full(n_l, l, dtype=np.int32))
            base += n_l
        hit_off[e + 1] = base

    n_hits = int(hit_off[-1])
    extras = {}
    if spec.keep_f64:
        extras["xyz64"] = np.stack([np.concatenate(xs), np.concatenate(ys), np.concatenate(zs)], axis=1)
    cat = lambda parts, dt: np.concatenate(parts).astype(dt) if parts else np.zeros(0, dt)
    layer = cat(lays, np.int32)
    var_l = np.array([[det.sigma(l)[0] ** 2, det.sigma(l)[1] ** 2] for l in range(L)], dtype=np.float64)
    batch = EventBatch(
        detector=det, spec=spec, hit_off=hit_off, trk_off=trk_off,
        x=cat(xs, np.float32), y=cat(ys, np.float32), z=cat(zs, np.float32),
        var_u=var_l[layer, 0].astype(np.float32) if n_hits else np.zeros(0, np.float32),
        var_v=var_l[layer, 1].astype(np.float32) if n_hits else np.zeros(0, np.float32),
        layer=layer, mc=cat(mcs, np.int64),
        trk_event=trk_event, trk_hits=trk_hits, truth=truth, truth_after=truth_after,
        vertex_state=vertex_state, extras=extras,
    )
    return batch


def concat(batches):
    """One batch holding the events of several batches in order (hit and track ids re-based)."""
    b0 = batches[0]
    hit_base = np.cumsum([0] + [b.n_hits for b in batches])
    trk_base = np.cumsum([0] + [b.n_tracks for b in batches])
    ev_base = np.cumsum([0] + [b.n_events for b in batches])
    cat = lambda k: np.concatenate([getattr(b, k) for b in batches])
    extras = {}
    if all("xyz64" in b.extras for b in batches):
        extras["xyz64"] = np.concatenate([b.extras["xyz64"] for b in batches])
    return EventBatch(
        detector=b0.detector, spec=b0.spec,
        hit_off=np.concatenate([[0]] + [b.hit_off[1:] + hb for b, hb in zip(batches, hit_base)]),
        trk_off=np.concatenate([[0]] + [b.trk_off[1:] + tb for b, tb in zip(batches, trk_base)]),
        x=cat("x"), y=cat("y"), z=cat("z"), var_u=cat("var_u"), var_v=cat("var_v"), layer=cat("layer"),
        mc=np.concatenate([np.where(b.mc >= 0, b.mc + tb, -1) for b, tb in zip(batches, trk_base)]),
        trk_event=np.concatenate([b.trk_event + eb for b, eb in zip(batches, ev_base)]),
        trk_hits=np.concatenate([np.where(b.trk_hits >= 0, b.trk_hits + hb, -1) for b, hb in zip(batches, hit_base)]),
        truth=cat("truth"), truth_after=cat("truth_after"), vertex_state=cat("vertex_state"), extras=extras,
    )


def forward_detector(n_layers: int = 10, spacing: float = 8.0, x_over_x0: float = 0.03, **kw) -> Detector:
    """An endcap-only tracker (the "endcap z" geometry of the paper's Sec. 2.2): n_layers pairs of
    disks at z = +-spacing, +-2 spacing, ... with outer radius 40 cm and inner radius 1 cm, in the
    same 3.8 T field; hits measured in r-phi (sigma_rphi) and r (sigma_z, 0.1 cm).  Tracks with
    1.7 <= |eta| <= 2.5 cross every disk of their side."""
    return Detector(radii=(40.0,) * n_layers, x_over_x0=(x_over_x0,) * n_layers,
                    disk_z=tuple(spacing * (l + 1) for l in range(n_layers)), disk_rmin=1.0, **kw)


FORWARD_ETA = (1.7, 2.5)
# Seed prior (cm, cm, cm, GeV^-1, rad, rad) for the endcap tracker: three hits on the first disks
# span a few cm of arc, so their curvature estimate is poorer than in the barrel and the prior on
# q/pT must be wider to stay uninformative (z is the first disk's, known exactly).
FORWARD_PRIOR = (0.3, 0.3, 1.0, 5.0, 0.1, 0.1)
