"""Pins of the oracle's helix propagation to a cylinder (Sec. 2.2 toy: ideal barrel, uniform Bz).

Each test checks the oracle against something other than itself: a textbook closed form,
a general-purpose ODE integration of the Lorentz force, symmetries of the problem, and
finite differences of the propagation itself for the transport Jacobian.
"""
import math

import numpy as np
import pytest

import oracle as O

K_B = 0.00299792458


def _state(rng, r0=0.0):
    pt = rng.uniform(0.5, 10.0)
    q = rng.choice([-1.0, 1.0])
    phi = rng.uniform(-math.pi, math.pi)
    th = rng.uniform(0.6, math.pi - 0.6)
    pos_ang = phi + rng.uniform(-0.1, 0.1)
    return np.array([r0 * math.cos(pos_ang), r0 * math.sin(pos_ang), rng.normal(0, 1), q / pt, phi, th])


def _wrap(a):
    return (a + math.pi) % (2 * math.pi) - math.pi


def test_origin_closed_form(det):
    """From the origin the transverse path to radius R is (2/|k|) asin(|k| R / 2)."""
    g = O.make_geom(det)
    rng = np.random.default_rng(1)
    for _ in range(200):
        p = _state(rng)
        p[0] = p[1] = 0.0
        R = rng.uniform(1.0, 40.0)
        st, out, _ = O.propagate(g, p, R)
        assert st == 0
        kappa = abs(K_B * det.bz * p[3])
        s = 2.0 / kappa * math.asin(kappa * R / 2.0)
        assert out[2] == pytest.approx(p[2] + s / math.tan(p[5]), abs=1e-10)
        assert math.hypot(out[0], out[1]) == pytest.approx(R, abs=1e-10)
        # exit azimuth of momentum: phi + kappa_signed * s
        ks = -K_B * det.bz * p[3]
        assert abs(_wrap(out[4] - (p[4] + ks * s))) < 1e-10


def _lorentz_rhs(bz, q):
    def f(_s, y):
        px, py, pz = y[3], y[4], y[5]
        p = math.sqrt(px * px + py * py + pz * pz)
        ux, uy, uz = px / p, py / p, pz / p
        # dp/ds = K_B q (u x B),  B = (0, 0, bz)
        return [ux, uy, uz, K_B * q * uy * bz, -K_B * q * ux * bz, 0.0]
    return f


def test_agrees_with_ode_integration_of_lorentz_force(det):
    """Integrate dp/ds = K_B q (u x B) with an 8th-order adaptive Runge-Kutta and stop on r = R."""
    integrate = pytest.importorskip("scipy.integrate")
    g = O.make_geom(det)
    rng = np.random.default_rng(2)
    for _ in range(40):
        p = _state(rng, r0=rng.uniform(3.0, 20.0))
        R = math.hypot(p[0], p[1]) + rng.uniform(1.0, 20.0)
        q = math.copysign(1.0, p[3])
        pt = 1.0 / abs(p[3])
        y0 = [p[0], p[1], p[2], pt * math.cos(p[4]), pt * math.sin(p[4]), pt / math.tan(p[5])]
        ev = lambda _s, y: math.hypot(y[0], y[1]) - R
        ev.terminal, ev.direction = True, 1
        sol = integrate.solve_ivp(_lorentz_rhs(det.bz, q), (0, 500.0), y0, method="DOP853", rtol=1e-13,
                                  atol=1e-13, events=ev)
        yE = sol.y_events[0][0]
        st, out, _ = O.propagate(g, p, R)
        assert st == 0
        assert np.allclose(out[:3], yE[:3], atol=1e-8)
        assert abs(_wrap(out[4] - math.atan2(yE[4], yE[3]))) < 1e-10
        assert out[5] == pytest.approx(math.atan2(math.hypot(yE[3], yE[4]), yE[5]), abs=1e-10)
        assert out[3] == p[3]


def test_rotation_invariance(det):
    g = O.make_geom(det)
    rng = np.random.default_rng(3)
    for _ in range(100):
        p = _state(rng, r0=rng.uniform(3.0, 20.0))
        R = math.hypot(p[0], p[1]) + rng.uniform(1.0, 15.0)
        a = rng.uniform(-math.pi, math.pi)
        c, s = math.cos(a), math.sin(a)
        pr = p.copy()
        pr[0], pr[1] = c * p[0] - s * p[1], s * p[0] + c * p[1]
        pr[4] = _wrap(p[4] + a)
        _, o1, _ = O.propagate(g, p, R)
        _, o2, _ = O.propagate(g, pr, R)
        assert o2[0] == pytest.approx(c * o1[0] - s * o1[1], abs=1e-10)
        assert o2[1] == pytest.approx(s * o1[0] + c * o1[1], abs=1e-10)
        assert o2[2] == pytest.approx(o1[2], abs=1e-10)
        assert abs(_wrap(o2[4] - o1[4] - a)) < 1e-10


def test_charge_conjugation_mirror(det):
    """Mirroring y -> -y and flipping the charge gives the mirrored trajectory."""
    g = O.make_geom(det)
    rng = np.random.default_rng(4)
    for _ in range(100):
        p = _state(rng, r0=rng.uniform(3.0, 20.0))
        R = math.hypot(p[0], p[1]) + rng.uniform(1.0, 15.0)
        m = p.copy()
        m[1], m[3], m[4] = -p[1], -p[3], -p[4]
        _, o1, _ = O.propagate(g, p, R)
        _, o2, _ = O.propagate(g, m, R)
        assert np.allclose([o2[0], -o2[1], o2[2], -o2[3], o2[5]], [o1[0], o1[1], o1[2], o1[3], o1[5]], atol=1e-10)
        assert abs(_wrap(-o2[4] - o1[4])) < 1e-10


@pytest.mark.parametrize("pt_hi", [10.0, 100.0, 1e5, 1e9])
def test_jacobian_matches_finite_differences(det, pt_hi):
    """Includes nearly straight helices (pT up to 1e9 GeV), as three-hit seed estimates of
    stiff tracks produce."""
    g = O.make_geom(det)
    rng = np.random.default_rng(5)
    for _ in range(60):
        p = _state(rng, r0=rng.uniform(3.0, 30.0))
        p[3] = math.copysign(1.0 / (pt_hi if pt_hi > 100 else rng.uniform(0.5, pt_hi)) * rng.uniform(0.5, 1.0), p[3])
        # steps large against the ~1e-12 cm rounding of the closed form, small against curvature
        steps = np.array([1e-4, 1e-4, 1e-4, 1e-4 * max(abs(p[3]), 0.05), 1e-5, 1e-5])
        R = math.hypot(p[0], p[1]) + rng.uniform(1.0, 10.0)
        st, _, J = O.propagate(g, p, R)
        assert st == 0
        Jfd = np.zeros((6, 6))
        for j in range(6):
            hp, hm = p.copy(), p.copy()
            hp[j] += steps[j]
            hm[j] -= steps[j]
            _, op, _ = O.propagate(g, hp, R)
            _, om, _ = O.propagate(g, hm, R)
            d = op - om
            d[4] = _wrap(d[4])
            Jfd[:, j] = d / (2 * steps[j])
        scale = np.maximum(np.abs(J), 1.0)
        assert np.max(np.abs(J - Jfd) / scale) < 1e-6


def test_agrees_with_generator_simulation(det):
    """The event generator's Newton solution on the exact helix is an independent crossing."""
    from synth import EventSpec, generate
    b = generate(EventSpec(seed=9, n_tracks=300, scatter=False, smear=False), det)
    g = O.make_geom(det)
    worst = 0.0
    for t in range(b.n_tracks):
        for l in range(1, det.n_layers):
            _, out, _ = O.propagate(g, b.truth[t, l - 1], det.radii[l])
            d = out - b.truth[t, l]
            d[4] = _wrap(d[4])
            worst = max(worst, np.max(np.abs(d)))
    assert worst < 1e-9


def test_continuous_at_the_straight_line_limit(det):
    """Curvature just above and just below the straight-line switch gives the same crossing
    and Jacobian as an exactly straight track."""
    g = O.make_geom(det)
    rng = np.random.default_rng(6)
    for _ in range(50):
        p = _state(rng, r0=rng.uniform(3.0, 30.0))
        R = math.hypot(p[0], p[1]) + rng.uniform(1.0, 10.0)
        p0 = p.copy()
        p0[3] = 0.0
        _, o0, J0 = O.propagate(g, p0, R)
        for w in (1e-11, 1e-9, 1e-7):
            p1 = p.copy()
            p1[3] = w
            _, o1, J1 = O.propagate(g, p1, R)
            # the curvature itself moves the crossing by about K_B Bz w s^2 / 2 < 0.006 w R^2
            assert np.allclose(o1, o0, atol=1e-12 + 0.01 * w * R * R)
            assert np.allclose(J1, J0, atol=1e-9 + 0.01 * w * R * R)


def test_no_reach_is_reported(det):
    g = O.make_geom(det)
    p = np.array([0.0, 0.0, 0.0, 1.0 / 0.2, 0.3, 1.2])  # pT 0.2 GeV: 2 rho = 35 cm < 40 cm
    st, _, _ = O.propagate(g, p, 40.0)
    assert st == 1
