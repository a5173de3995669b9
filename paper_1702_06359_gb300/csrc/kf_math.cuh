// Device-side Kalman-filter arithmetic for one track state (Sec. 2, 2.2 of arXiv:1702.06359):
// helix propagation to a barrel cylinder with its transport Jacobian, thin-layer scattering
// noise, chi2 of a hit and the Kalman update on the plane tangent to the cylinder.
//
// State p = (x, y, z, w = q/pT, phi, theta); covariance P as the 21-element packed lower
// triangle, row order.  Everything is written out with the sparsity of the Jacobian and of H
// (the paper's Matriplex generator idea of skipping known zeros and ones, Sec. 2.1): the
// congruence products J P J^T and M P M^T come from gen_sparse.py (sparse_gen.cuh), the rest is
// written by hand, so no 6x6 product is ever formed densely.  Templated on the real type R (float or
// double) so that one source serves the FP32, mixed and FP64 modes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ieee_cvt.cuh"
#include "sparse_gen.cuh"

namespace tkf {

constexpr double kCurv = 0.00299792458;  // GeV / (T cm)
constexpr double kPi = 3.14159265358979323846;

__host__ __device__ constexpr int sym(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

// ------------------------------------------------------------------ math wrappers per type
__host__ __device__ __forceinline__ void sc(float a, float *s, float *c) { sincosf(a, s, c); }
__host__ __device__ __forceinline__ void sc(double a, double *s, double *c) { sincos(a, s, c); }
__host__ __device__ __forceinline__ float sq(float a) { return sqrtf(a); }
__host__ __device__ __forceinline__ double sq(double a) { return sqrt(a); }
__host__ __device__ __forceinline__ float lg(float a) { return logf(a); }
__host__ __device__ __forceinline__ double lg(double a) { return log(a); }
__host__ __device__ __forceinline__ float at2(float y, float x) { return atan2f(y, x); }
__host__ __device__ __forceinline__ double at2(double y, double x) { return atan2(y, x); }
__host__ __device__ __forceinline__ float asn(float a) { return asinf(a); }
__host__ __device__ __forceinline__ double asn(double a) { return asin(a); }
__host__ __device__ __forceinline__ float ab(float a) { return fabsf(a); }
__host__ __device__ __forceinline__ double ab(double a) { return fabs(a); }
__host__ __device__ __forceinline__ float flr(float a) { return floorf(a); }
__host__ __device__ __forceinline__ double flr(double a) { return floor(a); }

// Variants where a few ulp do not matter (scattering width, polar-angle trig, 1/r of a hit,
// chi2 division): hardware approximations in float, the accurate functions in double.
__host__ __device__ __forceinline__ void fast_sc(float a, float *s, float *c)
{
#ifdef __CUDA_ARCH__
    __sincosf(a, s, c);
#else
    sincosf(a, s, c);
#endif
}
__host__ __device__ __forceinline__ void fast_sc(double a, double *s, double *c) { sincos(a, s, c); }
__host__ __device__ __forceinline__ float fast_log(float a)
{
#ifdef __CUDA_ARCH__
    return __logf(a);
#else
    return logf(a);
#endif
}
__host__ __device__ __forceinline__ double fast_log(double a) { return log(a); }
__host__ __device__ __forceinline__ float fast_rsqrt(float a)
{
#ifdef __CUDA_ARCH__
    return rsqrtf(a);
#else
    return 1.0f / sqrtf(a);
#endif
}
__host__ __device__ __forceinline__ double fast_rsqrt(double a) { return 1.0 / sqrt(a); }
__host__ __device__ __forceinline__ float fast_div(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
__host__ __device__ __forceinline__ double fast_div(double a, double b) { return a / b; }

template <class R> struct Lim;
template <> struct Lim<float> {
    static constexpr float series = 0.25f;  // |kappa s| below which the helix functions use series
    // Newton steps from the straight-line start (error <= ~0.1 cm for 4 cm steps): two bring
    // it below 1e-9 cm, under the float rounding of the crossing itself
    static constexpr int newton = 2;
    // a Newton step at most this fraction of the path: converged to the type's rounding (used by
    // the inward propagation, which may need more steps than `newton`)
    static constexpr float converged = 1e-6f;
};
template <> struct Lim<double> {
    static constexpr double series = 0.05;
    static constexpr int newton = 4;
    static constexpr double converged = 1e-13;
};

template <class R> __host__ __device__ __forceinline__ R wrap_phi(R phi)
{
    const R tp = R(2.0 * kPi);
    if (phi >= R(kPi)) phi -= tp;
    if (phi < R(-kPi)) phi += tp;
    return phi;
}

// S(a) = sin(a)/a, C(a) = (1 - cos a)/a and their derivatives dS/da, dC/da.  Near a = 0 the
// Taylor series are used (they keep full relative precision where the direct forms cancel).
template <class R> __host__ __device__ __forceinline__ void helix_fn(R a, R &S, R &C, R &Sd, R &Cd)
{
    if (ab(a) < Lim<R>::series) {
        const R a2 = a * a;
        S = R(1) + a2 * (R(-1.0 / 6) + a2 * (R(1.0 / 120) + a2 * (R(-1.0 / 5040) + a2 * R(1.0 / 362880))));
        C = a * (R(0.5) + a2 * (R(-1.0 / 24) + a2 * (R(1.0 / 720) + a2 * (R(-1.0 / 40320) + a2 * R(1.0 / 3628800)))));
        Sd = a * (R(-1.0 / 3) + a2 * (R(1.0 / 30) + a2 * (R(-1.0 / 840) + a2 * (R(1.0 / 45360) - a2 * R(1.0 / 3991680)))));
        Cd = R(0.5) + a2 * (R(-1.0 / 8) + a2 * (R(1.0 / 144) + a2 * (R(-1.0 / 5760) + a2 * R(1.0 / 403200))));
    } else {
        R sn, cs;
        sc(a, &sn, &cs);
        const R ia = R(1) / a;
        S = sn * ia;
        C = (R(1) - cs) * ia;
        Sd = (cs - S) * ia;
        Cd = (sn - C) * ia;
    }
}

// ------------------------------------------------------------------ propagation (Sec. 2.2)
//
// Exact propagation of the helix  x(s) = x0 + s (cos phi S(ks) - sin phi C(ks)),
// y(s) = y0 + s (sin phi S(ks) + cos phi C(ks)), z(s) = z0 + s cot(theta), phi(s) = phi + k s
// (k = -K Bz q/pT, s the transverse path) to the cylinder r = radius: s is found by Newton's
// method on g(s) = x(s)^2 + y(s)^2 - radius^2 from the straight-line solution.  The transport
// Jacobian is the derivative at fixed s plus (dp/ds)(ds/dp_in) with ds/dp_in from the
// constraint r(s, p_in) = radius; P <- J P J^T uses its sparsity (rows of q/pT and theta are
// unit rows, rows x, y, phi touch columns x, y, q/pT, phi only).
// Returns false when the cylinder is not reached.
//
// Modes:
//   kPropOut: the next crossing ahead (s > 0), Newton from the straight line's outer root.
//   kPropIn: the cylinder lies inside the state's radius (the backward pass runs the reversed
//     track outward-in).  The straight line then meets it twice ahead, and Newton starts from
//     the nearer root; when the tangent line misses the cylinder but the helix curves onto it,
//     the start is the exact crossing of the two circles: the track circle has centre
//     c = p0 + (-sin phi, cos phi)/k, and the position seen from c turns by k s, so
//     s = (signed angle from p0 - c to the crossing - c) / k, taken in (0, 2 pi/|k|].
//   kPropStep: the second of the two steps of Sec. 2.2, from a state on a layer's average
//     radius to a hit's own radius close by: s of either sign, the crossing where the track
//     moves outward, Newton from the straight line's nearer root written without cancellation,
//     (radius^2 - r0^2) / (A + sqrt(disc)).
enum : int { kPropOut = 0, kPropIn = 1, kPropStep = 2 };

template <class R, int kMode = kPropOut>
__host__ __device__ __forceinline__ bool propagate(R p[6], R P[21], R radius, R kb)
{
    const R x = p[0], y = p[1], z = p[2], w = p[3], phi = p[4], th = p[5];
    R sp, cp;
    sc(phi, &sp, &cp);
    const R kappa = -kb * w;
    const R A = x * cp + y * sp;
    const R r0 = sq(x * x + y * y);
    const R disc = A * A + (radius - r0) * (radius + r0);
    R s;
    if (kMode == kPropStep) {
        if (!(A > R(0)) || !(disc >= R(0))) return false;
        s = (radius - r0) * (radius + r0) / (A + sq(disc));
    } else if (kMode == kPropOut) {
        if (!(disc >= R(0))) return false;
        s = -A + sq(disc);
    } else if (disc >= R(0)) {
        s = -A - sq(disc);
    } else {
        if (!(ab(kappa) > R(0))) return false;
        const R ik = R(1) / kappa;
        const R cx = x - sp * ik, cy = y + cp * ik;  // centre of the track circle
        const R d2 = cx * cx + cy * cy, d = sq(d2);
        const R a = (radius * radius - ik * ik + d2) / (R(2) * d);  // chord's distance from the origin
        const R h2 = radius * radius - a * a;
        if (!(h2 >= R(0)) || !(d > R(0))) return false;
        const R h = sq(h2);
        const R ux = x - cx, uy = y - cy;  // p0 - c
        const R two_pi_rho = R(2.0 * kPi) * ab(ik);
        s = R(-1);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const R sg = k ? R(-1) : R(1);
            const R qx = (a * cx - sg * h * cy) / d - cx, qy = (a * cy + sg * h * cx) / d - cy;  // crossing - c
            R sk = at2(ux * qy - uy * qx, ux * qx + uy * qy) * ik;
            if (!(sk > R(0))) sk += two_pi_rho;
            if (s < R(0) || sk < s) s = sk;
        }
    }
    R S, C, Sd, Cd;
    // inward starts can be far from the crossing (a grazing entry, the circle intersection's
    // rounding): up to 3 newton + 2 steps.  The straight line's root of a crossing at more than
    // about 6 degrees from the tangent is as close as the outward start, and takes the outward
    // step count; any other start stops once a step moves s by less than Lim::converged of itself
    constexpr int n_newton = kMode == kPropIn ? 3 * Lim<R>::newton + 2 : Lim<R>::newton;
    const bool clear = disc > R(0.01) * radius * radius;
#pragma unroll
    for (int it = 0; it < n_newton; ++it) {
        const R a = kappa * s;
        helix_fn(a, S, C, Sd, Cd);
        const R sa = a * S, ca = R(1) - a * C;
        const R xs = x + s * (cp * S - sp * C);
        const R ys = y + s * (sp * S + cp * C);
        const R c1 = cp * ca - sp * sa, s1 = sp * ca + cp * sa;
        const R g = xs * xs + ys * ys - radius * radius;
        const R dg = R(2) * (xs * c1 + ys * s1);
        const R ds = g / dg;
        s -= ds;
        if (kMode == kPropIn && it + 1 >= Lim<R>::newton && (clear || ab(ds) <= Lim<R>::converged * ab(s))) break;
    }
    const R a = kappa * s;
    helix_fn(a, S, C, Sd, Cd);
    const R sa = a * S, ca = R(1) - a * C;
    const R xs = x + s * (cp * S - sp * C);
    const R ys = y + s * (sp * S + cp * C);
    const R c1 = cp * ca - sp * sa, s1 = sp * ca + cp * sa;
    const R D = xs * c1 + ys * s1;  // r dr/ds
    if (kMode == kPropStep ? !(D > R(1e-6) * radius) : (!(s > R(0)) || !(ab(D) > R(1e-6) * radius)))
        return false;
    if (!(ab(xs * xs + ys * ys - radius * radius) < R(1e-3) * radius)) return false;
    R st, ct;
    fast_sc(th, &st, &ct);
    const R cot = ct / st;

    // derivatives at fixed s
    const R s2kb = -kb * s * s;
    const R dx_dw = s2kb * (cp * Sd - sp * Cd);
    const R dy_dw = s2kb * (sp * Sd + cp * Cd);
    const R dx_dphi = -(ys - y), dy_dphi = xs - x;
    // ds/dp from r(s, p) = radius
    const R iD = R(1) / D;
    const R s_x = -xs * iD, s_y = -ys * iD;
    const R s_w = -(xs * dx_dw + ys * dy_dw) * iD;
    const R s_f = -(xs * dx_dphi + ys * dy_dphi) * iD;
    // Jacobian rows (non-trivial entries only)
    const R a0 = R(1) + c1 * s_x, a1 = c1 * s_y, a3 = dx_dw + c1 * s_w, a4 = dx_dphi + c1 * s_f;  // x
    const R b0 = s1 * s_x, b1 = R(1) + s1 * s_y, b3 = dy_dw + s1 * s_w, b4 = dy_dphi + s1 * s_f;  // y
    const R c0 = cot * s_x, cc1 = cot * s_y, c3 = cot * s_w, c4 = cot * s_f, c5 = -s / (st * st); // z (c2 = 1)
    const R f0 = kappa * s_x, f1 = kappa * s_y, f3 = -kb * s + kappa * s_w, f4 = R(1) + kappa * s_f; // phi

    // P' = J P J^T from J's sparsity pattern (generated: sparse_gen.cuh)
    R Q[21];
    transport_cov<R>(a0, a1, a3, a4, b0, b1, b3, b4, c0, cc1, c3, c4, c5, f0, f1, f3, f4, P, Q);
#pragma unroll
    for (int k = 0; k < 21; ++k) P[k] = Q[k];
    p[0] = xs;
    p[1] = ys;
    p[2] = z + s * cot;
    p[4] = wrap_phi(phi + a);
    return true;
}

// Propagation to the plane z = zp (an endcap disk, the "endcap z" of Sec. 2.2): from
// z(s) = z + s cot(theta) the transverse path is s = (zp - z) tan(theta) in closed form; the state
// is the helix there.  The Jacobian adds (dp/ds)(ds/dp_in) to the derivatives at fixed s, with
// ds/dz = -1/cot(theta) and ds/dtheta = s / (sin^2(theta) cot(theta)) from z(s, p_in) = zp (the
// path does not depend on x, y, q/pT, phi); P <- J P J^T from that sparsity (plane_cov).
// Returns false when the plane is behind, parallel, or more than a full turn away (a looper).
template <class R> __host__ __device__ __forceinline__ bool propagate_plane(R p[6], R P[21], R zp, R kb)
{
    const R x = p[0], y = p[1], z = p[2], w = p[3], phi = p[4], th = p[5];
    R st, ct;
    sc(th, &st, &ct);
    const R cot = ct / st;
    if (!(ab(cot) > R(0))) return false;
    const R s = (zp - z) / cot;
    const R kappa = -kb * w;
    if (!(s > R(0)) || !(ab(kappa) * s <= R(2.0 * kPi))) return false;
    R sp, cp;
    sc(phi, &sp, &cp);
    const R a = kappa * s;
    R S, C, Sd, Cd;
    helix_fn(a, S, C, Sd, Cd);
    const R sa = a * S, ca = R(1) - a * C;
    const R xs = x + s * (cp * S - sp * C);
    const R ys = y + s * (sp * S + cp * C);
    const R c1 = cp * ca - sp * sa, s1 = sp * ca + cp * sa;  // direction at the plane
    const R s2kb = -kb * s * s;
    const R dx_dw = s2kb * (cp * Sd - sp * Cd);
    const R dy_dw = s2kb * (sp * Sd + cp * Cd);
    const R sz = -R(1) / cot, sth = s / (st * st * cot);  // ds/dz, ds/dtheta
    R Q[21];
    plane_cov<R>(c1 * sz, dx_dw, -(ys - y), c1 * sth, s1 * sz, dy_dw, xs - x, s1 * sth, kappa * sz, -kb * s,
                 kappa * sth, P, Q);
#pragma unroll
    for (int k = 0; k < 21; ++k) P[k] = Q[k];
    p[0] = xs;
    p[1] = ys;
    p[2] = zp;
    p[4] = wrap_phi(phi + a);
    return true;
}

// ------------------------------------------------------------------ scattering noise
// Thin scatterer of thickness x/X0 crossed at angle alpha to the layer's normal: Highland
// width theta0 = 0.0136/(beta p) sqrt(t) (1 + 0.038 ln(t/beta^2)), t = (x/X0)/|cos alpha|;
// two kicks orthogonal to the direction add theta0^2 to theta, theta0^2/sin^2(theta) to phi,
// and (through pT = p sin(theta) at fixed p) the q/pT terms.
// disk: the layer is an endcap disk, whose normal is the z axis (|cos alpha| = |cos theta|).
template <class R>
__host__ __device__ __forceinline__ void scatter(const R p[6], R P[21], R xx0, R mass, bool disk = false)
{
    if (!(xx0 > R(0))) return;
    R st, ct, sp, cp;
    fast_sc(p[5], &st, &ct);
    fast_sc(p[4], &sp, &cp);
    const R w = p[3];
    const R mom = R(1) / (ab(w) * st);
    const R beta2 = mom * mom / (mom * mom + mass * mass);
    const R beta = sq(beta2);
    R cosa;
    if (disk) {
        cosa = ab(ct);
    } else {
        const R r = sq(p[0] * p[0] + p[1] * p[1]);
        cosa = ab(st * (p[0] * cp + p[1] * sp) / r);
    }
    const R t = xx0 / cosa;
    const R th0 = R(0.0136) / (beta * mom) * sq(t) * (R(1) + R(0.038) * fast_log(t / beta2));
    const R v = th0 * th0;
    const R cot = ct / st;
    P[sym(3, 3)] += w * w * cot * cot * v;
    P[sym(5, 3)] += -w * cot * v;
    P[sym(4, 4)] += v / (st * st);
    P[sym(5, 5)] += v;
}

// ------------------------------------------------------------------ measurement model
// Measurement on the plane tangent to the cylinder at the hit (Sec. 2.2): u along the tangent
// (-sin phi_h, cos phi_h, 0), v along z.  H = [[-s, c, 0, 0, 0, 0], [0, 0, 1, 0, 0, 0]].

// chi2 = r^T S^-1 r with S = H P H^T + V; returns +inf when S is not positive definite.
template <class R>
__host__ __device__ __forceinline__ R hit_chi2(const R p[6], const R P[21], R xh, R yh, R zh, R vu, R vv)
{
    const R ir = R(1) / sq(xh * xh + yh * yh);
    const R sh = yh * ir, ch = xh * ir;
    const R u = ch * (yh - p[1]) - sh * (xh - p[0]);
    const R v = zh - p[2];
    const R Suu = sh * (sh * P[sym(0, 0)] - ch * P[sym(1, 0)]) + ch * (ch * P[sym(1, 1)] - sh * P[sym(1, 0)]) + vu;
    const R Suv = ch * P[sym(2, 1)] - sh * P[sym(2, 0)];
    const R Svv = P[sym(2, 2)] + vv;
    const R det = Suu * Svv - Suv * Suv;
    if (!(det > R(0))) return R(INFINITY);
    return (u * (Svv * u - R(2) * Suv * v) + Suu * v * v) / det;
}

// chi2 = r^T S^-1 r from the residual (u, v) already formed with the hit's tangent
// (-sh, ch); returns +inf when S is not positive definite.
// The same from the six position terms of P it needs (P00, P10, P11, P20, P21, P22).
template <class R>
__host__ __device__ __forceinline__ R chi2_uv6(R p00, R p10, R p11, R p20, R p21, R p22, R u, R v, R sh, R ch, R vu,
                                               R vv)
{
    const R Suu = sh * (sh * p00 - ch * p10) + ch * (ch * p11 - sh * p10) + vu;
    const R Suv = ch * p21 - sh * p20;
    const R Svv = p22 + vv;
    const R det = Suu * Svv - Suv * Suv;
    if (!(det > R(0))) return R(INFINITY);
    return fast_div(u * (Svv * u - R(2) * Suv * v) + Suu * v * v, det);
}

// On an endcap disk (the hit measured in r-phi and r): rows u = (-sh, ch, 0) and
// v = (ch, sh, 0) of the x, y block of P; (u, v) already formed on the disk's plane.
template <class R>
__host__ __device__ __forceinline__ R chi2_disk(R p00, R p10, R p11, R u, R v, R sh, R ch, R vu, R vv)
{
    const R Suu = sh * (sh * p00 - ch * p10) + ch * (ch * p11 - sh * p10) + vu;
    const R Suv = sh * ch * (p11 - p00) + (ch * ch - sh * sh) * p10;
    const R Svv = ch * (ch * p00 + sh * p10) + sh * (sh * p11 + ch * p10) + vv;
    const R det = Suu * Svv - Suv * Suv;
    if (!(det > R(0))) return R(INFINITY);
    return fast_div(u * (Svv * u - R(2) * Suv * v) + Suu * v * v, det);
}

template <class R>
__host__ __device__ __forceinline__ R chi2_uv(const R P[21], R u, R v, R sh, R ch, R vu, R vv)
{
    return chi2_uv6<R>(P[sym(0, 0)], P[sym(1, 0)], P[sym(1, 1)], P[sym(2, 0)], P[sym(2, 1)], P[sym(2, 2)], u, v, sh,
                       ch, vu, vv);
}

// chi2 of a hit off the layer's cylinder (the two-step propagation of Sec. 2.2): the prediction
// p, P on the layer's average radius is carried along the helix to the hit's own radius rh
// (the kPropStep step of propagate), and the hit is compared there on its tangent plane
// (-sh, ch).  Only the two measured rows of the transported state are formed: M = H J (2x6),
// S = M P M^T + V.  sp, cp = sin, cos of phi; st = sin theta, cot = cot theta of p.
// Returns +inf when the step fails or S is not positive definite.
template <class R>
__host__ __device__ __forceinline__ R step_chi2(const R p[6], const R P[21], R sp, R cp, R st, R cot, R kb, R rh,
                                                R xh, R yh, R zh, R sh, R ch, R vu, R vv)
{
    const R x = p[0], y = p[1];
    const R kappa = -kb * p[3];
    const R A = x * cp + y * sp;
    const R r0 = sq(x * x + y * y);
    const R disc = A * A + (rh - r0) * (rh + r0);
    if (!(A > R(0)) || !(disc >= R(0))) return R(INFINITY);
    R s = (rh - r0) * (rh + r0) / (A + sq(disc));
    R S, C, Sd, Cd;
#pragma unroll
    for (int it = 0; it < Lim<R>::newton; ++it) {
        const R a = kappa * s;
        helix_fn(a, S, C, Sd, Cd);
        const R sa = a * S, ca = R(1) - a * C;
        const R xs = x + s * (cp * S - sp * C);
        const R ys = y + s * (sp * S + cp * C);
        const R c1 = cp * ca - sp * sa, s1 = sp * ca + cp * sa;
        s -= (xs * xs + ys * ys - rh * rh) / (R(2) * (xs * c1 + ys * s1));
    }
    const R a = kappa * s;
    helix_fn(a, S, C, Sd, Cd);
    const R sa = a * S, ca = R(1) - a * C;
    const R xs = x + s * (cp * S - sp * C);
    const R ys = y + s * (sp * S + cp * C);
    const R c1 = cp * ca - sp * sa, s1 = sp * ca + cp * sa;
    const R D = xs * c1 + ys * s1;
    if (!(D > R(1e-6) * rh) || !(ab(xs * xs + ys * ys - rh * rh) < R(1e-3) * rh)) return R(INFINITY);
    // rows x, y, z of the step's Jacobian (as in propagate)
    const R s2kb = -kb * s * s;
    const R dx_dw = s2kb * (cp * Sd - sp * Cd);
    const R dy_dw = s2kb * (sp * Sd + cp * Cd);
    const R dx_dphi = -(ys - y), dy_dphi = xs - x;
    const R iD = R(1) / D;
    const R s_x = -xs * iD, s_y = -ys * iD;
    const R s_w = -(xs * dx_dw + ys * dy_dw) * iD;
    const R s_f = -(xs * dx_dphi + ys * dy_dphi) * iD;
    // M row u = -sh (row x) + ch (row y), over columns x, y, q/pT, phi; row v = row z
    const R m0 = -sh * (R(1) + c1 * s_x) + ch * (s1 * s_x);
    const R m1 = -sh * (c1 * s_y) + ch * (R(1) + s1 * s_y);
    const R m3 = -sh * (dx_dw + c1 * s_w) + ch * (dy_dw + s1 * s_w);
    const R m4 = -sh * (dx_dphi + c1 * s_f) + ch * (dy_dphi + s1 * s_f);
    const R v0 = cot * s_x, v1 = cot * s_y, v3 = cot * s_w, v4 = cot * s_f, v5 = -s / (st * st);
    R Sm[3];  // M P M^T from M's sparsity pattern (generated: sparse_gen.cuh)
    measured_cov<R>(m0, m1, m3, m4, v0, v1, v3, v4, v5, P, Sm);
    const R Suu = Sm[0] + vu, Suv = Sm[1], Svv = Sm[2] + vv;
    const R u = ch * (yh - ys) - sh * (xh - xs);
    const R v = zh - (p[2] + s * cot);
    const R det = Suu * Svv - Suv * Suv;
    if (!(det > R(0))) return R(INFINITY);
    return fast_div(u * (Svv * u - R(2) * Suv * v) + Suu * v * v, det);
}

// ------------------------------------------------------------------ float <-> double without the FP64 unit
// (ieee_cvt.cuh): the mixed-precision update converts with integer operations on the bit fields.
#ifndef TKF_INT_CVT
#define TKF_INT_CVT 1
#endif

// cvt_up<U>(x): x (float or double) as U; cvt_down<R>(x): x (double) as R (float or double).
template <class U> __device__ __forceinline__ U cvt_up(float x)
{
#if TKF_INT_CVT
    if constexpr (sizeof(U) == 8) return f32_to_f64_bits(x);
#endif
    return U(x);
}
template <class U> __device__ __forceinline__ U cvt_up(double x) { return U(x); }
template <class R> __device__ __forceinline__ R cvt_down(float x) { return R(x); }
template <class R> __device__ __forceinline__ R cvt_down(double x)
{
#if TKF_INT_CVT
    if constexpr (sizeof(R) == 4) return f64_to_f32_bits(x);
#endif
    return R(x);
}

// 1/x for x > 0: in float the approximate division; in double Newton's iteration for the
// reciprocal, y <- y (2 - x y) written as y + y (1 - x y), from the correctly rounded
// single-precision reciprocal of x rounded to float (relative error below 2^-23; each step
// squares it, so two steps reach double rounding) -- four double operations where the IEEE
// division takes about three times as many on the scarce double-precision units.  An x outside
// the float range takes the IEEE division.
template <class U> __device__ __forceinline__ U recip(U x) { return U(1) / x; }
template <> __device__ __forceinline__ double recip<double>(double x)
{
#if TKF_INT_CVT
    const float xf = f64_to_f32_bits(x);
    const float yf = __frcp_rn(xf);
    if (!(xf > 1e-37f && xf < 1e37f)) return 1.0 / x;
    double y = f32_to_f64_bits(yf);
    y = fma(y, fma(-x, y, 1.0), y);
    y = fma(y, fma(-x, y, 1.0), y);
    return y;
#else
    return 1.0 / x;
#endif
}

// Kalman update with the Joseph-form covariance:
//   B = H P (2x6), S = B H^T + V, K = B^T S^-1, p += K r,
//   P' = (I - K H) P (I - K H)^T + K V K^T = P - K B - (B^T - K S) K^T   (element-wise below).
// The measurement geometry (the hit's tangent direction and the residual r on its plane) is
// formed in the state's type R; S, its inverse, the gain, the state update and the Joseph form
// are computed in U (double in the mixed mode).  Returns false when S is not positive definite;
// writes the hit's chi2 to *chi2.
// kDisk: the hit lies on an endcap disk and is measured on the disk's plane: the second row of
// H is the radial direction (cos phi_h, sin phi_h, 0) instead of z.
template <class U, class R, bool kDisk = false>
__device__ __forceinline__ bool kalman_update(R pR[6], R PR[21], R xh_, R yh_, R zh_, R vu_, R vv_, U *chi2)
{
    const R irR = R(1) / sq(xh_ * xh_ + yh_ * yh_);
    const R shR = yh_ * irR, chR = xh_ * irR;
    const R uR = chR * (yh_ - pR[1]) - shR * (xh_ - pR[0]);
    const R vR = kDisk ? chR * (xh_ - pR[0]) + shR * (yh_ - pR[1]) : zh_ - pR[2];
    const U u = cvt_up<U>(uR), v = cvt_up<U>(vR);
    const U sh = cvt_up<U>(shR), ch = cvt_up<U>(chR);
    U P[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) P[k] = cvt_up<U>(PR[k]);
    U B0[6], B1[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        B0[j] = ch * P[sym(1, j)] - sh * P[sym(0, j)];
        B1[j] = kDisk ? ch * P[sym(0, j)] + sh * P[sym(1, j)] : P[sym(2, j)];
    }
    const U Suu = ch * B0[1] - sh * B0[0] + cvt_up<U>(vu_);
    const U Suv = kDisk ? ch * B0[0] + sh * B0[1] : B0[2];
    const U Svv = (kDisk ? ch * B1[0] + sh * B1[1] : B1[2]) + cvt_up<U>(vv_);
    const U det = Suu * Svv - Suv * Suv;
    if (!(det > U(0))) return false;
    const U id = recip<U>(det);
    const U i00 = Svv * id, i01 = -Suv * id, i11 = Suu * id;
    *chi2 = u * (i00 * u + i01 * v) + v * (i01 * u + i11 * v);
    U K0[6], K1[6], D0[6], D1[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        K0[i] = B0[i] * i00 + B1[i] * i01;
        K1[i] = B0[i] * i01 + B1[i] * i11;
        D0[i] = fma(-K1[i], Suv, fma(-K0[i], Suu, B0[i]));
        D1[i] = fma(-K1[i], Svv, fma(-K0[i], Suv, B1[i]));
    }
    // state update in the state's type (the gain rounded to it)
#pragma unroll
    for (int i = 0; i < 6; ++i) pR[i] = pR[i] + cvt_down<R>(K0[i]) * uR + cvt_down<R>(K1[i]) * vR;
    pR[4] = wrap_phi(pR[4]);
    // Joseph form, element by element: P - (K B + D K^T) in one fused chain
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            U t = K0[i] * B0[j];
            t = fma(K1[i], B1[j], t);
            t = fma(D0[i], K0[j], t);
            t = fma(D1[i], K1[j], t);
            PR[sym(i, j)] = cvt_down<R>(P[sym(i, j)] - t);
        }
    return true;
}

}  // namespace tkf
