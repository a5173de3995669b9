/*
 * ORACLE -- test infrastructure only.  A plain, slow, single-threaded FP64 restatement of
 * the Kalman-filter track fit and combinatorial track building described in Cerati et al.,
 * "Kalman filter tracking on parallel architectures" (arXiv:1702.06359).  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg load this file; the product
 * path never does.  It shares no code, header or table with the CUDA library.
 *
 * Everything is written in the textbook form with full 6x6 / 2x6 / 2x2 matrices so that it
 * can be checked against the equations by eye; no sparsity is exploited.
 *
 * State p = (x, y, z, q/pT, phi, theta): global Cartesian position plus polar momentum, the
 * hybrid coordinates of Sec. 2.2.  Units cm, GeV, T, rad.
 *
 * Where the paper is silent, the readings below are used (each is listed with its reason in
 * the design notes of the repository):
 *   - propagation to a barrel cylinder is the exact helix/cylinder intersection (Sec. 2.2,
 *     ideal barrel, uniform Bz), one step, smallest positive transverse path;
 *   - the measurement is made on the plane tangent to the cylinder at the hit (Sec. 2.2):
 *     u = rphi offset along the tangent, v = z offset;
 *   - thin-layer multiple scattering with the Highland width, added after the update of a
 *     layer, except on the outermost layer;
 *   - building: window = chi2-cut bounding box of S, one hole branch per parent that finds
 *     no compatible hit, branches ranked by (nHits desc, chi2 asc, parent rank asc, hit id
 *     asc), best N kept (Sec. 2: "branching to explore multiple candidate tracks per seed");
 *     a hit is compatible if it lies on the same half of the cylinder as the prediction and
 *     its chi2 is below the cut;
 *   - hits off their layer's cylinder (hit_dr > 0, the simplified CMS geometry of Sec. 2.2):
 *     a layer's hit is reached by the exact propagation from the previous layer to the hit's
 *     own radius, and the update is made on the plane tangent there.  In building, the window
 *     is opened around the prediction on the layer's average radius, its half-widths grown by
 *     how far the track moves along the cylinder and in z while its radius changes by hit_dr;
 *     a hit is a candidate if its residual to that prediction lies inside the window; its
 *     chi2 is then taken at its own radius.  (The paper's second, per-hit propagation starts
 *     from the prediction on the average radius; the two transports compose to this one.)
 *   - endcap disks (disk_z[l] > 0; the "endcap z" of Sec. 2.2): a layer is a pair of planes
 *     z = +-disk_z[l]; a state goes to the one on the side of its z by the exact helix/plane
 *     intersection; a disk hit is measured on the disk's plane in r-phi (u, along the tangent
 *     (-sin phi_h, cos phi_h, 0)) and r (v, along (cos phi_h, sin phi_h, 0)); the window is the
 *     chi2-cut box in (u, v) mapped to phi and to the eta bins of the radii it spans, eta of a
 *     disk hit being asinh(z / r_hit); a compatible hit lies on the disk the state reached (not
 *     the opposite endcap's, which the (u, v) measurement alone cannot tell apart).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "tkf_oracle.h"

#define NPAR 6
static const double ORC_KB = 0.00299792458; /* GeV / (T cm) */
static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ small matrix helpers */

static void mat_mul(int n, int m, int k, const double *A, const double *B, double *C)
{ /* C[n x k] = A[n x m] B[m x k], all row-major */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < k; ++j) {
            double s = 0.0;
            for (int t = 0; t < m; ++t) s += A[i * m + t] * B[t * k + j];
            C[i * k + j] = s;
        }
}

static void mat_transpose(int n, int m, const double *A, double *At)
{ /* At[m x n] = A[n x m]^T */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) At[j * n + i] = A[i * m + j];
}

/* C = A P A^T for square 6x6 A, P */
static void sandwich6(const double *A, const double *P, double *C)
{
    double AP[36], At[36];
    mat_mul(6, 6, 6, A, P, AP);
    mat_transpose(6, 6, A, At);
    mat_mul(6, 6, 6, AP, At, C);
    for (int i = 0; i < 6; ++i) /* the product is symmetric; remove rounding asymmetry */
        for (int j = 0; j < i; ++j) {
            const double m = 0.5 * (C[i * 6 + j] + C[j * 6 + i]);
            C[i * 6 + j] = m; C[j * 6 + i] = m;
        }
}

static double wrap_phi(double phi)
{ /* into [-pi, pi) */
    while (phi >= ORC_PI) phi -= 2.0 * ORC_PI;
    while (phi < -ORC_PI) phi += 2.0 * ORC_PI;
    return phi;
}

/* ------------------------------------------------------------------ propagation (Sec. 2.2) */

/* sin(x)/x and its derivative, written so that nothing cancels near x = 0 (the series are
 * used where their first omitted term is below 1e-17). */
static double sinc(double x) { return fabs(x) < 1e-4 ? 1.0 - x * x / 6.0 : sin(x) / x; }
static double dsinc(double x)
{
    return fabs(x) < 1e-3 ? -x / 3.0 + x * x * x / 30.0 : (x * cos(x) - sin(x)) / (x * x);
}

/*
 * Exact propagation of a helix in a uniform field Bz to the cylinder r = R.
 * Helix with curvature kappa = -K_B Bz q/pT (signed d phi / d s_T), s_T the transverse path:
 *   x(s) = x0 + (sin(phi0 + kappa s) - sin phi0) / kappa = x0 + s cos(phi0 + kappa s/2) sinc(kappa s/2)
 *   y(s) = y0 - (cos(phi0 + kappa s) - cos phi0) / kappa = y0 + s sin(phi0 + kappa s/2) sinc(kappa s/2)
 *   z(s) = z0 + s cot(theta),  phi(s) = phi0 + kappa s,
 * the right-hand forms following from sin a - sin b = 2 cos((a+b)/2) sin((a-b)/2) and
 * cos a - cos b = -2 sin((a+b)/2) sin((a-b)/2); they stay exact as kappa -> 0.
 * The crossing is the intersection of the circle |x| = R with the track circle, centre
 * c = p0 + n0/kappa (n0 = (-sin phi0, cos phi0)), radius rho = 1/|kappa|: with
 * d = |c| the chord lies at distance a = (R^2 - rho^2 + d^2)/(2d) from the origin along c, and
 * d^2 - rho^2 = r0^2 + 2 (p0 . n0)/kappa.  The turning angle from p0 to a crossing p (seen from
 * c, counter-clockwise) is atan2(v0 x v1, v0 . v1) with v0 = -n0/kappa, v1 = (p - p0) - n0/kappa;
 * multiplying both arguments by kappa^2 > 0 gives atan2(-kappa n0 x dp, 1 - kappa n0 . dp).
 * The smallest positive turning angle in the direction of motion gives s = angle / |kappa|.
 * The transport Jacobian J = dp_out/dp_in is the analytic derivative at fixed s plus
 * (dp_out/ds)(ds/dp_in), with ds/dp_in = -(dr/dp_in)/(dr/ds) from the constraint r(s, p_in) = R.
 */
static int helix_at(const orc_geom *g, const double pin[6], double s, int plane, double pout[6], double J[36]);

int orc_propagate(const orc_geom *g, const double pin[6], double R, double pout[6], double J[36])
{
    const double x0 = pin[0], y0 = pin[1], w = pin[3], phi0 = pin[4];
    const double kappa = -ORC_KB * g->bz * w;
    const double nx = -sin(phi0), ny = cos(phi0);
    double s;

    if (fabs(kappa) < 1e-12) { /* straight line: |p0 + s u|^2 = R^2 */
        const double ux = cos(phi0), uy = sin(phi0);
        const double b = x0 * ux + y0 * uy;
        const double disc = b * b - (x0 * x0 + y0 * y0 - R * R);
        if (disc < 0.0) return ORC_ERR_NOREACH;
        s = -b + sqrt(disc);
        if (!(s > 0.0)) return ORC_ERR_NOREACH;
    } else {
        const double cx = x0 + nx / kappa, cy = y0 + ny / kappa;
        const double d = sqrt(cx * cx + cy * cy);
        if (d == 0.0) return ORC_ERR_NOREACH;
        const double r02 = x0 * x0 + y0 * y0, B = x0 * nx + y0 * ny;
        const double a = (R * R + r02 + 2.0 * B / kappa) / (2.0 * d);
        const double h2 = R * R - a * a;
        if (h2 < 0.0) return ORC_ERR_NOREACH;
        const double h = sqrt(h2);
        const double ex = cx / d, ey = cy / d;
        double best = -1.0;
        for (int sign = -1; sign <= 1; sign += 2) {
            const double px = a * ex - sign * h * ey, py = a * ey + sign * h * ex;
            const double dx = px - x0, dy = py - y0;
            double ang = atan2(-kappa * (nx * dy - ny * dx), 1.0 - kappa * (nx * dx + ny * dy)); /* ccw */
            if (kappa < 0.0) ang = -ang;                                                        /* direction of motion */
            if (ang <= 0.0) ang += 2.0 * ORC_PI;                                                 /* into (0, 2 pi] */
            const double st = ang / fabs(kappa);
            if (st > 0.0 && (best < 0.0 || st < best)) best = st;
        }
        if (best < 0.0) return ORC_ERR_NOREACH;
        s = best;
    }

    return helix_at(g, pin, s, 0, pout, J);
}

/*
 * The state at transverse path s along the helix of pin, and the transport Jacobian for a
 * crossing defined by the constraint c(s, p_in) = 0 with c = r - R (plane = 0: a cylinder) or
 * c = z - Zp (plane = 1): J = dp_out/dp_in at fixed s plus (dp_out/ds)(ds/dp_in), with
 * ds/dp_in = -(dc/dp_in)/(dc/ds).
 */
static int helix_at(const orc_geom *g, const double pin[6], double s, int plane, double pout[6], double J[36])
{
    const double x0 = pin[0], y0 = pin[1], z0 = pin[2], w = pin[3], phi0 = pin[4], th = pin[5];
    const double kappa = -ORC_KB * g->bz * w;
    const double cot_th = cos(th) / sin(th);
    const double half = 0.5 * kappa * s, mid = phi0 + half;
    const double sn = sinc(half);
    const double x1 = x0 + s * cos(mid) * sn;
    const double y1 = y0 + s * sin(mid) * sn;
    const double phi1 = phi0 + kappa * s;
    const double z1 = z0 + s * cot_th;
    pout[0] = x1; pout[1] = y1; pout[2] = z1; pout[3] = w; pout[4] = wrap_phi(phi1); pout[5] = th;

    if (!J) return ORC_OK;

    /* partial derivatives at fixed s: F[i][j] = d pout_i / d pin_j */
    double F[36];
    memset(F, 0, sizeof F);
    for (int i = 0; i < 6; ++i) F[i * 6 + i] = 1.0;
    const double dkdw = -ORC_KB * g->bz;
    const double dsn = dsinc(half);
    /* d/dkappa of s cos(mid) sinc(half) with d mid/d kappa = d half/d kappa = s/2 */
    const double dx_dk = s * (-sin(mid) * 0.5 * s * sn + cos(mid) * dsn * 0.5 * s);
    const double dy_dk = s * (cos(mid) * 0.5 * s * sn + sin(mid) * dsn * 0.5 * s);
    F[0 * 6 + 4] = -(y1 - y0);
    F[1 * 6 + 4] = x1 - x0;
    F[0 * 6 + 3] = dx_dk * dkdw;
    F[1 * 6 + 3] = dy_dk * dkdw;
    F[2 * 6 + 5] = -s / (sin(th) * sin(th));
    F[4 * 6 + 3] = s * dkdw;

    /* derivative along the path */
    double dp_ds[6] = {cos(phi1), sin(phi1), cot_th, 0.0, kappa, 0.0};
    double ds_dp[6];
    if (plane) {
        /* constraint z = Zp:  ds/dp_j = -(dz/dp_j) / (dz/ds) */
        if (cot_th == 0.0) return ORC_ERR_NOREACH;
        for (int j = 0; j < 6; ++j) ds_dp[j] = -F[2 * 6 + j] / cot_th;
    } else {
        /* constraint r^2 = x^2 + y^2 = R^2:  ds/dp_j = -(x dx/dp_j + y dy/dp_j) / (x dx/ds + y dy/ds) */
        const double drds = x1 * dp_ds[0] + y1 * dp_ds[1];
        if (drds == 0.0) return ORC_ERR_NOREACH;
        for (int j = 0; j < 6; ++j) ds_dp[j] = -(x1 * F[0 * 6 + j] + y1 * F[1 * 6 + j]) / drds;
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) J[i * 6 + j] = F[i * 6 + j] + dp_ds[i] * ds_dp[j];
    return ORC_OK;
}

/*
 * Exact propagation of the helix to the plane z = Zp (an endcap disk, Sec. 2.2): z(s) =
 * z0 + s cot(theta) = Zp gives s = (Zp - z0) tan(theta), which must be positive (the plane lies
 * ahead); the state there is the helix at that s.  A track that would turn through more than a
 * full circle before reaching the plane (a looper) does not reach it.
 */
int orc_propagate_plane(const orc_geom *g, const double pin[6], double Zp, double pout[6], double J[36])
{
    const double th = pin[5];
    const double cot_th = cos(th) / sin(th);
    if (cot_th == 0.0) return ORC_ERR_NOREACH;
    const double s = (Zp - pin[2]) / cot_th;
    if (!(s > 0.0)) return ORC_ERR_NOREACH;
    if (!(fabs(ORC_KB * g->bz * pin[3]) * s <= 2.0 * ORC_PI)) return ORC_ERR_NOREACH;
    const int st = helix_at(g, pin, s, 1, pout, J);
    pout[2] = Zp; /* z0 + s cot(theta) is the plane up to rounding */
    return st;
}

/* ------------------------------------------------------------------ multiple scattering */

/*
 * Thin-scatterer process noise at layer l (Highland width, unit charge, mass hypothesis m):
 *   theta0 = 0.0136/(beta p) sqrt(t) (1 + 0.038 ln(t / beta^2)),  t = (x/X0) / |cos alpha|,
 * alpha the angle between the direction and the layer's normal (radial on a cylinder, z on
 * a disk).  Two independent kicks of
 * width theta0 orthogonal to the direction change theta by d1 and phi by d2/sin(theta); with
 * |p| fixed, q/pT changes by -(q/pT) cot(theta) d1.
 */
void orc_scatter(const orc_geom *g, int layer, const double p[6], double P[36])
{
    const double xt = g->x_over_x0[layer];
    if (xt <= 0.0) return;
    const double w = p[3], phi = p[4], th = p[5];
    const double mom = 1.0 / (fabs(w) * sin(th));
    const double beta = mom / sqrt(mom * mom + g->mass * g->mass);
    const double r = sqrt(p[0] * p[0] + p[1] * p[1]);
    const double d[3] = {sin(th) * cos(phi), sin(th) * sin(phi), cos(th)};
    const int disk = g->disk_z[layer] > 0.0;                        /* a disk's normal is the z axis */
    const double nrm[3] = {disk ? 0.0 : p[0] / r, disk ? 0.0 : p[1] / r, disk ? 1.0 : 0.0};
    const double cos_a = fabs(d[0] * nrm[0] + d[1] * nrm[1] + d[2] * nrm[2]);
    const double t = xt / cos_a;
    const double th0 = 0.0136 / (beta * mom) * sqrt(t) * (1.0 + 0.038 * log(t / (beta * beta)));
    const double v = th0 * th0;
    const double cot = cos(th) / sin(th);
    /* Jacobian of (w, phi, theta) w.r.t. the two kick angles (d1 along e_theta, d2 along e_phi) */
    double G[6][2] = {{0, 0}, {0, 0}, {0, 0}, {-w * cot, 0}, {0, 1.0 / sin(th)}, {1.0, 0}};
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) P[i * 6 + j] += v * (G[i][0] * G[j][0] + G[i][1] * G[j][1]);
}

/* ------------------------------------------------------------------ Kalman update (Sec. 2.2) */

/* Measurement model on the plane tangent to the cylinder at the hit: rows of H are the
 * tangent direction (-sin phi_h, cos phi_h, 0) and the z axis.  On an endcap disk the plane is
 * the disk's own: rows (-sin phi_h, cos phi_h, 0) (r-phi) and the radial direction
 * (cos phi_h, sin phi_h, 0) (r). */
static void meas_model(const double p[6], const orc_hit *h, double H[12], double r[2], double V[4])
{
    const double ph = atan2(h->y, h->x);
    const double sh = sin(ph), ch = cos(ph);
    memset(H, 0, 12 * sizeof(double));
    H[0] = -sh; H[1] = ch;
    r[0] = -sh * (h->x - p[0]) + ch * (h->y - p[1]);
    if (h->disk) {
        H[6 + 0] = ch; H[6 + 1] = sh;
        r[1] = ch * (h->x - p[0]) + sh * (h->y - p[1]);
    } else {
        H[6 + 2] = 1.0;
        r[1] = h->z - p[2];
    }
    V[0] = h->var_u; V[1] = 0.0; V[2] = 0.0; V[3] = h->var_v;
}

static int innovation(const double P[36], const double H[12], const double V[4], double S[4], double Si[4])
{
    double Ht[12], PHt[12];
    mat_transpose(2, 6, H, Ht);
    mat_mul(6, 6, 2, P, Ht, PHt);
    mat_mul(2, 6, 2, H, PHt, S);
    for (int i = 0; i < 4; ++i) S[i] += V[i];
    const double det = S[0] * S[3] - S[1] * S[2];
    if (!(det > 0.0)) return ORC_ERR_SINGULAR;
    Si[0] = S[3] / det; Si[1] = -S[1] / det; Si[2] = -S[2] / det; Si[3] = S[0] / det;
    return ORC_OK;
}

double orc_chi2(const double p[6], const double P[36], const orc_hit *h)
{
    double H[12], r[2], V[4], S[4], Si[4];
    meas_model(p, h, H, r, V);
    if (innovation(P, H, V, S, Si) != ORC_OK) return INFINITY;
    return r[0] * (Si[0] * r[0] + Si[1] * r[1]) + r[1] * (Si[2] * r[0] + Si[3] * r[1]);
}

/*
 * Kalman update with the Joseph-form covariance:
 *   S = H P H^T + V,  K = P H^T S^-1,  p <- p + K r,
 *   P <- (I - K H) P (I - K H)^T + K V K^T,  chi2 = r^T S^-1 r (predicted S).
 */
int orc_update(double p[6], double P[36], const orc_hit *h, double *chi2)
{
    double H[12], r[2], V[4], S[4], Si[4];
    meas_model(p, h, H, r, V);
    int st = innovation(P, H, V, S, Si);
    if (st != ORC_OK) return st;
    double Ht[12], PHt[12], K[12];
    mat_transpose(2, 6, H, Ht);
    mat_mul(6, 6, 2, P, Ht, PHt);
    mat_mul(6, 2, 2, PHt, Si, K);
    if (chi2) *chi2 = r[0] * (Si[0] * r[0] + Si[1] * r[1]) + r[1] * (Si[2] * r[0] + Si[3] * r[1]);
    for (int i = 0; i < 6; ++i) p[i] += K[i * 2 + 0] * r[0] + K[i * 2 + 1] * r[1];
    p[4] = wrap_phi(p[4]);

    double KH[36], A[36], APAt[36], KV[12], Kt[12], KVKt[36];
    mat_mul(6, 2, 6, K, H, KH);
    for (int i = 0; i < 36; ++i) A[i] = -KH[i];
    for (int i = 0; i < 6; ++i) A[i * 6 + i] += 1.0;
    sandwich6(A, P, APAt);
    mat_mul(6, 2, 2, K, V, KV);
    mat_transpose(6, 2, K, Kt);
    mat_mul(6, 2, 6, KV, Kt, KVKt);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) P[i * 6 + j] = APAt[i * 6 + j] + KVKt[i * 6 + j];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < i; ++j) {
            const double m = 0.5 * (P[i * 6 + j] + P[j * 6 + i]);
            P[i * 6 + j] = m; P[j * 6 + i] = m;
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------ seed estimate */

/*
 * Initial state from three hits (the seeding stage of Sec. 2): the circle through the
 * three (x, y) points gives the curvature and the charge sign, phi is the tangent at the
 * first hit in the direction of motion, cot(theta) = (z3 - z1) / (transverse arc 1->3),
 * and the position is the first hit.  Prior covariance is diagonal (g->prior_sigma).
 */
int orc_seed_estimate(const orc_geom *g, const orc_hit *h1, const orc_hit *h2, const orc_hit *h3,
                      double p[6], double P[36])
{
    const double x1 = h1->x, y1 = h1->y, x2 = h2->x, y2 = h2->y, x3 = h3->x, y3 = h3->y;
    const double D = 2.0 * (x1 * (y2 - y3) + x2 * (y3 - y1) + x3 * (y1 - y2));
    double kappa, phi, s13;
    if (D == 0.0) { /* collinear: straight line */
        kappa = 0.0;
        phi = atan2(y3 - y1, x3 - x1);
        s13 = hypot(x3 - x1, y3 - y1);
    } else {
        const double n1 = x1 * x1 + y1 * y1, n2 = x2 * x2 + y2 * y2, n3 = x3 * x3 + y3 * y3;
        const double cx = (n1 * (y2 - y3) + n2 * (y3 - y1) + n3 * (y1 - y2)) / D;
        const double cy = (n1 * (x3 - x2) + n2 * (x1 - x3) + n3 * (x2 - x1)) / D;
        const double rho = hypot(x1 - cx, y1 - cy);
        const double turn = (x2 - x1) * (y3 - y2) - (y2 - y1) * (x3 - x2);
        const int ccw = turn > 0.0;
        kappa = (ccw ? 1.0 : -1.0) / rho;
        const double r1x = x1 - cx, r1y = y1 - cy, r3x = x3 - cx, r3y = y3 - cy;
        const double tx = ccw ? -r1y : r1y, ty = ccw ? r1x : -r1x;
        phi = atan2(ty, tx);
        double ang = atan2(r1x * r3y - r1y * r3x, r1x * r3x + r1y * r3y);
        if (!ccw) ang = -ang;
        if (ang <= 0.0) ang += 2.0 * ORC_PI;
        s13 = ang * rho;
    }
    const double cot = (h3->z - h1->z) / s13;
    p[0] = x1; p[1] = y1; p[2] = h1->z;
    p[3] = -kappa / (ORC_KB * g->bz);
    p[4] = wrap_phi(phi);
    p[5] = atan2(1.0, cot);
    memset(P, 0, 36 * sizeof(double));
    for (int i = 0; i < 6; ++i) P[i * 6 + i] = g->prior_sigma[i] * g->prior_sigma[i];
    if (h1->disk) P[2 * 6 + 2] = 0.0; /* on an endcap disk z is the disk's, known exactly */
    return ORC_OK;
}

/* The cylinder a layer's state is taken to: the hit's own radius when hits lie off the
 * layers' cylinders (hit_dr > 0) and the layer has a hit, else the layer's radius. */
static double target_radius(const orc_geom *g, int layer, const orc_hit *h)
{
    return (g->hit_dr > 0.0 && h) ? sqrt(h->x * h->x + h->y * h->y) : g->radius[layer];
}

/* Propagation to layer l: its cylinder (at target_radius), or for an endcap layer the disk on
 * the side of the state's z (states between two disks of one side stay on that side). */
static int propagate_layer(const orc_geom *g, int layer, const double p[6], const orc_hit *h, double q[6],
                           double J[36])
{
    if (g->disk_z[layer] > 0.0)
        return orc_propagate_plane(g, p, p[2] >= 0.0 ? g->disk_z[layer] : -g->disk_z[layer], q, J);
    return orc_propagate(g, p, target_radius(g, layer, h), q, J);
}

/* ------------------------------------------------------------------ fit (Sec. 2) */

/*
 * Kalman fit of one track over layers first..last with a known hit per layer (-1 = none):
 * the state starts on layer `first` (no propagation there); each later layer is reached by
 * exact propagation; the hit (if any) is added by the Kalman update; scattering noise of the
 * layer follows unless it is the outermost layer of the detector.
 */
int orc_fit_track(const orc_geom *g, const double pin[6], const double Pin[36], const orc_hit *hits,
                  const int *hit_of_layer, int first, int last, double pout[6], double Pout[36],
                  double *chi2, int *nhits)
{
    double p[6], P[36], J[36], q[6], PJ[36];
    memcpy(p, pin, sizeof p);
    memcpy(P, Pin, sizeof P);
    double c2 = 0.0;
    int nh = 0;
    for (int l = first; l <= last; ++l) {
        const int hid = hit_of_layer[l];
        if (l > first) {
            int st = propagate_layer(g, l, p, hid >= 0 ? &hits[hid] : 0, q, J);
            if (st != ORC_OK) return st;
            sandwich6(J, P, PJ);
            memcpy(p, q, sizeof p);
            memcpy(P, PJ, sizeof P);
        }
        if (hid >= 0) {
            double dc2;
            int st = orc_update(p, P, &hits[hid], &dc2);
            if (st != ORC_OK) return st;
            c2 += dc2;
            nh += 1;
        }
        if (l < g->n_layers - 1) orc_scatter(g, l, p, P);
    }
    memcpy(pout, p, sizeof p);
    memcpy(Pout, P, sizeof P);
    if (chi2) *chi2 = c2;
    if (nhits) *nhits = nh;
    return ORC_OK;
}

/* ------------------------------------------------------------------ backward pass (Sec. 2: final fit) */

/*
 * Inward Kalman filter over a track's hit list from layer `last` down to layer `first`
 * (first <= last), refining the final fit's estimate towards the production point.  The state
 * on layer `last` (typically the forward fit's result there) is taken with its covariance
 * multiplied by cov_scale (>= 1: the forward information is mostly discounted, so the pass is
 * nearly an independent fit in the opposite direction); then, layer by layer from `last` inward:
 * the update with the layer's hit, the layer's material (the scattering kick that the forward
 * fit adds on its way out of the layer), the propagation to the next smaller cylinder.  The
 * result lies on layer `first` after its update and its material: the state on the track
 * segment just inside that layer, which on layer 0 is the track as it left the production
 * region (the generator's truth there, taken before the layer's kick); chi2 and nhits are the
 * backward pass's own.
 *
 * Inward propagation is the outward propagation of the reversed track: the map
 * (x, y, z, q/pT, phi, theta) -> (x, y, z, -q/pT, phi + pi, pi - theta) describes the same helix
 * run backwards (transverse path s -> -s: the centre and radius of the track circle stay, the
 * direction of motion flips), so the first crossing of the smaller cylinder along the reversed
 * track is the previous crossing of the original one.  The map is its own inverse with the
 * diagonal Jacobian D = diag(1, 1, 1, -1, 1, -1) (covariance D P D); the measurement depends on
 * the position only, and the scattering noise of the reversed state is D Q D (its q/pT-theta
 * term is odd in both), so the update and the scattering apply unchanged to the reversed state.
 */
static void reverse_track(const double a[6], double b[6])
{
    b[0] = a[0];
    b[1] = a[1];
    b[2] = a[2];
    b[3] = -a[3];
    b[4] = a[4] > 0.0 ? a[4] - ORC_PI : a[4] + ORC_PI;
    b[5] = ORC_PI - a[5];
}

static void reverse_cov(const double A[36], double s, double B[36])
{
    static const double D[6] = {1.0, 1.0, 1.0, -1.0, 1.0, -1.0};
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) B[i * 6 + j] = s * D[i] * D[j] * A[i * 6 + j];
}

int orc_fit_backward(const orc_geom *g, const double pin[6], const double Pin[36], double cov_scale,
                     const orc_hit *hits, const int *hit_of_layer, int last, int first, double pout[6],
                     double Pout[36], double *chi2, int *nhits)
{
    double p[6], P[36], J[36], q[6], PJ[36];
    if (first < 0 || last < first || last >= g->n_layers || !(cov_scale > 0.0)) return ORC_ERR_INVALID;
    reverse_track(pin, p);
    reverse_cov(Pin, cov_scale, P);
    double c2 = 0.0;
    int nh = 0;
    for (int l = last; l >= first; --l) {
        const int hid = hit_of_layer[l];
        if (l < last) {
            int st = propagate_layer(g, l, p, hid >= 0 ? &hits[hid] : 0, q, J);
            if (st != ORC_OK) return st;
            sandwich6(J, P, PJ);
            memcpy(p, q, sizeof p);
            memcpy(P, PJ, sizeof P);
        }
        if (hid >= 0) {
            double dc2;
            int st = orc_update(p, P, &hits[hid], &dc2);
            if (st != ORC_OK) return st;
            c2 += dc2;
            nh += 1;
        }
        orc_scatter(g, l, p, P);
    }
    reverse_track(p, pout);
    reverse_cov(P, 1.0, Pout);
    if (chi2) *chi2 = c2;
    if (nhits) *nhits = nh;
    return ORC_OK;
}

int orc_fit_backward_batch(const orc_geom *g, const orc_hit *hits, int n, const double *par_in,
                           const double *cov_in, double cov_scale, const int *hit_ids, int last, int first,
                           double *par_out, double *cov_out, double *chi2, int *nhits, int *status)
{
    for (int i = 0; i < n; ++i)
        status[i] = orc_fit_backward(g, par_in + 6 * i, cov_in + 36 * i, cov_scale, hits,
                                     hit_ids + g->n_layers * i, last, first, par_out + 6 * i, cov_out + 36 * i,
                                     chi2 + i, nhits + i);
    return ORC_OK;
}

/* ------------------------------------------------------------------ hit index (binning) */

int orc_eta_bin(const orc_geom *g, int layer, double z)
{
    const double eta = asinh(z / g->radius[layer]);
    int b = (int)floor((eta - g->eta_min) / g->eta_bin_w);
    if (b < 0) b = 0;
    if (b >= g->n_eta_bins) b = g->n_eta_bins - 1;
    return b;
}

int orc_hit_eta_bin(const orc_geom *g, const orc_hit *h)
{
    if (g->disk_z[h->layer] <= 0.0) return orc_eta_bin(g, h->layer, h->z);
    const double eta = asinh(h->z / sqrt(h->x * h->x + h->y * h->y));
    int b = (int)floor((eta - g->eta_min) / g->eta_bin_w);
    if (b < 0) b = 0;
    if (b >= g->n_eta_bins) b = g->n_eta_bins - 1;
    return b;
}

int orc_phi_bin(const orc_geom *g, double phi)
{
    int b = (int)floor((phi + ORC_PI) / (2.0 * ORC_PI) * g->n_phi_bins);
    if (b < 0) b = 0;
    if (b >= g->n_phi_bins) b = g->n_phi_bins - 1;
    return b;
}

static const orc_hit *g_sort_hits;
static const int *g_sort_bin;
static int cmp_hit_order(const void *a, const void *b)
{
    const int i = *(const int *)a, j = *(const int *)b;
    const int li = g_sort_hits[i].layer, lj = g_sort_hits[j].layer;
    if (li != lj) return li < lj ? -1 : 1;
    if (g_sort_bin[i] != g_sort_bin[j]) return g_sort_bin[i] < g_sort_bin[j] ? -1 : 1;
    return i < j ? -1 : (i > j);
}

/* Bins every hit of one event by (layer, eta bin, phi bin) and orders hit ids by
 * (layer, eta bin, phi bin, id); bin_off[l * (nb + 1) + b] is the CSR offset of bin b of
 * layer l into `order` (nb = n_eta_bins * n_phi_bins, bin = eta_bin * n_phi_bins + phi_bin). */
int orc_hit_index(const orc_geom *g, int n, const orc_hit *hits, int *bin_of_hit, int *order, int *bin_off)
{
    const int nb = g->n_eta_bins * g->n_phi_bins;
    for (int i = 0; i < n; ++i) {
        const orc_hit *h = &hits[i];
        if (h->layer < 0 || h->layer >= g->n_layers) return ORC_ERR_INVALID;
        bin_of_hit[i] = orc_hit_eta_bin(g, h) * g->n_phi_bins + orc_phi_bin(g, atan2(h->y, h->x));
        order[i] = i;
    }
    g_sort_hits = hits;
    g_sort_bin = bin_of_hit;
    qsort(order, (size_t)n, sizeof(int), cmp_hit_order);
    for (int k = 0; k < g->n_layers * (nb + 1); ++k) bin_off[k] = 0;
    for (int i = 0; i < n; ++i) bin_off[hits[i].layer * (nb + 1) + bin_of_hit[i] + 1] += 1;
    int base = 0; /* layers follow one another in `order` */
    for (int l = 0; l < g->n_layers; ++l) {
        int *off = bin_off + l * (nb + 1);
        off[0] = base;
        for (int b = 0; b < nb; ++b) off[b + 1] += off[b];
        base = off[nb];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ building (Sec. 2, 3.2) */

typedef struct {
    double p[6], P[36], chi2;
    int nhits, parent, hit; /* hit = event hit id added on this layer, -1 for a hole */
    int hits[ORC_MAX_LAYERS];
} orc_cand;

static int cmp_branch(const void *a, const void *b)
{
    const orc_cand *x = (const orc_cand *)a, *y = (const orc_cand *)b;
    if (x->nhits != y->nhits) return x->nhits > y->nhits ? -1 : 1;
    if (x->chi2 != y->chi2) return x->chi2 < y->chi2 ? -1 : 1;
    if (x->parent != y->parent) return x->parent < y->parent ? -1 : 1;
    const unsigned hx = (unsigned)x->hit, hy = (unsigned)y->hit; /* a hole (-1) sorts last */
    return hx < hy ? -1 : (hx > hy);
}

static int eta_to_bin(const orc_geom *g, double eta)
{
    const double f = floor((eta - g->eta_min) / g->eta_bin_w);
    if (!(f >= 0.0)) return 0; /* also -inf */
    if (f >= g->n_eta_bins - 1) return g->n_eta_bins - 1;
    return (int)f;
}

static void phi_bins(const orc_geom *g, double ph, double dphi, int *pb0, int *pb1)
{
    const double f0 = (ph - dphi + ORC_PI) / (2.0 * ORC_PI) * g->n_phi_bins;
    const double f1 = (ph + dphi + ORC_PI) / (2.0 * ORC_PI) * g->n_phi_bins;
    *pb0 = (int)floor(f0);
    *pb1 = (int)floor(f1);
    if (*pb1 - *pb0 + 1 >= g->n_phi_bins) { *pb0 = 0; *pb1 = g->n_phi_bins - 1; }
}

/* Window on an endcap disk: the chi2-cut box |u| <= U (r-phi), |v| <= W (r) of the innovation
 * covariance at phi_h = phi of the prediction.  A hit at (r_h, phi_p + d) has
 * u = r_p sin(d) and v = r_h - r_p cos(d), so the box holds |d| <= asin(U / r_p) and radii from
 * r_p cos(asin(U / r_p)) - W to r_p + W, whose eta bins (eta = asinh(z / r) on the disk at z)
 * are scanned. */
static void disk_window_bins(const orc_geom *g, int layer, const double p[6], const double P[36],
                             double var_u, double var_v, int *eb0, int *eb1, int *pb0, int *pb1,
                             double *Uo, double *Wo)
{
    const double rp = sqrt(p[0] * p[0] + p[1] * p[1]);
    const double ph = atan2(p[1], p[0]);
    orc_hit probe = {p[0], p[1], p[2], var_u, var_v, layer, 1};
    double H[12], r[2], V[4], S[4], Si[4];
    meas_model(p, &probe, H, r, V);
    innovation(P, H, V, S, Si);
    const double U = sqrt(g->chi2_cut * S[0]) * (1.0 + g->window_margin);
    const double W = sqrt(g->chi2_cut * S[3]) * (1.0 + g->window_margin);
    *Uo = U;
    *Wo = W;
    const double dphi = asin(U / rp < 1.0 ? U / rp : 1.0);
    const double r_lo = rp * cos(dphi) - W, r_hi = rp + W;
    const double zd = p[2];
    const double e_far = asinh(zd / r_hi);                                   /* the largest radius */
    const double e_near = r_lo > 0.0 ? asinh(zd / r_lo) : (zd > 0.0 ? INFINITY : -INFINITY);
    *eb0 = eta_to_bin(g, zd > 0.0 ? e_far : e_near);
    *eb1 = eta_to_bin(g, zd > 0.0 ? e_near : e_far);
    phi_bins(g, ph, dphi, pb0, pb1);
}

static void window_bins(const orc_geom *g, int layer, const double p[6], const double P[36],
                        double var_u, double var_v, int *eb0, int *eb1, int *pb0, int *pb1,
                        double *Uo, double *Wo)
{
    if (g->disk_z[layer] > 0.0) {
        disk_window_bins(g, layer, p, P, var_u, var_v, eb0, eb1, pb0, pb1, Uo, Wo);
        return;
    }
    /* chi2-cut bounding box of the innovation covariance at phi_h = phi of the prediction */
    const double R = g->radius[layer];
    const double ph = atan2(p[1], p[0]);
    orc_hit probe = {R * cos(ph), R * sin(ph), p[2], var_u, var_v, layer, 0};
    double H[12], r[2], V[4], S[4], Si[4];
    meas_model(p, &probe, H, r, V);
    innovation(P, H, V, S, Si);
    double U = sqrt(g->chi2_cut * S[0]) * (1.0 + g->window_margin);
    double W = sqrt(g->chi2_cut * S[3]) * (1.0 + g->window_margin);
    if (g->hit_dr > 0.0) {
        /* hits up to hit_dr off the cylinder: while the radius changes by hit_dr the track
         * covers t = hit_dr / cos(alpha) of transverse path (alpha between its direction and
         * the radial direction, cos(alpha) floored at 0.01), moving t sin(alpha) along the
         * cylinder plus at most t^2 |kappa| of bending, and t |cot(theta)| in z */
        const double r0 = sqrt(p[0] * p[0] + p[1] * p[1]);
        const double ca = fabs(p[0] * cos(p[4]) + p[1] * sin(p[4])) / r0;
        const double sa = fabs(p[0] * sin(p[4]) - p[1] * cos(p[4])) / r0;
        const double t = g->hit_dr / (ca > 0.01 ? ca : 0.01);
        const double kappa = fabs(ORC_KB * g->bz * p[3]);
        U += (1.0 + g->window_margin) * t * (sa + t * kappa);
        W += (1.0 + g->window_margin) * t * fabs(cos(p[5]) / sin(p[5]));
        /* that travel is uncertain too: to first order the crossing moves along the cylinder by
         * hit_dr tan(alpha) and in z by t cot(theta), so the state's spread in
         * alpha = phi - phi_pos (phi_pos = u / R) and in theta spreads the prediction at the
         * hit's radius by (t / cos alpha) sigma_alpha along the cylinder and by
         * t (sigma_theta / sin^2 theta + tan(alpha) |cot theta| sigma_alpha) in z.  The standard
         * deviation of a sum is at most the sum of the standard deviations, so adding
         * sqrt(cut) times these to U and W makes the window contain the chi2 < cut ellipse at the
         * hit's own radius as well. */
        const double cfl = ca > 0.01 ? ca : 0.01;
        const double sig_alpha = sqrt(P[4 * 6 + 4]) + sqrt(S[0]) / R;
        const double sig_theta = sqrt(P[5 * 6 + 5]);
        const double st = sin(p[5]);
        U += (1.0 + g->window_margin) * sqrt(g->chi2_cut) * t / cfl * sig_alpha;
        W += (1.0 + g->window_margin) * sqrt(g->chi2_cut) * t *
             (sig_theta / (st * st) + sa / cfl * fabs(cos(p[5]) / st) * sig_alpha);
    }
    *Uo = U;
    *Wo = W;
    const double dphi = asin(U / R < 1.0 ? U / R : 1.0);
    *eb0 = orc_eta_bin(g, layer, p[2] - W);
    *eb1 = orc_eta_bin(g, layer, p[2] + W);
    const double f0 = (ph - dphi + ORC_PI) / (2.0 * ORC_PI) * g->n_phi_bins;
    const double f1 = (ph + dphi + ORC_PI) / (2.0 * ORC_PI) * g->n_phi_bins;
    *pb0 = (int)floor(f0);
    *pb1 = (int)floor(f1);
    if (*pb1 - *pb0 + 1 >= g->n_phi_bins) { *pb0 = 0; *pb1 = g->n_phi_bins - 1; }
}

static int near(double a, double b, double tol)
{
    const double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    return fabs(a - b) <= tol * (m > 1.0 ? m : 1.0);
}

/*
 * Combinatorial building of one seed through layers first..n_layers-1.
 * For each layer and each candidate in rank order: propagate; collect every compatible hit
 * of the window (or of the whole layer when brute_force; brute_force = 2 also drops the
 * residual window of hits off the cylinder) as a branch; a candidate with no
 * compatible hit yields one hole branch.  All branches of the seed are ranked and the best
 * n_cand kept (n_cand <= 0: keep all); hit branches get the Kalman update, then every kept
 * branch gets the scattering noise of the layer (except on the outermost layer).
 */
static int build_seed(const orc_geom *g, const orc_event *ev, const double sp[6], const double sP[36],
                      double schi2, int snhits, const int *shits, orc_seed_result *res, orc_stats *stats)
{
    int cap = 16, n = 1;
    orc_cand *C = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)cap);
    memcpy(C[0].p, sp, sizeof C[0].p);
    memcpy(C[0].P, sP, sizeof C[0].P);
    C[0].chi2 = schi2;
    C[0].nhits = snhits;
    C[0].parent = 0;
    C[0].hit = -1;
    for (int l = 0; l < ORC_MAX_LAYERS; ++l) C[0].hits[l] = l < g->n_layers ? shits[l] : -1;
    res->fragile_layer = g->n_layers;
    const double tol = g->tie_tol;

    for (int l = g->first_build_layer; l < g->n_layers; ++l) {
        int nb = 0, bcap = 16;
        orc_cand *B = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)bcap);
        for (int c = 0; c < n; ++c) {
            double q[6], J[36], Q[36];
            if (stats) stats->n_prop += 1;
            if (propagate_layer(g, l, C[c].p, 0, q, J) != ORC_OK) continue; /* dropped */
            sandwich6(J, C[c].P, Q);
            int found = 0;
            int eb0, eb1, pb0, pb1;
            double U, W;
            window_bins(g, l, q, Q, ev->var_u_max[l], ev->var_v_max[l], &eb0, &eb1, &pb0, &pb1, &U, &W);
            const int nbin = g->n_eta_bins * g->n_phi_bins;
            const int *off = ev->bin_off + l * (nbin + 1);
            int k_lo, k_hi, e_lo, e_hi;
            if (g->brute_force) { e_lo = 0; e_hi = 0; k_lo = 0; k_hi = 0; }
            else { e_lo = eb0; e_hi = eb1; k_lo = pb0; k_hi = pb1; }
            for (int e = e_lo; e <= e_hi; ++e)
                for (int k = k_lo; k <= k_hi; ++k) {
                    int i0, i1;
                    if (g->brute_force) { i0 = off[0]; i1 = off[nbin]; }
                    else {
                        const int pb = ((k % g->n_phi_bins) + g->n_phi_bins) % g->n_phi_bins;
                        i0 = off[e * g->n_phi_bins + pb];
                        i1 = off[e * g->n_phi_bins + pb + 1];
                    }
                    for (int t = i0; t < i1; ++t) {
                        const int hid = ev->order[t];
                        const orc_hit *h = &ev->hits[hid];
                        if (stats) stats->n_hits_examined += 1;
                        if (q[0] * h->x + q[1] * h->y <= 0.0) continue; /* far half of the cylinder */
                        if (h->disk && h->z * q[2] <= 0.0) continue;    /* the other endcap's disk */
                        const double *qh = q, *Qh = Q;
                        double q2[6], J2[36], Q2[36];
                        if (g->hit_dr > 0.0 && g->disk_z[l] <= 0.0) {
                            /* the window around the prediction on the average radius, then the
                             * state at the hit's own radius */
                            double H[12], r[2], V[4];
                            meas_model(q, h, H, r, V);
                            /* brute_force 2: no window at all, every hit of the layer is
                             * scored at its own radius (the check that the window loses none) */
                            const int inside = g->brute_force == 2 || (fabs(r[0]) <= U && fabs(r[1]) <= W);
                            /* within tol of an edge: the window decision is fragile if the hit
                             * would pass the chi2 cut */
                            const int edge = g->brute_force != 2 &&
                                             (fabs(fabs(r[0]) - U) <= tol * U || fabs(fabs(r[1]) - W) <= tol * W);
                            if (!inside && !edge) continue;
                            if (stats) stats->n_steps += 1;
                            if (orc_propagate(g, C[c].p, target_radius(g, l, h), q2, J2) != ORC_OK) continue;
                            sandwich6(J2, C[c].P, Q2);
                            qh = q2;
                            Qh = Q2;
                            if (edge && orc_chi2(qh, Qh, h) < g->chi2_cut * (1.0 + tol) && res->fragile_layer > l)
                                res->fragile_layer = l;
                            if (!inside) continue;
                        }
                        const double c2 = orc_chi2(qh, Qh, h);
                        if (near(c2, g->chi2_cut, tol) && res->fragile_layer > l) res->fragile_layer = l;
                        if (!(c2 < g->chi2_cut)) continue;
                        if (nb == bcap) { bcap *= 2; B = (orc_cand *)realloc(B, sizeof(orc_cand) * (size_t)bcap); }
                        orc_cand *b = &B[nb++];
                        memcpy(b->p, qh, sizeof b->p);
                        memcpy(b->P, Qh, sizeof b->P);
                        b->chi2 = C[c].chi2 + c2;
                        b->nhits = C[c].nhits + 1;
                        b->parent = c;
                        b->hit = hid;
                        memcpy(b->hits, C[c].hits, sizeof b->hits);
                        b->hits[l] = hid;
                        found = 1;
                    }
                }
            if (!found) {
                if (nb == bcap) { bcap *= 2; B = (orc_cand *)realloc(B, sizeof(orc_cand) * (size_t)bcap); }
                orc_cand *b = &B[nb++];
                memcpy(b->p, q, sizeof q);
                memcpy(b->P, Q, sizeof Q);
                b->chi2 = C[c].chi2;
                b->nhits = C[c].nhits;
                b->parent = c;
                b->hit = -1;
                memcpy(b->hits, C[c].hits, sizeof b->hits);
                b->hits[l] = -1;
            }
        }
        qsort(B, (size_t)nb, sizeof(orc_cand), cmp_branch);
        const int keep = (g->n_cand > 0 && nb > g->n_cand) ? g->n_cand : nb;
        const int look = keep < nb ? keep + 1 : keep;
        for (int i = 0; i + 1 < look; ++i)
            if (B[i].nhits == B[i + 1].nhits && near(B[i].chi2, B[i + 1].chi2, tol) && res->fragile_layer > l)
                res->fragile_layer = l;
        for (int i = 0; i < keep; ++i) {
            if (B[i].hit >= 0) {
                double dc2;
                if (stats) stats->n_updates += 1;
                orc_update(B[i].p, B[i].P, &ev->hits[B[i].hit], &dc2);
            }
            if (l < g->n_layers - 1) orc_scatter(g, l, B[i].p, B[i].P);
        }
        if (stats) stats->n_kept += keep;
        free(C);
        C = B;
        n = keep;
        cap = bcap;
        if (n == 0) break;
    }
    (void)cap;
    res->n_cand = n;
    const int nout = n < res->cap ? n : res->cap;
    for (int i = 0; i < nout; ++i) {
        memcpy(res->par + 6 * i, C[i].p, 6 * sizeof(double));
        memcpy(res->cov + 36 * i, C[i].P, 36 * sizeof(double));
        res->chi2[i] = C[i].chi2;
        res->nhits[i] = C[i].nhits;
        for (int l = 0; l < g->n_layers; ++l) res->hits[i * g->n_layers + l] = C[i].hits[l];
    }
    free(C);
    return ORC_OK;
}

int orc_build_seed(const orc_geom *g, const orc_event *ev, const double sp[6], const double sP[36],
                   double schi2, int snhits, const int *shits, orc_seed_result *res, orc_stats *stats)
{
    if (g->n_layers > ORC_MAX_LAYERS || g->first_build_layer < 1) return ORC_ERR_INVALID;
    return build_seed(g, ev, sp, sP, schi2, snhits, shits, res, stats);
}

/* ------------------------------------------------------------------ batch helpers */

int orc_seed_batch(const orc_geom *g, const orc_hit *hits, int n, const int *seed_hits, double *par, double *cov)
{
    for (int i = 0; i < n; ++i) {
        const int *s = seed_hits + 3 * i;
        int st = orc_seed_estimate(g, &hits[s[0]], &hits[s[1]], &hits[s[2]], par + 6 * i, cov + 36 * i);
        if (st != ORC_OK) return st;
    }
    return ORC_OK;
}

int orc_fit_batch(const orc_geom *g, const orc_hit *hits, int n, const double *par_in, const double *cov_in,
                  const int *hit_ids, int first, int last, double *par_out, double *cov_out, double *chi2,
                  int *nhits, int *status)
{
    for (int i = 0; i < n; ++i)
        status[i] = orc_fit_track(g, par_in + 6 * i, cov_in + 36 * i, hits, hit_ids + g->n_layers * i, first,
                                  last, par_out + 6 * i, cov_out + 36 * i, chi2 + i, nhits + i);
    return ORC_OK;
}

int orc_build_batch(const orc_geom *g, const orc_event *ev, int n, const double *sp, const double *sP,
                    const double *schi2, const int *snhits, const int *shits, int cap, int *n_cand,
                    double *par, double *cov, double *chi2, int *nhits, int *hits, int *fragile,
                    orc_stats *stats)
{
    for (int i = 0; i < n; ++i) {
        orc_seed_result r;
        r.cap = cap;
        r.par = par + (size_t)i * cap * 6;
        r.cov = cov + (size_t)i * cap * 36;
        r.chi2 = chi2 + (size_t)i * cap;
        r.nhits = nhits + (size_t)i * cap;
        r.hits = hits + (size_t)i * cap * g->n_layers;
        int st = orc_build_seed(g, ev, sp + 6 * i, sP + 36 * i, schi2[i], snhits[i], shits + g->n_layers * i, &r, stats);
        if (st != ORC_OK) return st;
        n_cand[i] = r.n_cand;
        fragile[i] = r.fragile_layer;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ seeding from hit triplets */
/*
 * Sec. 2 names seeding as the first stage (the initial estimate from a few hits of the innermost
 * layers) and leaves it unspecified.  Reading used here, written out as a definition and
 * evaluated by brute force over every hit of layers 1, 2 and 3 of the event:
 *   - a seed is a triplet (a, b, c) of hits on layers 0, 1, 2, compatible with a helix that
 *     leaves the beam line (x = y = 0) with transverse momentum >= pt_min, confirmed by a hit e
 *     on layer 3; r below is a hit's transverse radius, R_l the layer radius;
 *   - pair (a, b): transverse chord |b - a| <= 2 (R_1 - R_0) (a track moving outwards, not the
 *     far crossing of a looping circle); the circle through the beam line point, a and b has
 *     |curvature| <= kappa_max; the r-z line through a and b meets r = 0 within |z| <= z_vertex;
 *   - triplet: chord |c - b| <= 2 (R_2 - R_1); the circle through a, b, c (not collinear) has
 *     curvature <= kappa_max and passes the beam line point at d0 = (|U|^2 - rho^2) / (2 rho)
 *     (U its centre, rho its radius: the point's power divided by the diameter, its signed
 *     distance from the circle to first order), |d0| <= d0_max; the third hit's z lies within
 *     dz_max of the r-z line through a and b, taken at r_c;
 *   - confirmation: a hit e on layer 3 with chord |e - c| <= 2 (R_3 - R_2), signed distance
 *     f = (|e - U|^2 - rho^2) / (2 rho) from the triplet circle with |f| <= conf_rphi, and z
 *     within conf_z of the r-z line through b and c, taken at r_e;
 *   - score s = (d0 / d0_max)^2 + (dz / dz_max)^2 + min over confirming e of
 *     (f / conf_rphi)^2 + (dz3 / conf_z)^2; each first-layer hit keeps its passing triplet of
 *     smallest score (equal scores: smallest layer-1 id, then layer-2 id), so a hit starts at
 *     most one seed.
 */
double orc_seed_kappa_max(const orc_geom *g, const orc_seed_cuts *c)
{
    return ORC_KB * g->bz / c->pt_min * (1.0 + c->kappa_slack);
}

static double seed_rt(const orc_hit *h) { return sqrt(h->x * h->x + h->y * h->y); }

static double seed_chord(const orc_hit *a, const orc_hit *b)
{
    return sqrt((b->x - a->x) * (b->x - a->x) + (b->y - a->y) * (b->y - a->y));
}

/* circumscribed circle of three points (centre where the perpendicular bisectors meet); 0 when
 * the points are collinear */
static int circumcircle(double ax, double ay, double bx, double by, double cx, double cy, double *ux, double *uy,
                        double *rho)
{
    const double d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by));
    if (d == 0.0) return 0;
    const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    *ux = (a2 * (by - cy) + b2 * (cy - ay) + c2 * (ay - by)) / d;
    *uy = (a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax)) / d;
    *rho = sqrt((ax - *ux) * (ax - *ux) + (ay - *uy) * (ay - *uy));
    return 1;
}

/* pair stage; returns 1 if it passes */
static int seed_pair(const orc_geom *g, const orc_seed_cuts *c, const orc_hit *a, const orc_hit *b, orc_seed_quant *q)
{
    const double ra = seed_rt(a), rb = seed_rt(b);
    double ux, uy, rho;
    q->chord01 = seed_chord(a, b);
    q->kappa01 = 0.0;  /* a, b and the beam line point on one straight line */
    if (circumcircle(0.0, 0.0, a->x, a->y, b->x, b->y, &ux, &uy, &rho))
        q->kappa01 = (a->x * b->y - a->y * b->x > 0.0 ? 1.0 : -1.0) / rho;
    if (rb == ra) return 0;
    q->zv = a->z - ra * (b->z - a->z) / (rb - ra);
    return q->chord01 <= 2.0 * (g->radius[1] - g->radius[0]) && fabs(q->kappa01) <= orc_seed_kappa_max(g, c) &&
           fabs(q->zv) <= c->z_vertex;
}

/* triplet stage (the pair passed); circle centre and radius returned for the confirmation */
static int seed_triplet(const orc_geom *g, const orc_seed_cuts *c, const orc_hit *a, const orc_hit *b,
                        const orc_hit *cc, orc_seed_quant *q, double *ux, double *uy, double *rho)
{
    const double ra = seed_rt(a), rb = seed_rt(b), rc = seed_rt(cc);
    q->chord12 = seed_chord(b, cc);
    if (!circumcircle(a->x, a->y, b->x, b->y, cc->x, cc->y, ux, uy, rho)) {
        q->collinear = 1;
        return 0;
    }
    q->kappa = 1.0 / *rho;
    q->d0 = (*ux * *ux + *uy * *uy - *rho * *rho) / (2.0 * *rho);
    q->dz = cc->z - (a->z + (b->z - a->z) * (rc - ra) / (rb - ra));
    return q->chord12 <= 2.0 * (g->radius[2] - g->radius[1]) && q->kappa <= orc_seed_kappa_max(g, c) &&
           fabs(q->d0) <= c->d0_max && fabs(q->dz) <= c->dz_max;
}

/* confirmation stage */
static int seed_confirm(const orc_geom *g, const orc_seed_cuts *c, const orc_hit *b, const orc_hit *cc,
                        const orc_hit *e, double ux, double uy, double rho, orc_seed_quant *q)
{
    const double rb = seed_rt(b), rc = seed_rt(cc), re = seed_rt(e);
    q->chord23 = seed_chord(cc, e);
    q->f3 = ((e->x - ux) * (e->x - ux) + (e->y - uy) * (e->y - uy) - rho * rho) / (2.0 * rho);
    if (rc == rb) {
        q->dz3 = 1e30;
        return 0;
    }
    q->dz3 = e->z - (b->z + (cc->z - b->z) * (re - rb) / (rc - rb));
    return q->chord23 <= 2.0 * (g->radius[3] - g->radius[2]) && fabs(q->f3) <= c->conf_rphi &&
           fabs(q->dz3) <= c->conf_z;
}

int orc_seed_eval(const orc_geom *g, const orc_seed_cuts *c, const orc_hit *a, const orc_hit *b, const orc_hit *cc,
                  const orc_hit *e, orc_seed_quant *q)
{
    memset(q, 0, sizeof *q);
    int ok = seed_pair(g, c, a, b, q);
    if (!cc) return ok;
    double ux = 0.0, uy = 0.0, rho = 0.0;
    ok = seed_triplet(g, c, a, b, cc, q, &ux, &uy, &rho) && ok;
    if (!e || q->collinear) return ok;
    return seed_confirm(g, c, b, cc, e, ux, uy, rho, q) && ok;
}

/* |x| / cut for each quantity of one stage; folds the stage's decision into *margin: every
 * quantity of a passing stage, the single failing quantity of a stage that fails on one */
static void fold_margin(const double *ratio, int n, double *margin)
{
    int fails = 0, k_fail = -1;
    double m = 1e30;
    for (int k = 0; k < n; ++k) {
        if (ratio[k] > 1.0) {
            ++fails;
            k_fail = k;
        }
        const double d = fabs(ratio[k] - 1.0);
        if (d < m) m = d;
    }
    if (fails == 0 && m < *margin) *margin = m;
    if (fails == 1 && fabs(ratio[k_fail] - 1.0) < *margin) *margin = fabs(ratio[k_fail] - 1.0);
}

static void seed_of(const orc_geom *g, const orc_seed_cuts *c, int n, const orc_hit *hits, int ia, orc_seed_pick *p)
{
    const double kmax = orc_seed_kappa_max(g, c);
    const double lim01 = 2.0 * (g->radius[1] - g->radius[0]), lim12 = 2.0 * (g->radius[2] - g->radius[1]);
    const double lim23 = 2.0 * (g->radius[3] - g->radius[2]);
    double best = 1e300, second = 1e300;
    p->h1 = p->h2 = p->h3 = -1;
    p->n_pass = 0;
    p->score = 0.0;
    p->margin = 1e30;
    const orc_hit *a = &hits[ia];
    for (int ib = 0; ib < n; ++ib) {
        if (hits[ib].layer != 1) continue;
        orc_seed_quant q;
        memset(&q, 0, sizeof q);
        const int pair_ok = seed_pair(g, c, a, &hits[ib], &q);
        if (seed_rt(&hits[ib]) == seed_rt(a)) continue;
        const double r01[3] = {q.chord01 / lim01, fabs(q.kappa01) / kmax, fabs(q.zv) / c->z_vertex};
        fold_margin(r01, 3, &p->margin);
        if (!pair_ok) continue;
        for (int ic = 0; ic < n; ++ic) {
            if (hits[ic].layer != 2) continue;
            double ux, uy, rho;
            const int trip_ok = seed_triplet(g, c, a, &hits[ib], &hits[ic], &q, &ux, &uy, &rho);
            if (q.collinear) {
                q.collinear = 0;
                continue;
            }
            const double r12[4] = {q.chord12 / lim12, q.kappa / kmax, fabs(q.d0) / c->d0_max, fabs(q.dz) / c->dz_max};
            fold_margin(r12, 4, &p->margin);
            if (!trip_ok) continue;
            double c3 = 0.0;
            int h3 = -1;
            if (c->confirm) {
                c3 = 1e300;
                for (int ie = 0; ie < n; ++ie) {
                    if (hits[ie].layer != 3) continue;
                    const int conf_ok = seed_confirm(g, c, &hits[ib], &hits[ic], &hits[ie], ux, uy, rho, &q);
                    const double r23[3] = {q.chord23 / lim23, fabs(q.f3) / c->conf_rphi, fabs(q.dz3) / c->conf_z};
                    fold_margin(r23, 3, &p->margin);
                    if (!conf_ok) continue;
                    const double v = (q.f3 / c->conf_rphi) * (q.f3 / c->conf_rphi) + (q.dz3 / c->conf_z) * (q.dz3 / c->conf_z);
                    if (v < c3) {
                        c3 = v;
                        h3 = ie;
                    }
                }
                if (h3 < 0) continue;
            }
            const double s = (q.d0 / c->d0_max) * (q.d0 / c->d0_max) + (q.dz / c->dz_max) * (q.dz / c->dz_max) + c3;
            ++p->n_pass;
            /* hits are visited in increasing id order, so a strict comparison keeps the smallest
               ids among equal scores */
            if (s < best) {
                second = best;
                best = s;
                p->h1 = ib;
                p->h2 = ic;
                p->h3 = h3;
            } else if (s < second) {
                second = s;
            }
        }
    }
    if (p->h1 >= 0) p->score = best;
    p->gap = second < 1e299 ? second - best : 1e30;
}

int orc_find_seeds_of(const orc_geom *g, const orc_seed_cuts *c, int n, const orc_hit *hits, int n_first,
                      const int *first, orc_seed_pick *pick)
{
    if (g->n_layers < 4 || c->pt_min <= 0.0 || c->z_vertex <= 0.0 || c->d0_max <= 0.0 || c->dz_max <= 0.0 ||
        c->conf_rphi <= 0.0 || c->conf_z <= 0.0)
        return ORC_ERR_INVALID;
    for (int k = 0; k < n_first; ++k) {
        if (first[k] < 0 || first[k] >= n || hits[first[k]].layer != 0) return ORC_ERR_INVALID;
        seed_of(g, c, n, hits, first[k], &pick[k]);
    }
    return ORC_OK;
}

int orc_find_seeds(const orc_geom *g, const orc_seed_cuts *c, int n, const orc_hit *hits, orc_seed_pick *pick)
{
    for (int i = 0; i < n; ++i) {
        memset(&pick[i], 0, sizeof pick[i]);
        pick[i].h1 = pick[i].h2 = pick[i].h3 = -1;
        pick[i].margin = pick[i].gap = 1e30;
        if (hits[i].layer != 0) continue;
        const int st = orc_find_seeds_of(g, c, n, hits, 1, &i, &pick[i]);
        if (st != ORC_OK) return st;
    }
    return ORC_OK;
}
