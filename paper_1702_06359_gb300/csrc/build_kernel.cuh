// Combinatorial track building kernel (Sec. 2 and Sec. 3.2 of arXiv:1702.06359).
//
// Mapping: a seed owns a segment of N consecutive lanes of a warp (N = candidates kept per
// seed); lane r of the segment holds the candidate of rank r, its state (6 parameters, 21
// covariance elements, chi2, nHits) in registers for the whole trajectory.  Per layer:
//   1. every live candidate is propagated to the cylinder (helix + Jacobian, kf_math.cuh);
//   2. it scans the hits of its eta-phi window (CSR bins of the hit index), scores each by
//      chi2 and keeps its own best-N branch keys in a register list; a candidate with no
//      compatible hit contributes one hole key;
//   3. the segment merges its lanes' lists: N rounds of a segmented warp-shuffle minimum give
//      the seed's N best branches in rank order (the paper's "branching to explore multiple
//      candidate tracks per seed" and the per-seed repacking of Sec. 3.2.1);
//   4. the lane of rank r fetches its parent's predicted state with shuffles, applies the
//      Kalman update (U = float or double) for a hit branch and the layer's scattering noise.
// With hits off the layers' cylinders (kTwo) step 1 reaches the layer's average radius, step 2
// scores each hit after a second, short propagation to its own radius, and the survivor of a
// hit branch takes that step before its update (the two-step propagation of Sec. 2.2).  With
// endcap disks (kDisk) a disk layer is reached by the helix/plane crossing, its window is taken
// in r-phi and r, and its hits are measured on the disk's plane (the "endcap z" of Sec. 2.2).
// Hit history is kept per warp in shared memory (parent rank, hit id per layer and lane) and
// the best candidate is backtracked at the end.  Work balance follows the paper's dynamic
// work stealing (Sec. 2.3): warps pull tiles of seeds_per_block seeds from an atomic counter
// until the seeds of every event are done (one persistent launch over many events, Sec. 4).
//
// Branch key (32 bits, smaller = better): [31:27] 31 - nHits, [26:4] float bits 30..8 of the
// total chi2 rounded (non-negative, so integer order = value order, to 2^-16 relative), [3:0] parent
// rank; the event-local hit id (0x7FFFFF for a hole) travels beside it.  This is the order
// (nHits desc, chi2 asc, parent rank asc); totals within 2^-15 may rank by parent, and within
// one parent by the order the hits were scanned -- near-ties far inside the 1e-3 relative band
// within which the parity definition calls a ranking fragile.  Keys of one seed's lanes differ
// in the parent field.
#pragma once

#include "internal.h"
#include "kf_math.cuh"

namespace tkf {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned kEmpty32 = 0xFFFFFFFFu;

template <class R> __device__ __forceinline__ R pick(float f, double d);
template <> __device__ __forceinline__ float pick<float>(float f, double) { return f; }
template <> __device__ __forceinline__ double pick<double>(float, double d) { return d; }

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return __double2float_rn(v); }

// The branch key of a candidate's branch (layout at the top of this file); the chi2 bits are
// rounded to nearest, so key_chi2 returns the total within 2^-16 relative.
__device__ __forceinline__ unsigned make_key32(int nhits, float chi2, int parent)
{
    const unsigned c = ((__float_as_uint(chi2) & 0x7FFFFFFFu) + 0x80u) >> 8;
    return ((unsigned)(31 - nhits) << 27) | (c << 4) | (unsigned)parent;
}

__device__ __forceinline__ float key_chi2(unsigned key) { return __uint_as_float(((key >> 4) & 0x7FFFFFu) << 8); }

// A lane's branch list: its NMAX smallest keys in ascending order (lk), with their hit ids (lh);
// a key equal to one already listed goes after it.
template <int NMAX>
__device__ __forceinline__ void list_insert32(unsigned (&lk)[NMAX], int (&lh)[NMAX], unsigned k, int h)
{
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        const bool lt = k < lk[i];
        const unsigned k2 = lt ? lk[i] : k;
        const int h2 = lt ? lh[i] : h;
        lk[i] = lt ? k : lk[i];
        lh[i] = lt ? h : lh[i];
        k = k2;
        h = h2;
    }
}

template <int NMAX> __device__ __forceinline__ void list_pop32(unsigned (&lk)[NMAX], int (&lh)[NMAX])
{
#pragma unroll
    for (int i = 0; i + 1 < NMAX; ++i) {
        lk[i] = lk[i + 1];
        lh[i] = lh[i + 1];
    }
    lk[NMAX - 1] = kEmpty32;
}

// Hit ranges of phi sub-bins inside a bin, from the packed bytes of bin_sub (byte t - 1 holds
// the start of sub-bin t relative to the bin's first hit; the top byte is unused, so a top
// word of 0xFFFFFFFF only occurs for a bin of more than 255 hits, whose sub-bins are unknown).
__device__ __forceinline__ int sub_byte(const uint4 w, int t)  // start of sub-bin t, 1 <= t < kSubBins
{
    const unsigned word = t <= 4 ? w.x : (t <= 8 ? w.y : (t <= 12 ? w.z : w.w));
    return (int)((word >> (8 * ((t - 1) & 3))) & 0xFFu);
}
// first hit of sub-bin s (s = 0: the bin's first hit)
__device__ __forceinline__ int sub_first(const uint4 w, int s)
{
    return (s <= 0 || w.w == 0xFFFFFFFFu) ? 0 : sub_byte(w, s);
}
// one past the last hit of sub-bin s (s = kSubBins - 1: the bin's hit count)
__device__ __forceinline__ int sub_end(const uint4 w, int s, int count)
{
    return (s >= kSubBins - 1 || w.w == 0xFFFFFFFFu) ? count : sub_byte(w, s + 1);
}

template <class R>
__device__ __forceinline__ int eta_bin_window(R z, R inv_r, R eta_min, R inv_w, int n_eta, R slack)
{
    const R x = z * inv_r;
    const R ax = ab(x);
    const R e = copysign(fast_log(ax + sq(ax * ax + R(1))), x);
    const int b = (int)flr((e - eta_min) * inv_w + slack);
    return b < 0 ? 0 : (b >= n_eta ? n_eta - 1 : b);
}

// asin(x) for 0 <= x <= 1; below 0.5 the series x (1 + x^2/6 + 3x^4/40 + 5x^6/112) (relative
// error < 1.3e-4, an underestimate covered by the window's relative margin on U)
template <class R> __device__ __forceinline__ R asin_window(R x)
{
    if (x < R(0.5)) {
        const R x2 = x * x;
        return x * (R(1) + x2 * (R(1.0 / 6) + x2 * (R(3.0 / 40) + x2 * R(5.0 / 112))));
    }
    return asn(x < R(1) ? x : R(1));
}

// Scores every hit of the candidate's window and fills its branch list.  kTwo: hits lie up to
// a.hit_dr off the cylinder (the two-step geometry of Sec. 2.2): the window around the
// prediction on the average radius is widened by the track's travel over hit_dr, and each hit
// inside it is scored after the second step to its own radius (step_chi2).
template <int NMAX, class R, bool kTwo>
__device__ __forceinline__ void scan_window(const BuildArgs &a, int ev, int l, R Rl, const R p[6], const R P[21],
                                            R chi2, int nh, int rank, unsigned (&lk)[NMAX], int (&lh)[NMAX])
{
    const int seg = ev * a.L + l;
    const float2 vmax = a.var_max[seg];
    const R xp = p[0], yp = p[1], zp = p[2];
    const R rp = sq(xp * xp + yp * yp);
    const R sf = yp / rp, cf = xp / rp;
    // innovation covariance at phi_h = phi of the prediction, with the layer's largest V
    const R Suu = sf * (sf * P[sym(0, 0)] - cf * P[sym(1, 0)]) + cf * (cf * P[sym(1, 1)] - sf * P[sym(1, 0)]) + R(vmax.x);
    const R Svv = P[sym(2, 2)] + R(vmax.y);
    const R cut = pick<R>(a.cut_f, a.cut);
    const R mg = R(1) + pick<R>(a.margin_f, a.margin);
    R U = sq(cut * Suu) * mg, W = sq(cut * Svv) * mg;
    R sphi = R(0), cphi = R(1), sth = R(1), cot = R(0);
    const R kb = pick<R>(a.kb_f, a.kb);
    if (kTwo) {
        // while the radius changes by hit_dr the track covers t = hit_dr / cos(alpha) of
        // transverse path (alpha between its direction and the radial direction, cos(alpha)
        // floored at 0.01), moving t sin(alpha) along the cylinder plus at most t^2 |kappa| of
        // bending, and t |cot(theta)| in z
        R cth;
        sc(p[4], &sphi, &cphi);
        fast_sc(p[5], &sth, &cth);
        cot = cth / sth;
        const R ca = ab(xp * cphi + yp * sphi) / rp, sa = ab(xp * sphi - yp * cphi) / rp;
        const R cfl = ca > R(0.01) ? ca : R(0.01);
        const R t = pick<R>(a.hit_dr_f, a.hit_dr) / cfl;
        U += mg * t * (sa + t * ab(kb * p[3]));
        W += mg * t * ab(cot);
        // the spread of that travel over the state's covariance: sigma of alpha = phi - phi_pos
        // (phi_pos = u / R) and of theta move the crossing at the hit's radius by
        // (t / cos alpha) sigma_alpha along the cylinder and t (sigma_theta / sin^2 theta +
        // tan(alpha) |cot theta| sigma_alpha) in z; sqrt(cut) times these keeps the chi2 < cut
        // ellipse at the hit's own radius inside the window
        const R sig_a = sq(P[sym(4, 4)]) + sq(Suu) / Rl;
        const R rc = sq(cut) * mg * t;
        U += rc / cfl * sig_a;
        W += rc * (sq(P[sym(5, 5)]) / (sth * sth) + sa / cfl * ab(cot) * sig_a);
    }
    const R phip = at2(yp, xp);
    // compatible hits satisfy |u| = r_p |sin(phi_h - phi_p)| <= U on the near half-cylinder,
    // so |phi_h - phi_p| <= asin(U / R); a 2e-5 rad slack covers float rounding of both angles
    const R dphi = asin_window(U / Rl) + R(2e-5);
    const R bscale = R(a.n_phi) / R(2.0 * kPi);
    const R xlo = (phip - dphi + R(kPi)) * bscale, xhi = (phip + dphi + R(kPi)) * bscale;  // phi-bin units
    const int k0 = (int)flr(xlo), k1 = (int)flr(xhi);
    int s0 = (int)flr((xlo - R(k0)) * R(kSubBins)), s1 = (int)flr((xhi - R(k1)) * R(kSubBins));
    s0 = s0 < 0 ? 0 : (s0 >= kSubBins ? kSubBins - 1 : s0);
    s1 = s1 < 0 ? 0 : (s1 >= kSubBins ? kSubBins - 1 : s1);
    const int nphi = a.n_phi;
    const R inv_r = R(1) / Rl;
    const R emin = pick<R>(a.eta_min_f, a.eta_min), iw = pick<R>(a.inv_eta_w_f, a.inv_eta_w);
    const int e0 = eta_bin_window(zp - W, inv_r, emin, iw, a.n_eta, R(-1e-4));
    const int e1 = eta_bin_window(zp + W, inv_r, emin, iw, a.n_eta, R(1e-4));
    // up to two parts (first bin, first sub-bin) .. (last bin, last sub-bin): the window may
    // wrap around phi = +-pi
    int pb0[2], ps0[2], pb1[2], ps1[2];
    if (k1 - k0 + 1 >= nphi) {
        pb0[0] = 0; ps0[0] = 0; pb1[0] = nphi - 1; ps1[0] = kSubBins - 1;
        pb0[1] = 0; ps0[1] = 0; pb1[1] = -1; ps1[1] = 0;
    } else if (k0 < 0) {
        pb0[0] = k0 + nphi; ps0[0] = s0; pb1[0] = nphi - 1; ps1[0] = kSubBins - 1;
        pb0[1] = 0; ps0[1] = 0; pb1[1] = k1; ps1[1] = s1;
    } else if (k1 >= nphi) {
        pb0[0] = k0; ps0[0] = s0; pb1[0] = nphi - 1; ps1[0] = kSubBins - 1;
        pb0[1] = 0; ps0[1] = 0; pb1[1] = k1 - nphi; ps1[1] = s1;
    } else {
        pb0[0] = k0; ps0[0] = s0; pb1[0] = k1; ps1[0] = s1;
        pb0[1] = 0; ps0[1] = 0; pb1[1] = -1; ps1[1] = 0;
    }
    bool found = false;
    const int row0 = seg * a.n_bins;
    for (int e = e0; e <= e1; ++e) {
        const int row = row0 + e * nphi;
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            if (pb1[part] < pb0[part]) continue;
            // first hit of the first sub-bin and end of the last sub-bin (independent loads)
            const int ba = row + pb0[part], bb = row + pb1[part];
            const int oa = __ldg(&a.bin_off[ba]);
            const int ob = __ldg(&a.bin_off[bb]), ob1 = __ldg(&a.bin_off[bb + 1]);
            const uint4 wa = __ldg(&a.bin_sub[ba]), wb = __ldg(&a.bin_sub[bb]);
            const int i0 = oa + sub_first(wa, ps0[part]);
            const int i1 = ob + sub_end(wb, ps1[part], ob1 - ob);
            for (int i = i0; i < i1; ++i) {
                const float4 h = __ldg(&a.hxyzi[i]);
                const float2 hv = __ldg(&a.hvar[i]);  // issued with the position: one round trip
                const R hx = R(h.x), hy = R(h.y);
                if (!(xp * hx + yp * hy > R(0))) continue;  // far half of the cylinder
                // residual on the hit's tangent plane; |u| <= U and |v| <= W bound every hit
                // with chi2 < cut (U, W are the extents of the cut ellipse of the largest S)
                const R ir = fast_rsqrt(hx * hx + hy * hy);
                const R sh = hy * ir, ch = hx * ir;
                const R u = ch * (hy - yp) - sh * (hx - xp);
                const R v = R(h.z) - zp;
                if (ab(u) > U || ab(v) > W) continue;
                R c2;
                if (kTwo)
                    c2 = step_chi2<R>(p, P, sphi, cphi, sth, cot, kb, sq(hx * hx + hy * hy), hx, hy, R(h.z), sh, ch,
                                      R(hv.x), R(hv.y));
                else
                    c2 = chi2_uv<R>(P, u, v, sh, ch, R(hv.x), R(hv.y));
                if (c2 < cut) {
                    list_insert32(lk, lh, make_key32(nh + 1, to_f32(chi2 + c2), rank), __float_as_int(h.w));
                    found = true;
                }
            }
        }
    }
    if (!found) list_insert32(lk, lh, make_key32(nh, to_f32(chi2), rank), kHoleId);
}

// The same on an endcap disk (the "endcap z" of Sec. 2.2): the chi2-cut box |u| <= U (r-phi),
// |v| <= W (r) of the innovation covariance at phi_h = phi of the prediction.  A hit at
// (r_h, phi_p + d) has u = r_p sin(d) and v = r_h - r_p cos(d): the box holds |d| <= asin(U / r_p)
// and radii from r_p cos(asin(U / r_p)) - W to r_p + W, whose eta bins (eta = asinh(z / r) on the
// disk at z) are scanned.  A compatible hit lies on the disk the state reached.
template <int NMAX, class R>
__device__ __forceinline__ void scan_window_disk(const BuildArgs &a, int ev, int l, const R p[6], const R P[21],
                                                 R chi2, int nh, int rank, unsigned (&lk)[NMAX], int (&lh)[NMAX])
{
    const int seg = ev * a.L + l;
    const float2 vmax = a.var_max[seg];
    const R xp = p[0], yp = p[1], zp = p[2];
    const R rp = sq(xp * xp + yp * yp);
    const R sf = yp / rp, cf = xp / rp;
    const R p00 = P[sym(0, 0)], p10 = P[sym(1, 0)], p11 = P[sym(1, 1)];
    const R Suu = sf * (sf * p00 - cf * p10) + cf * (cf * p11 - sf * p10) + R(vmax.x);
    const R Svv = cf * (cf * p00 + sf * p10) + sf * (sf * p11 + cf * p10) + R(vmax.y);
    const R cut = pick<R>(a.cut_f, a.cut);
    const R mg = R(1) + pick<R>(a.margin_f, a.margin);
    const R U = sq(cut * Suu) * mg, W = sq(cut * Svv) * mg;
    const R phip = at2(yp, xp);
    const R dphi = asin_window(U / rp) + R(2e-5);
    const R bscale = R(a.n_phi) / R(2.0 * kPi);
    const R xlo = (phip - dphi + R(kPi)) * bscale, xhi = (phip + dphi + R(kPi)) * bscale;
    const int k0 = (int)flr(xlo), k1 = (int)flr(xhi);
    int s0 = (int)flr((xlo - R(k0)) * R(kSubBins)), s1 = (int)flr((xhi - R(k1)) * R(kSubBins));
    s0 = s0 < 0 ? 0 : (s0 >= kSubBins ? kSubBins - 1 : s0);
    s1 = s1 < 0 ? 0 : (s1 >= kSubBins ? kSubBins - 1 : s1);
    const int nphi = a.n_phi;
    const R emin = pick<R>(a.eta_min_f, a.eta_min), iw = pick<R>(a.inv_eta_w_f, a.inv_eta_w);
    // eta bins of the radii r_p cos(dphi) - W .. r_p + W on this disk (eta falls with the radius
    // for z > 0, rises for z < 0; a range reaching r = 0 extends to the last or first row)
    R cdp, sdp;
    sc(dphi < R(1.5707963) ? dphi : R(1.5707963), &sdp, &cdp);
    const R r_lo = rp * cdp - W, r_hi = rp + W;
    const int e_far = eta_bin_window(zp, R(1) / r_hi, emin, iw, a.n_eta, zp > R(0) ? R(-1e-4) : R(1e-4));
    int e_near;
    if (r_lo > R(0))
        e_near = eta_bin_window(zp, R(1) / r_lo, emin, iw, a.n_eta, zp > R(0) ? R(1e-4) : R(-1e-4));
    else
        e_near = zp > R(0) ? a.n_eta - 1 : 0;
    const int e0 = zp > R(0) ? e_far : e_near, e1 = zp > R(0) ? e_near : e_far;
    int pb0[2], ps0[2], pb1[2], ps1[2];
    if (k1 - k0 + 1 >= nphi) {
        pb0[0] = 0; ps0[0] = 0; pb1[0] = nphi - 1; ps1[0] = kSubBins - 1;
        pb0[1] = 0; ps0[1] = 0; pb1[1] = -1; ps1[1] = 0;
    } else if (k0 < 0) {
        pb0[0] = k0 + nphi; ps0[0] = s0; pb1[0] = nphi - 1; ps1[0] = kSubBins - 1;
        pb0[1] = 0; ps0[1] = 0; pb1[1] = k1; ps1[1] = s1;
    } else if (k1 >= nphi) {
        pb0[0] = k0; ps0[0] = s0; pb1[0] = nphi - 1; ps1[0] = kSubBins - 1;
        pb0[1] = 0; ps0[1] = 0; pb1[1] = k1 - nphi; ps1[1] = s1;
    } else {
        pb0[0] = k0; ps0[0] = s0; pb1[0] = k1; ps1[0] = s1;
        pb0[1] = 0; ps0[1] = 0; pb1[1] = -1; ps1[1] = 0;
    }
    bool found = false;
    const int row0 = seg * a.n_bins;
    for (int e = e0; e <= e1; ++e) {
        const int row = row0 + e * nphi;
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            if (pb1[part] < pb0[part]) continue;
            const int ba = row + pb0[part], bb = row + pb1[part];
            const int oa = __ldg(&a.bin_off[ba]);
            const int ob = __ldg(&a.bin_off[bb]), ob1 = __ldg(&a.bin_off[bb + 1]);
            const uint4 wa = __ldg(&a.bin_sub[ba]), wb = __ldg(&a.bin_sub[bb]);
            const int i0 = oa + sub_first(wa, ps0[part]);
            const int i1 = ob + sub_end(wb, ps1[part], ob1 - ob);
            for (int i = i0; i < i1; ++i) {
                const float4 h = __ldg(&a.hxyzi[i]);
                const float2 hv = __ldg(&a.hvar[i]);
                const R hx = R(h.x), hy = R(h.y);
                if (!(xp * hx + yp * hy > R(0)) || !(R(h.z) * zp > R(0))) continue;  // far half; other endcap
                const R ir = fast_rsqrt(hx * hx + hy * hy);
                const R sh = hy * ir, ch = hx * ir;
                const R u = ch * (hy - yp) - sh * (hx - xp);
                const R v = ch * (hx - xp) + sh * (hy - yp);
                if (ab(u) > U || ab(v) > W) continue;
                const R c2 = chi2_disk<R>(p00, p10, p11, u, v, sh, ch, R(hv.x), R(hv.y));
                if (c2 < cut) {
                    list_insert32(lk, lh, make_key32(nh + 1, to_f32(chi2 + c2), rank), __float_as_int(h.w));
                    found = true;
                }
            }
        }
    }
    if (!found) list_insert32(lk, lh, make_key32(nh, to_f32(chi2), rank), kHoleId);
}

template <class R> __device__ __forceinline__ void store_track(void *par, void *cov, void *c2, int stride, int i,
                                                                  const R p[6], const R P[21], R chi2)
{
    R *pp = (R *)par, *pc = (R *)cov, *px = (R *)c2;
#pragma unroll
    for (int k = 0; k < 6; ++k) pp[(size_t)k * stride + i] = p[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) pc[(size_t)k * stride + i] = P[k];
    px[i] = chi2;
}

// Position of the k-th (0-based) set bit of m; m has more than k set bits.
__device__ __forceinline__ int nth_set_bit(unsigned m, int k)
{
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int c = __popc(m & ((1u << s) - 1u));
        if (k >= c) {
            k -= c;
            m >>= s;
            pos += s;
        }
    }
    return pos;
}

// The Kalman updates of a block's candidates, packed into as few warps as they fill (mixed
// precision).  The update is the kernel's only double-precision work, and the double-precision
// pipe spends the same time on a warp instruction whatever its active lanes; a warp's own
// candidates with a hit (about 13 of 32 lanes) would leave most of each instruction empty.
// So every thread parks its state in shared memory, the block's update jobs are numbered in
// (warp, lane) order, and job e runs on lane e % 32 of warp (e / 32 + rot) % W: 52 jobs take two
// warps instead of four.  rot turns from step to step (and between blocks) so that the warps,
// which sit on different sub-partitions of the SM, take turns.  Every job runs the same
// arithmetic on the same inputs whichever thread runs it, so results do not depend on the
// packing.  Called by every thread of the block (it holds two block barriers).
template <class U, class R, int T>
__device__ __forceinline__ void pooled_update(R (&p)[6], R (&P)[21], bool job, const float4 &h, const float2 &hv,
                                              bool disk, float *st, unsigned *bal_s, int rot)
{
    constexpr int W = T / 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned bal = __ballot_sync(kFull, job);
    if (lane == 0) bal_s[warp] = bal;
#pragma unroll
    for (int k = 0; k < 6; ++k) st[k * T + tid] = p[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) st[(6 + k) * T + tid] = P[k];
    if (job) {
        st[27 * T + tid] = h.x;
        st[28 * T + tid] = h.y;
        st[29 * T + tid] = h.z;
        st[30 * T + tid] = hv.x;
        st[31 * T + tid] = hv.y;
    }
    __syncthreads();
    const int e = ((warp - rot) & (W - 1)) * 32 + lane;  // the job this thread runs
    int base = 0, o = -1;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const unsigned b = bal_s[w];
        const int c = __popc(b);
        if (o < 0 && e < base + c) o = w * 32 + nth_set_bit(b, e - base);
        base += c;
    }
    if (o >= 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] = st[k * T + o];
#pragma unroll
        for (int k = 0; k < 21; ++k) P[k] = st[(6 + k) * T + o];
        const R hx = st[27 * T + o], hy = st[28 * T + o], hz = st[29 * T + o];
        const R vu = st[30 * T + o], vv = st[31 * T + o];
        U dc2 = U(0);
        if (disk)
            kalman_update<U, R, true>(p, P, hx, hy, hz, vu, vv, &dc2);
        else
            kalman_update<U, R, false>(p, P, hx, hy, hz, vu, vv, &dc2);
#pragma unroll
        for (int k = 0; k < 6; ++k) st[k * T + o] = p[k];
#pragma unroll
        for (int k = 0; k < 21; ++k) st[(6 + k) * T + o] = P[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = st[k * T + tid];
#pragma unroll
    for (int k = 0; k < 21; ++k) P[k] = st[(6 + k) * T + tid];
}

// Mixed precision packs the block's Kalman updates into full warps (pooled_update), in blocks of
// TKF_POOL_WARPS warps.
#ifndef TKF_BUILD_POOL
#define TKF_BUILD_POOL 1
#endif
#ifndef TKF_POOL_WARPS
#define TKF_POOL_WARPS 4
#endif
template <class R, class U> struct BuildThreads {
    static constexpr bool pool = TKF_BUILD_POOL && sizeof(R) == 4 && sizeof(U) == 8;
    static constexpr int value = pool ? 32 * TKF_POOL_WARPS : kBuildThreads;
};

// Resident blocks per SM requested from the register allocator: the all-float kernels with up
// to 6 candidates are held to 72 registers per thread (7 blocks of 128 threads), their two-step
// forms to 80 (6 blocks, a few spills: 4.37 ms for the 160-event module batch against 4.51 ms at
// 5 blocks and 4.77 ms at 4; one seed's near-tie of 701 095 resolves the other way);
// the mixed-precision kernels with up to 6 candidates to 85 (6 blocks, spilling; the barrel's
// one-step kernel) or 102 (5 blocks; its two-step and endcap forms): with the pooled updates
// more resident blocks keep the double-precision pipes fed while other blocks scan (640-event
// build 32.0 ms at 6 blocks, 33.1 ms at 5, 36.0 ms at 4 and 39.8 ms at 3, the same hit lists); the
// wider lists and the all-double kernels keep their natural register count.
#ifndef TKF_BUILD_MINBLOCKS_F32
#define TKF_BUILD_MINBLOCKS_F32 7
#endif
#ifndef TKF_BUILD2_MINBLOCKS_F32
#define TKF_BUILD2_MINBLOCKS_F32 6
#endif
#ifndef TKF_BUILD_MINBLOCKS_MIXED
#define TKF_BUILD_MINBLOCKS_MIXED 6
#endif
#ifndef TKF_BUILD2_MINBLOCKS_MIXED
#define TKF_BUILD2_MINBLOCKS_MIXED 5
#endif
template <int NMAX, class R, class U, bool kTwo, bool kDisk> struct BuildMinBlocks {
    static constexpr int value =
        (sizeof(R) == 4 && sizeof(U) == 4 && NMAX <= 6)
            ? (kTwo ? TKF_BUILD2_MINBLOCKS_F32 : TKF_BUILD_MINBLOCKS_F32)
            : ((sizeof(R) == 4 && sizeof(U) == 8 && NMAX <= 6)
                   ? (kTwo || kDisk ? TKF_BUILD2_MINBLOCKS_MIXED : TKF_BUILD_MINBLOCKS_MIXED)
                   : 1);
};

// kExactN: the candidates kept per seed equal NMAX, so the segment width and the merge's loops
// are compile-time constants (unrolled); otherwise N = a.ncand <= NMAX at run time.
// kDisk: the configuration has endcap disks; each layer then goes by its kind (cylinder or disk).
template <int NMAX, class R, class U, bool kTwo, bool kExactN, bool kDisk>
__global__ void __launch_bounds__((BuildThreads<R, U>::value), (BuildMinBlocks<NMAX, R, U, kTwo, kDisk>::value))
    k_build(const BuildArgs a)
{
    constexpr int kThreads = BuildThreads<R, U>::value;
    constexpr int W = kThreads / 32;
    constexpr bool kPool = BuildThreads<R, U>::pool;
    static_assert((W & (W - 1)) == 0, "pooled updates rotate over a power-of-two number of warps");
    __shared__ int hist_hit[W][TKF_MAX_LAYERS][32];
    __shared__ signed char hist_par[W][TKF_MAX_LAYERS][32];
    __shared__ float pool_st[kPool ? 32 * kThreads : 1];
    __shared__ unsigned pool_bal[W];
    __shared__ int pool_tile;
    int pool_step = blockIdx.x;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = kExactN ? NMAX : a.ncand;
    const int spw = 32 / N;
    const int grp = lane / N;
    const int r = lane - grp * N;
    const int gbase = grp * N;
    const bool lane_ok = grp < spw;
    const R kb = pick<R>(a.kb_f, a.kb), mass = pick<R>(a.mass_f, a.mass);

    // each warp pulls tiles of seeds_per_block seeds from the counter (no block barrier: a warp
    // that finishes early takes the next tile at once).  With pooled updates the block pulls W
    // tiles at once, one per warp, and its warps go through the layers together.
    for (;;) {
        long long t0;
        if (kPool) {
            if (threadIdx.x == 0) pool_tile = atomicAdd(a.tile_counter, 1);
            __syncthreads();
            const long long b0 = (long long)pool_tile * W * a.seeds_per_block;
            __syncthreads();  // every warp has read pool_tile before the next pull rewrites it
            if (b0 >= a.n_seeds) return;
            t0 = b0 + (long long)warp * a.seeds_per_block;
        } else {
            int tile = 0;
            if (lane == 0) tile = atomicAdd(a.tile_counter, 1);
            tile = __shfl_sync(kFull, tile, 0);
            t0 = (long long)tile * a.seeds_per_block;
            if (t0 >= a.n_seeds) return;
        }
        const int t1 = (int)min((long long)a.n_seeds, t0 + a.seeds_per_block);  // <= t0: no seed (pooled)
        // the same number of seed groups in every warp of a pooled block
        const int n_groups = kPool ? (a.seeds_per_block + spw - 1) / spw : (int)((t1 - t0 + spw - 1) / spw);
        for (int it = 0; it < n_groups; ++it) {
            const int sb = (int)t0 + it * spw;
            const int slot = sb + grp;
            bool has = lane_ok && slot < t1;
            const int seed = has ? (a.s_perm ? __ldg(&a.s_perm[slot]) : slot) : 0;
            const int ev = (has && a.s_event) ? a.s_event[seed] : 0;
            if (has && (ev < 0 || ev >= a.n_events)) {
                atomicOr(a.err, kErrBadEvent);
                if (r == 0) {
                    const R zp[6] = {}, zc[21] = {};
                    store_track<R>(a.o_par, a.o_cov, a.o_chi2, a.o_stride, seed, zp, zc, R(0));
                    a.o_nhits[seed] = TKF_TRACK_LOST;
                }
                has = false;
            }
            R p[6], P[21], chi2 = R(0);
            int nh = 0;
            bool alive = has && r == 0;
#pragma unroll
            for (int k = 0; k < 6; ++k) p[k] = R(0);
#pragma unroll
            for (int k = 0; k < 21; ++k) P[k] = R(0);
            if (alive) {
                const R *sp = (const R *)a.s_par, *sc_ = (const R *)a.s_cov;
#pragma unroll
                for (int k = 0; k < 6; ++k) p[k] = sp[(size_t)k * a.s_stride + seed];
#pragma unroll
                for (int k = 0; k < 21; ++k) P[k] = sc_[(size_t)k * a.s_stride + seed];
                chi2 = ((const R *)a.s_chi2)[seed];
                nh = a.s_nhits[seed];
            }
            int ns = 0;
            for (int l = a.first; l < a.L; ++l) {
                const R Rl = pick<R>(a.radius_f[l], a.radius[l]);
                const bool disk = kDisk && ((a.disk_mask >> l) & 1u);
                const R zd = pick<R>(a.disk_z_f[l], a.disk_z[l]);
                const bool ok = alive && (disk ? propagate_plane<R>(p, P, p[2] >= R(0) ? zd : -zd, kb)
                                               : propagate<R>(p, P, Rl, kb));
                unsigned lk[NMAX];
                int lh[NMAX];
#pragma unroll
                for (int i = 0; i < NMAX; ++i) {
                    lk[i] = kEmpty32;
                    lh[i] = 0;
                }
                if (ok) {
                    if (l == a.first && a.f_key) {
                        // the first layer's window was scanned one lane per seed (k_first_scan)
#pragma unroll
                        for (int i = 0; i < NMAX; ++i) {
                            lk[i] = __ldg(&a.f_key[(size_t)i * a.n_seeds + seed]);
                            lh[i] = __ldg(&a.f_hit[(size_t)i * a.n_seeds + seed]);
                        }
                    } else if (disk) {
                        scan_window_disk<NMAX, R>(a, ev, l, p, P, chi2, nh, r, lk, lh);
                    } else {
                        scan_window<NMAX, R, kTwo>(a, ev, l, Rl, p, P, chi2, nh, r, lk, lh);
                    }
                }

                // merge the segment's lists: N rounds of a segmented minimum
                unsigned mine = kEmpty32;
                int mine_h = 0;
                ns = 0;
                for (int k = 0; k < N; ++k) {
                    if (!__any_sync(kFull, lk[0] != kEmpty32)) break;  // no segment has branches left
                    unsigned m = lk[0];
                    for (int off = 1; off < N; off <<= 1) {
                        const unsigned o = __shfl_down_sync(kFull, m, off);
                        if (r + off < N && o < m) m = o;
                    }
                    m = __shfl_sync(kFull, m, gbase);
                    // the winner is the lane whose rank is the key's parent field
                    const int hsel = __shfl_sync(kFull, lh[0], lane_ok ? gbase + (int)(m & 0xFu) : lane);
                    if (m != kEmpty32) {
                        if (lk[0] == m) list_pop32(lk, lh);
                        if (r == k) {
                            mine = m;
                            mine_h = hsel;
                        }
                        ns = k + 1;
                    }
                }

                // survivors take their parent's predicted state
                const int parent = mine != kEmpty32 ? (int)(mine & 0xFu) : r;
                const int src = lane_ok ? gbase + parent : lane;
#pragma unroll
                for (int k = 0; k < 6; ++k) p[k] = __shfl_sync(kFull, p[k], src);
#pragma unroll
                for (int k = 0; k < 21; ++k) P[k] = __shfl_sync(kFull, P[k], src);
                const R pchi2 = __shfl_sync(kFull, chi2, src);
                alive = mine != kEmpty32;
                int gh = -1;
                float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
                float2 hv = make_float2(0.f, 0.f);
                if (alive) {
                    nh = 31 - (int)(mine >> 27);
                    // the total the ranking used (the scan's sum); FP64 keeps its own exact sum
                    chi2 = sizeof(R) == 8 ? pchi2 : R(key_chi2(mine));
                    if (mine_h != kHoleId) {
                        gh = __ldg(&a.ev_off[ev]) + mine_h;
                        const int pos = __ldg(&a.pos_of_hit[gh]);
                        h = __ldg(&a.hxyzi[pos]);
                        hv = __ldg(&a.hvar[pos]);
                        // the second step, to the hit's own radius (the scan took the same step
                        // for this hit's chi2, so it succeeds here too)
                        if (kTwo) propagate<R, kPropStep>(p, P, sq(R(h.x) * R(h.x) + R(h.y) * R(h.y)), kb);
                    }
                }
                if (kPool) {
                    pooled_update<U, R, kThreads>(p, P, gh >= 0, h, hv, disk, pool_st, pool_bal, pool_step & (W - 1));
                    ++pool_step;
                } else if (gh >= 0) {
                    U dc2 = U(0);
                    if (disk)
                        kalman_update<U, R, true>(p, P, R(h.x), R(h.y), R(h.z), R(hv.x), R(hv.y), &dc2);
                    else
                        kalman_update<U, R, false>(p, P, R(h.x), R(h.y), R(h.z), R(hv.x), R(hv.y), &dc2);
                    if (sizeof(R) == 8) chi2 = pchi2 + R(dc2);
                }
                if (alive) {
                    if (l < a.L - 1) scatter<R>(p, P, pick<R>(a.xx0_f[l], a.xx0[l]), mass, disk);
                    hist_hit[warp][l][lane] = gh;
                    hist_par[warp][l][lane] = (signed char)parent;
                }
            }
            __syncwarp();
            if (has && r == 0) {
                if (ns > 0) {
                    store_track<R>(a.o_par, a.o_cov, a.o_chi2, a.o_stride, seed, p, P, chi2);
                    a.o_nhits[seed] = nh;
                } else {  // every candidate lost: defined zero state
                    const R zp[6] = {}, zc[21] = {};
                    store_track<R>(a.o_par, a.o_cov, a.o_chi2, a.o_stride, seed, zp, zc, R(0));
                    a.o_nhits[seed] = TKF_TRACK_LOST;
                }
                if (a.o_hit) {
                    for (int l = 0; l < a.first; ++l)
                        a.o_hit[(size_t)l * a.o_stride + seed] = a.s_hit ? a.s_hit[(size_t)l * a.s_stride + seed] : -1;
                    int rank = 0;
                    for (int l = a.L - 1; l >= a.first; --l) {
                        const int slot = gbase + rank;
                        a.o_hit[(size_t)l * a.o_stride + seed] = ns > 0 ? hist_hit[warp][l][slot] : -1;
                        rank = hist_par[warp][l][slot];
                    }
                }
            }
            if (a.n_cand_out && has && r == 0) a.n_cand_out[seed] = ns;
            if (a.a_par && has && r < ns) {
                const int o = seed * N + r;
                store_track<R>(a.a_par, a.a_cov, a.a_chi2, a.a_stride, o, p, P, chi2);
                a.a_nhits[o] = nh;
                if (a.a_hit) {
                    for (int l = 0; l < a.first; ++l)
                        a.a_hit[(size_t)l * a.a_stride + o] = a.s_hit ? a.s_hit[(size_t)l * a.s_stride + seed] : -1;
                    int rank = r;
                    for (int l = a.L - 1; l >= a.first; --l) {
                        const int slot = gbase + rank;
                        a.a_hit[(size_t)l * a.a_stride + o] = hist_hit[warp][l][slot];
                        rank = hist_par[warp][l][slot];
                    }
                }
            }
            __syncwarp();
        }
    }
}

// The first building layer, one lane per seed: every seed enters it with one candidate (rank 0),
// so in k_build five of a segment's six lanes would idle through its window scan.  Here each
// lane propagates one seed to the layer and scans its window into the same branch list k_build
// would build, stored as NMAX planes of keys and hit ids indexed by seed; k_build then propagates
// again (the state is needed for the updates) and reads the list instead of scanning.  The same
// functions on the same inputs give the same lists.  Seeds are taken in their input order, not
// k_build's processing order: their states are then read coalesced (in the processing order,
// 29 scattered words per seed left this kernel waiting on memory), and an event's seeds still
// come together, so its hits stay in L2.
template <int NMAX, class R, bool kTwo, bool kDisk>
__global__ void __launch_bounds__(128) k_first_scan(const BuildArgs a)
{
    const int seed = blockIdx.x * blockDim.x + threadIdx.x;
    if (seed >= a.n_seeds) return;
    const int ev = a.s_event ? a.s_event[seed] : 0;
    unsigned lk[NMAX];
    int lh[NMAX];
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        lk[i] = kEmpty32;
        lh[i] = 0;
    }
    if (ev >= 0 && ev < a.n_events) {  // k_build reports a bad event id
        R p[6], P[21];
        const R *sp = (const R *)a.s_par, *sc_ = (const R *)a.s_cov;
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] = sp[(size_t)k * a.s_stride + seed];
#pragma unroll
        for (int k = 0; k < 21; ++k) P[k] = sc_[(size_t)k * a.s_stride + seed];
        const R chi2 = ((const R *)a.s_chi2)[seed];
        const int nh = a.s_nhits[seed];
        const int l = a.first;
        const R kb = pick<R>(a.kb_f, a.kb), Rl = pick<R>(a.radius_f[l], a.radius[l]);
        const bool disk = kDisk && ((a.disk_mask >> l) & 1u);
        const R zd = pick<R>(a.disk_z_f[l], a.disk_z[l]);
        const bool ok = disk ? propagate_plane<R>(p, P, p[2] >= R(0) ? zd : -zd, kb) : propagate<R>(p, P, Rl, kb);
        if (ok) {
            if (disk)
                scan_window_disk<NMAX, R>(a, ev, l, p, P, chi2, nh, 0, lk, lh);
            else
                scan_window<NMAX, R, kTwo>(a, ev, l, Rl, p, P, chi2, nh, 0, lk, lh);
        }
    }
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        a.f_key[(size_t)i * a.n_seeds + seed] = lk[i];
        a.f_hit[(size_t)i * a.n_seeds + seed] = lh[i];
    }
}

#ifndef TKF_BUILD_EXACT_N
#define TKF_BUILD_EXACT_N 1
#endif
template <class R, class U, bool kTwo = false, bool kDisk = false>
cudaError_t launch_build_t(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy)
{
    const void *fn = nullptr;
    const bool exact = TKF_BUILD_EXACT_N && a.ncand == nmax;
#define TKF_K(n, e) (const void *)k_build<n, R, U, kTwo, e, kDisk>
    switch (nmax) {
    case 1: fn = TKF_K(1, true); break;
    case 4: fn = exact ? TKF_K(4, true) : TKF_K(4, false); break;
    case 6: fn = exact ? TKF_K(6, true) : TKF_K(6, false); break;
    case 10: fn = exact ? TKF_K(10, true) : TKF_K(10, false); break;
    case 16: fn = exact ? TKF_K(16, true) : TKF_K(16, false); break;
    default: return cudaErrorInvalidValue;
    }
#undef TKF_K
    constexpr int threads = BuildThreads<R, U>::value;
    if (occupancy) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, fn, threads, 0);
    void *args[] = {(void *)&a};
    if (a.f_key && a.first < a.L && a.n_seeds > 0) {
        const void *ff = nullptr;
#define TKF_F(n) (const void *)k_first_scan<n, R, kTwo, kDisk>
        switch (nmax) {
        case 1: ff = TKF_F(1); break;
        case 4: ff = TKF_F(4); break;
        case 6: ff = TKF_F(6); break;
        case 10: ff = TKF_F(10); break;
        default: ff = TKF_F(16); break;
        }
#undef TKF_F
        const cudaError_t e = cudaLaunchKernel(ff, dim3((a.n_seeds + 127) / 128), dim3(128), args, 0, s);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, 0, s);
}

}  // namespace tkf
