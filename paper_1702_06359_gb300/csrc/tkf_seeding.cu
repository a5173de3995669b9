// Seeding from hit triplets on layers 0, 1, 2 with a confirmation hit on layer 3 (the seeding
// stage of Sec. 2, which the paper names without specifying): tkf_find_seeds.
//
// The search walks the hit index: for each layer-0 hit, the layer-1 cells (eta row, phi
// sixteenths) that a circle from the beam line through the hit can reach with |curvature| <=
// kappa_max and a z-vertex within z_vertex; for every pair that passes, the layer-2 cells around
// the pair's extrapolation; for every triplet that passes, the layer-3 cells around the triplet
// circle's crossing.  The windows only choose index ranges; every hit in them is tested against
// the exact cuts, so the seeds are those of a scan over all hits of the layers.  A warp owns 32
// consecutive index positions and shares their work out over its lanes through queues in shared
// memory (k_seed_find below); the lane of each layer-0 hit keeps that hit's triplet of smallest
// score.  Seeds are then compacted in the index order of their first hits (event by event,
// eta-phi cell by cell), which keeps a warp's seeds near one another for the building that
// follows.
//
// Circle quantities are evaluated in the frame of the first hit a: with b' = b - a and
// c' = c - a, the circle through a, b, c has centre a + w / (2 det) (det = b' x c',
// w = (c'_y |b'|^2 - b'_y |c'|^2, b'_x |c'|^2 - c'_x |b'|^2)), curvature 2 |det| / |w| and unit
// normal n = sign(det) w / |w|, and a point p lies at f(p) = kappa |p - a|^2 / 2 - (p - a) . n
// from it (the point's power divided by the diameter).  None of these subtracts two numbers
// of the size of the radius, so they keep FP32 accuracy for the straight tracks of high pT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "internal.h"
#include "kf_math.cuh"

using namespace tkf;

namespace {

constexpr int kSeedThreads = 256;
constexpr float kInf = 3.0e38f;

struct SeedGeom {
    int L, n_eta, n_phi, n_bins, n_events;
    float R[4];           // radii of layers 0..3
    float eta_min, inv_eta_w, phi_scale;
    float kmax;           // curvature limit
    float zv, d0, dz, w3, z3;
    float lim01, lim12, lim23;  // transverse chord limits 2 (R_{l+1} - R_l)
    float hit_dr;
    int confirm;
};

__device__ __forceinline__ int seed_find_event(const int *off, int n_events, int i)
{  // largest e with off[e] <= i
    int lo = 0, hi = n_events;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&off[mid]) <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// eta bins [b0, b1] of z in [z_lo, z_hi] on the cylinder of radius R (eta = asinh(z / R)), with
// 1e-3 of slack in eta for the index's own rounding
__device__ __forceinline__ void eta_bins(const SeedGeom &g, float R, float z_lo, float z_hi, int &b0, int &b1)
{
    auto eta = [&](float z) {
        const float t = z / R, at = fabsf(t);
        return copysignf(fast_log(at + sqrtf(at * at + 1.f)), t);
    };
    b0 = (int)floorf((eta(z_lo) - 1e-3f - g.eta_min) * g.inv_eta_w);
    b1 = (int)floorf((eta(z_hi) + 1e-3f - g.eta_min) * g.inv_eta_w);
    b0 = max(0, min(b0, g.n_eta - 1));
    b1 = max(0, min(b1, g.n_eta - 1));
}

// The phi window [phi - half, phi + half] as at most two runs of consecutive (phi bin, phi
// sixteenth) cells of an eta row (two when it wraps around phi = +-pi): run r covers cells
// lo[r] .. hi[r], a cell numbered bin * kSubBins + sixteenth (hi < lo: empty).
struct PhiWin {
    int lo[2], hi[2];
};

__device__ __forceinline__ PhiWin phi_window(const SeedGeom &g, float phi, float half)
{
    PhiWin w;
    w.lo[1] = 0;
    w.hi[1] = -1;
    const float tp = 2.f * (float)kPi;
    phi -= tp * floorf((phi + (float)kPi) / tp);  // into [-pi, pi)
    const float c_lo = (phi - half + (float)kPi) * g.phi_scale, c_hi = (phi + half + (float)kPi) * g.phi_scale;
    const int nphi = g.n_phi, last = nphi * kSubBins - 1;
    if (!(c_hi - c_lo < (float)(nphi - 1)) || !(c_lo > (float)-nphi) || !(c_hi < (float)(2 * nphi))) {
        w.lo[0] = 0;  // the whole row
        w.hi[0] = last;
        return w;
    }
    const int k0 = (int)floorf(c_lo), k1 = (int)floorf(c_hi);
    const int s0 = min(max((int)floorf((c_lo - (float)k0) * (float)kSubBins), 0), kSubBins - 1);
    const int s1 = min(max((int)floorf((c_hi - (float)k1) * (float)kSubBins), 0), kSubBins - 1);
    if (k0 < 0) {
        w.lo[0] = (k0 + nphi) * kSubBins + s0;
        w.hi[0] = last;
        w.hi[1] = k1 * kSubBins + s1;
    } else if (k1 >= nphi) {
        w.lo[0] = k0 * kSubBins + s0;
        w.hi[0] = last;
        w.hi[1] = (k1 - nphi) * kSubBins + s1;
    } else {
        w.lo[0] = k0 * kSubBins + s0;
        w.hi[0] = k1 * kSubBins + s1;
    }
    return w;
}

// start of phi sixteenth t (1 <= t < kSubBins) of a bin from its packed bin_sub word (byte t - 1)
__device__ __forceinline__ int sixteenth_start(const uint4 w, int t)
{
    const unsigned word = t <= 4 ? w.x : (t <= 8 ? w.y : (t <= 12 ? w.z : w.w));
    return (int)((word >> (8 * ((t - 1) & 3))) & 0xFFu);
}

// A walk over the hits of a window: eta rows eb .. e1 of one (event, layer) segment, runs 0 and 1
// of the phi window in each row.  [j, jend) is the range being read; [jn, jen) the next one,
// fetched ahead (its index loads are issued when the walk moves to the current range, so they
// arrive while the current range is read); (eb, r) is the row and run the fetch after that takes.
struct Walk {
    int eb, e1, r, j, jend, jn, jen;
};

// the positions of run r of the phi window in eta row eb of segment seg
__device__ __forceinline__ void run_range(const SeedGeom &g, const int *bin_off, const uint4 *bin_sub, int seg,
                                          int eb, int lo, int hi, int &j, int &jend)
{
    const int row = seg * g.n_bins + eb * g.n_phi;
    const int ps0 = lo & (kSubBins - 1), ps1 = hi & (kSubBins - 1);
    const int ba = row + lo / kSubBins, bb = row + hi / kSubBins;
    const int oa = __ldg(&bin_off[ba]), ob = __ldg(&bin_off[bb]), ob1 = __ldg(&bin_off[bb + 1]);
    const uint4 wa = __ldg(&bin_sub[ba]), wb = __ldg(&bin_sub[bb]);
    j = oa + ((ps0 <= 0 || wa.w == 0xFFFFFFFFu) ? 0 : sixteenth_start(wa, ps0));
    jend = ob + ((ps1 >= kSubBins - 1 || wb.w == 0xFFFFFFFFu) ? ob1 - ob : sixteenth_start(wb, ps1 + 1));
}

// fetches the next run of the window into [jn, jen) (empty once the window is exhausted)
__device__ __forceinline__ void walk_fetch(const SeedGeom &g, const int *bin_off, const uint4 *bin_sub, int seg,
                                           const PhiWin &w, Walk &k)
{
    k.jn = k.jen = 0;
    while (k.eb <= k.e1) {
        if (k.r >= 2) {
            k.r = 0;
            ++k.eb;
            continue;
        }
        const int lo = k.r == 0 ? w.lo[0] : w.lo[1], hi = k.r == 0 ? w.hi[0] : w.hi[1];
        ++k.r;
        if (hi < lo) continue;
        run_range(g, bin_off, bin_sub, seg, k.eb, lo, hi, k.jn, k.jen);
        return;
    }
}

// a walk over eta rows e0 .. e1: the first run current, the second fetched
__device__ __forceinline__ Walk walk_start(const SeedGeom &g, const int *bin_off, const uint4 *bin_sub, int seg,
                                           const PhiWin &w, int e0, int e1)
{
    Walk k{e0, e1, 0, 0, 0, 0, 0};
    walk_fetch(g, bin_off, bin_sub, seg, w, k);
    k.j = k.jn;
    k.jend = k.jen;
    walk_fetch(g, bin_off, bin_sub, seg, w, k);
    return k;
}

// the next hit position of the walk: false when exhausted; moves over empty runs
__device__ __forceinline__ bool walk_next(const SeedGeom &g, const int *bin_off, const uint4 *bin_sub, int seg,
                                          const PhiWin &w, Walk &k, int &pos)
{
    while (k.j >= k.jend) {
        if (k.jn >= k.jen && k.eb > k.e1) return false;
        k.j = k.jn;
        k.jend = k.jen;
        walk_fetch(g, bin_off, bin_sub, seg, w, k);
    }
    pos = k.j++;
    return true;
}

// Queues of one warp: its 32 first hits (slot = lane), passing pairs waiting for their layer-2
// scan, layer-2 hits within the pair's chord and z cuts waiting for the circle through the
// three, passing triplets waiting for their confirmation scan.  Entries are appended in (step,
// lane) order, so the queues' contents do not depend on timing.
constexpr int kQueue = 64;
constexpr int kQueueF = 96;  // a step appends up to 64 to fewer than 32 queued
struct WarpQueues {
    float4 a[32];  // x, y, z, r of the slot's first hit
    float pha[32];
    int seg0[32];  // event * L
    int p_slot[kQueue], p_b[kQueue];
    float p_k01[kQueue], p_slope[kQueue];
    int f_slot[kQueueF], f_b[kQueueF], f_c[kQueueF];
    float f_dz[kQueueF];
    int t_slot[kQueue], t_b[kQueue], t_c[kQueue];
    float t_s2[kQueue], t_kap[kQueue], t_nx[kQueue], t_ny[kQueue], t_d0[kQueue];
};

// Every lane reaches the warp-wide operations below: the loops are warp-uniform, and the lanes
// without work carry their flags through them.
// Held to 3 blocks of 256 threads per SM (80 registers, a few bytes spilled; the queues take
// 42 KB of shared memory per block).
#ifndef TKF_SEED_MINBLOCKS
#define TKF_SEED_MINBLOCKS 3
#endif
__global__ void __launch_bounds__(kSeedThreads, TKF_SEED_MINBLOCKS)
k_seed_find(const SeedGeom g, const float4 *__restrict__ hxyzi, const int *__restrict__ bin_off,
            const uint4 *__restrict__ bin_sub, const int *__restrict__ ev_off, int n, int *__restrict__ res_b,
            int *__restrict__ res_c, float *__restrict__ res_s)
{
    __shared__ WarpQueues s_q[kSeedThreads / 32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    WarpQueues &q = s_q[threadIdx.x >> 5];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;

    // this lane's first hit
    bool valid = false;
    int e = 0, seg0 = 0;
    float ax = 0.f, ay = 0.f, az = 0.f, ra = 1.f, pha = 0.f;
    if (t < n) {
        e = seed_find_event(ev_off, g.n_events, t);
        seg0 = e * g.L;
        if (t < __ldg(&bin_off[(seg0 + 1) * g.n_bins])) {
            const float4 A = hxyzi[t];
            ax = A.x; ay = A.y; az = A.z;
            ra = sqrtf(ax * ax + ay * ay);
            valid = ra > 1e-6f;  // a hit on the beam line starts no seed
            if (!valid) ra = 1.f;
            pha = atan2f(ay, ax);
        }
    }
    q.a[lane] = make_float4(ax, ay, az, ra);
    q.pha[lane] = pha;
    q.seg0[lane] = seg0;
    float best_s = kInf;
    int best_b = 0x7fffffff, best_c = 0x7fffffff;

    // layer-1 window: circles from the beam line through a with |kappa| <= kmax, z-vertex cut
    Walk cb{0, -1, 0, 0, 0, 0, 0};
    int e0 = 0, e1 = -1;
    PhiWin w1;
    w1.lo[0] = w1.lo[1] = 0;
    w1.hi[0] = w1.hi[1] = -1;
    if (valid) {
        const float R1 = g.R[1];
        const float rlo = R1 - g.hit_dr, rhi = R1 + g.hit_dr;
        const float zpad = 1e-3f + 1e-5f * fabsf(az);
        const float zc_lo = fminf(az * rlo / ra - g.zv * (rlo / ra - 1.f), az * rhi / ra - g.zv * (rhi / ra - 1.f));
        const float zc_hi = fmaxf(az * rlo / ra + g.zv * (rlo / ra - 1.f), az * rhi / ra + g.zv * (rhi / ra - 1.f));
        eta_bins(g, R1, zc_lo - zpad, zc_hi + zpad, e0, e1);
        const float s1 = g.kmax * rhi * 0.5f;
        const float half = s1 >= 1.f ? 4.f : asinf(s1) - asinf(g.kmax * ra * 0.5f) + 2e-3f;
        w1 = phi_window(g, pha, half);
        cb = walk_start(g, bin_off, bin_sub, seg0 + 1, w1, e0, e1);
    }
    bool more = valid;
    __syncwarp();

    int n_p = 0, n_f = 0, n_t = 0;  // queued pairs, layer-2 candidates and triplets (warp-uniform)

    // the confirmation scan of the first cnt queued triplets, one per lane, folded into the
    // best triplet of each slot (held by the slot's lane); then the queue's rest moves up
    auto confirm = [&](int cnt) {
        const bool has = lane < cnt;
        int ts = 0, tb = 0, tc = 0, b_id = 0, c_id = 0;
        float s = kInf;
        if (has) {
            ts = q.t_slot[lane];
            tb = q.t_b[lane];
            tc = q.t_c[lane];
            const float s2 = q.t_s2[lane];
            const float4 B = hxyzi[tb], Cc = hxyzi[tc];
            b_id = __float_as_int(B.w);
            c_id = __float_as_int(Cc.w);
            if (!g.confirm) {
                s = s2;
            } else {
                const float4 A = q.a[ts];
                const float kap = q.t_kap[lane], nx = q.t_nx[lane], ny = q.t_ny[lane], d0 = q.t_d0[lane];
                const float rb = sqrtf(B.x * B.x + B.y * B.y), rc = sqrtf(Cc.x * Cc.x + Cc.y * Cc.y);
                if (rc != rb) {
                    const float slope23 = (Cc.z - B.z) / (rc - rb);
                    // where the circle crosses r = R3 nearest to c: its centre is U = a + rho n, and
                    // the crossing lies along U at (R3^2 + 2 rho d0) / (2 |U|) (|U|^2 - rho^2 = 2 rho d0)
                    const float rho = 1.f / kap;
                    const float ux = A.x + rho * nx, uy = A.y + rho * ny;
                    const float D = sqrtf(ux * ux + uy * uy);
                    const float R3 = g.R[3];
                    const float along = (R3 * R3 + 2.f * rho * d0) / (2.f * D);
                    const float h2 = R3 * R3 - along * along;
                    if (h2 >= 0.f) {
                        const float h = sqrtf(h2), ex = ux / D, ey = uy / D;
                        const float px1 = along * ex - h * ey, py1 = along * ey + h * ex;
                        const float px2 = along * ex + h * ey, py2 = along * ey - h * ex;
                        const bool first = (px1 - Cc.x) * (px1 - Cc.x) + (py1 - Cc.y) * (py1 - Cc.y) <=
                                           (px2 - Cc.x) * (px2 - Cc.x) + (py2 - Cc.y) * (py2 - Cc.y);
                        const float ph3 = atan2f(first ? py1 : py2, first ? px1 : px2);
                        const float zc3 = B.z + slope23 * (R3 - rb);
                        int h0b, h1b;
                        const float wz = g.z3 + 1e-3f + 1e-5f * fabsf(zc3) + g.hit_dr * fabsf(slope23);
                        eta_bins(g, R3, zc3 - wz, zc3 + wz, h0b, h1b);
                        const PhiWin w3 =
                            phi_window(g, ph3, (3.f * g.w3 + 0.02f + 2.f * g.hit_dr * kap) / (R3 - g.hit_dr) + 2e-3f);
                        const int seg3 = q.seg0[ts] + 3;
                        Walk ce = walk_start(g, bin_off, bin_sub, seg3, w3, h0b, h1b);
                        float c3 = kInf;
                        int je;
                        while (walk_next(g, bin_off, bin_sub, seg3, w3, ce, je)) {
                            {
                                const float4 E = hxyzi[je];
                                const float d23x = E.x - Cc.x, d23y = E.y - Cc.y;
                                if (!(sqrtf(d23x * d23x + d23y * d23y) <= g.lim23)) continue;
                                const float qx = E.x - A.x, qy = E.y - A.y;
                                const float f3 = kap * (qx * qx + qy * qy) * 0.5f - (qx * nx + qy * ny);
                                const float re = sqrtf(E.x * E.x + E.y * E.y);
                                const float dz3 = E.z - (B.z + slope23 * (re - rb));
                                if (!(fabsf(f3) <= g.w3) || !(fabsf(dz3) <= g.z3)) continue;
                                const float pu = f3 / g.w3, pv = dz3 / g.z3;
                                c3 = fminf(c3, pu * pu + pv * pv);
                            }
                        }
                        if (c3 < kInf) s = s2 + c3;
                    }
                }
            }
        }
        unsigned m = __ballot_sync(full, s < kInf);
        while (m) {
            const int k = __ffs(m) - 1;
            m &= m - 1u;
            const int ks = __shfl_sync(full, ts, k), kb = __shfl_sync(full, b_id, k), kc = __shfl_sync(full, c_id, k);
            const float kv = __shfl_sync(full, s, k);
            if (lane == ks && (kv < best_s || (kv == best_s && (kb < best_b || (kb == best_b && kc < best_c))))) {
                best_s = kv;
                best_b = kb;
                best_c = kc;
            }
        }
        // the queue's rest (fewer than 32 entries) to its front
        const bool mv = lane + cnt < n_t;
        int r_slot = 0, r_b = 0, r_c = 0;
        float r_s2 = 0.f, r_kap = 0.f, r_nx = 0.f, r_ny = 0.f, r_d0 = 0.f;
        if (mv) {
            const int k = lane + cnt;
            r_slot = q.t_slot[k]; r_b = q.t_b[k]; r_c = q.t_c[k]; r_s2 = q.t_s2[k];
            r_kap = q.t_kap[k]; r_nx = q.t_nx[k]; r_ny = q.t_ny[k]; r_d0 = q.t_d0[k];
        }
        __syncwarp();
        if (mv) {
            q.t_slot[lane] = r_slot; q.t_b[lane] = r_b; q.t_c[lane] = r_c; q.t_s2[lane] = r_s2;
            q.t_kap[lane] = r_kap; q.t_nx[lane] = r_nx; q.t_ny[lane] = r_ny; q.t_d0[lane] = r_d0;
        }
        n_t -= cnt;
        __syncwarp();
    };

    // the circle through the first cnt queued candidates (a, b, c), one per lane: curvature and
    // d0 cuts and the score without confirmation; passing triplets join the triplet queue
    auto circle = [&](int cnt) {
        const bool has = lane < cnt;
        int fs = 0, fb = 0, fc = 0;
        float dz = 0.f;
        if (has) {
            fs = q.f_slot[lane]; fb = q.f_b[lane]; fc = q.f_c[lane]; dz = q.f_dz[lane];
        }
        const float best_fs = __shfl_sync(full, best_s, fs);
        bool pass = false;
        float s2 = 0.f, kap = 0.f, nx = 0.f, ny = 0.f, d0 = 0.f;
        if (has) {
            const float4 A = q.a[fs], B = hxyzi[fb], Cc = hxyzi[fc];
            const float bx = B.x - A.x, by = B.y - A.y, cx = Cc.x - A.x, cy = Cc.y - A.y;
            const float det = bx * cy - by * cx;
            if (det != 0.f) {
                const float bb2 = bx * bx + by * by, cc2 = cx * cx + cy * cy;
                const float wx = cy * bb2 - by * cc2, wy = bx * cc2 - cx * bb2;
                const float wn = sqrtf(wx * wx + wy * wy);
                kap = 2.f * fabsf(det) / wn;
                const float sg = det > 0.f ? 1.f : -1.f;
                nx = sg * wx / wn;
                ny = sg * wy / wn;
                d0 = kap * (A.x * A.x + A.y * A.y) * 0.5f + (A.x * nx + A.y * ny);
                if (kap <= g.kmax && fabsf(d0) <= g.d0) {
                    const float u = d0 / g.d0, v = dz / g.dz;
                    s2 = u * u + v * v;
                    pass = !(s2 > best_fs);  // the confirmation term only adds
                }
            }
        }
        const unsigned m = __ballot_sync(full, pass);
        if (pass) {
            const int k = n_t + __popc(m & below);
            q.t_slot[k] = fs; q.t_b[k] = fb; q.t_c[k] = fc; q.t_s2[k] = s2;
            q.t_kap[k] = kap; q.t_nx[k] = nx; q.t_ny[k] = ny; q.t_d0[k] = d0;
        }
        n_t += __popc(m);
        // the queue's rest (up to 63 entries) to its front, 32 at a time
        for (int base = 0; base < n_f - cnt; base += 32) {
            const bool mv = base + lane + cnt < n_f;
            int r_slot = 0, r_b = 0, r_c = 0;
            float r_dz = 0.f;
            if (mv) {
                const int k = base + lane + cnt;
                r_slot = q.f_slot[k]; r_b = q.f_b[k]; r_c = q.f_c[k]; r_dz = q.f_dz[k];
            }
            __syncwarp();
            if (mv) {
                const int k = base + lane;
                q.f_slot[k] = r_slot; q.f_b[k] = r_b; q.f_c[k] = r_c; q.f_dz[k] = r_dz;
            }
            __syncwarp();
        }
        n_f -= cnt;
        __syncwarp();
        if (n_t >= 32) confirm(32);
    };

    while (true) {
        // (1) pairs: each lane tests the next hit of its first hit's layer-1 window
        while (n_p < 32 && __any_sync(full, more)) {
            bool pass = false;
            int jb = 0;
            float k01 = 0.f, slope = 0.f;
            if (more) {
                more = walk_next(g, bin_off, bin_sub, seg0 + 1, w1, cb, jb);
                if (more) {
                    const float4 B = hxyzi[jb];
                    const float bx = B.x - ax, by = B.y - ay;
                    const float chord01 = sqrtf(bx * bx + by * by);
                    if (chord01 <= g.lim01 && chord01 != 0.f) {
                        const float rb = sqrtf(B.x * B.x + B.y * B.y);
                        k01 = 2.f * (ax * B.y - ay * B.x) / (ra * rb * chord01);
                        if (fabsf(k01) <= g.kmax && rb != ra) {
                            slope = (B.z - az) / (rb - ra);
                            pass = fabsf(az - ra * slope) <= g.zv;
                        }
                    }
                }
            }
            const unsigned m = __ballot_sync(full, pass);
            if (pass) {
                const int k = n_p + __popc(m & below);
                q.p_slot[k] = lane;
                q.p_b[k] = jb;
                q.p_k01[k] = k01;
                q.p_slope[k] = slope;
            }
            n_p += __popc(m);
        }
        __syncwarp();
        if (n_p == 0) break;
        // (2) up to 32 queued pairs, one per lane: the layer-2 window of each
        const int take = min(n_p, 32);
        bool cmore = lane < take;
        int ps = 0, pb = 0;
        float k01 = 0.f, slope = 0.f;
        if (cmore) {
            ps = q.p_slot[lane]; pb = q.p_b[lane]; k01 = q.p_k01[lane]; slope = q.p_slope[lane];
        }
        {
            const bool mv = lane + take < n_p;
            int r_slot = 0, r_b = 0;
            float r_k = 0.f, r_sl = 0.f;
            if (mv) {
                r_slot = q.p_slot[lane + take]; r_b = q.p_b[lane + take];
                r_k = q.p_k01[lane + take]; r_sl = q.p_slope[lane + take];
            }
            __syncwarp();
            if (mv) {
                q.p_slot[lane] = r_slot; q.p_b[lane] = r_b; q.p_k01[lane] = r_k; q.p_slope[lane] = r_sl;
            }
            n_p -= take;
        }
        float4 A = make_float4(0.f, 0.f, 0.f, 1.f);
        float4 B = make_float4(0.f, 0.f, 0.f, 0.f);
        float rb = 0.f;
        int pseg = 0;
        Walk cc{0, -1, 0, 0, 0, 0, 0};
        PhiWin w2;
        w2.lo[0] = w2.lo[1] = 0;
        w2.hi[0] = w2.hi[1] = -1;
        if (cmore) {
            A = q.a[ps];
            pseg = q.seg0[ps];
            B = hxyzi[pb];
            rb = sqrtf(B.x * B.x + B.y * B.y);
            // layer-2 window: z along the r-z line of a and b, phi around the crossing of the circle
            // through the beam line, a and b, widened by the d0 cut's lever arm
            const float R2 = g.R[2], ra_ = A.w;
            const float zc = A.z + slope * (R2 - ra_);
            const float wz = g.dz + 1e-3f + 1e-5f * fabsf(zc) + g.hit_dr * fabsf(slope);
            int f0, f1;
            eta_bins(g, R2, zc - wz, zc + wz, f0, f1);
            // the circles through a and b that pass within d0 of the beam line differ from the one
            // through it by about d0 (R2 - ra) (R2 - rb) / (ra rb) at R2: twice that, plus slack
            float half = 4.f, mid = q.pha[ps];
            if (fabsf(k01) * (R2 + g.hit_dr) * 0.5f < 1.f) {
                const float lever = (R2 - ra_) * (R2 - rb) / (ra_ * rb);
                half = (2.f * g.d0 * fabsf(lever) + 0.01f + 2.f * g.hit_dr * fabsf(k01)) / (R2 - g.hit_dr) + 2e-3f;
                mid = q.pha[ps] + asinf(k01 * R2 * 0.5f) - asinf(k01 * ra_ * 0.5f);
            }
            w2 = phi_window(g, mid, half);
            cc = walk_start(g, bin_off, bin_sub, pseg + 2, w2, f0, f1);
        }
        __syncwarp();
        // (3) each lane tests the next two hits of its pair's layer-2 window against the chord and
        // z cuts; the queue of those that pass goes through the circle cuts 32 at a time.  (One hit
        // per step: 17.3 ms on the 640-event seeding batch, two: 15.8 ms, four: 16.7 ms; two
        // layer-1 hits per pair step were slower too.)
        const float lim12sq = g.lim12 * g.lim12;
        auto near_z = [&](int jc, float &dz) {
            const float4 Cc = hxyzi[jc];
            const float d12x = Cc.x - B.x, d12y = Cc.y - B.y;
            const float rc = sqrtf(Cc.x * Cc.x + Cc.y * Cc.y);
            dz = Cc.z - (A.z + slope * (rc - A.w));
            return d12x * d12x + d12y * d12y <= lim12sq && fabsf(dz) <= g.dz;
        };
        while (__any_sync(full, cmore)) {
            bool p0 = false, p1 = false;
            int jc0 = 0, jc1 = 0;
            float dz0 = 0.f, dz1 = 0.f;
            if (cmore) {
                cmore = walk_next(g, bin_off, bin_sub, pseg + 2, w2, cc, jc0);
                if (cmore) {
                    p0 = near_z(jc0, dz0);
                    cmore = walk_next(g, bin_off, bin_sub, pseg + 2, w2, cc, jc1);
                    if (cmore) p1 = near_z(jc1, dz1);
                }
            }
            const unsigned m0 = __ballot_sync(full, p0), m1 = __ballot_sync(full, p1);
            if (p0) {
                const int k = n_f + __popc(m0 & below);
                q.f_slot[k] = ps; q.f_b[k] = pb; q.f_c[k] = jc0; q.f_dz[k] = dz0;
            }
            n_f += __popc(m0);
            if (p1) {
                const int k = n_f + __popc(m1 & below);
                q.f_slot[k] = ps; q.f_b[k] = pb; q.f_c[k] = jc1; q.f_dz[k] = dz1;
            }
            n_f += __popc(m1);
            __syncwarp();
            while (n_f >= 32) circle(32);
        }
    }
    if (n_f > 0) circle(n_f);
    if (n_t > 0) confirm(n_t);
    if (!valid || t >= n) {
        if (t < n) res_b[t] = -1;
        return;
    }
    if (best_s < kInf) {
        const int base = __ldg(&ev_off[e]);
        res_b[t] = base + best_b;
        res_c[t] = base + best_c;
        res_s[t] = best_s;
    } else {
        res_b[t] = -1;
    }
}

// seeds per block of kSeedThreads positions
__global__ void __launch_bounds__(kSeedThreads) k_seed_count(const int *res_b, int n, int *block_count)
{
    __shared__ int warp_n[kSeedThreads / 32];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool has = t < n && res_b[t] >= 0;
    const int c = __popc(__ballot_sync(0xffffffffu, has));
    if ((threadIdx.x & 31) == 0) warp_n[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kSeedThreads / 32; ++w) s += warp_n[w];
        block_count[blockIdx.x] = s;
    }
}

// exclusive scan of the block counts in one block; the total goes to *total
__global__ void __launch_bounds__(1024) k_seed_scan(int *count, int n, int *total)
{
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < n ? count[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int incl = x + (w > 0 ? warp_sums[w - 1] : 0) + carry;
        if (i < n) count[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// seeds written in position order: block b's seeds start at base[b]
__global__ void __launch_bounds__(kSeedThreads)
k_seed_scatter(const float4 *hxyzi, const int *ev_off, int n_events, const int *res_b, const int *res_c,
               const float *res_s, int n, const int *base, int max_seeds, int *seed_hits, int *seed_event,
               float *seed_score)
{
    __shared__ int warp_n[kSeedThreads / 32];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool has = t < n && res_b[t] >= 0;
    const unsigned m = __ballot_sync(0xffffffffu, has);
    if (lane == 0) warp_n[w] = __popc(m);
    __syncthreads();
    if (!has) return;
    int pos = base[blockIdx.x] + __popc(m & ((1u << lane) - 1u));
    for (int k = 0; k < w; ++k) pos += warp_n[k];
    if (pos >= max_seeds) return;
    const int e = seed_find_event(ev_off, n_events, t);
    seed_hits[pos] = __ldg(&ev_off[e]) + __float_as_int(hxyzi[t].w);
    seed_hits[(size_t)max_seeds + pos] = res_b[t];
    seed_hits[2 * (size_t)max_seeds + pos] = res_c[t];
    seed_event[pos] = e;
    if (seed_score) seed_score[pos] = res_s[t];
}

int seed_fail(tkf_ctx *ctx, int code, const std::string &msg)
{
    ctx->err = msg;
    return code;
}

int seed_cuda(tkf_ctx *ctx, cudaError_t e, const char *what)
{
    return seed_fail(ctx, e == cudaErrorMemoryAllocation ? TKF_ERR_NOMEM : TKF_ERR_CUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" void tkf_default_seed_cuts(tkf_seed_cuts *c)
{
    if (!c) return;
    c->pt_min = 0.5;
    c->kappa_slack = 0.15;
    c->z_vertex = 4.0;
    c->d0_max = 0.08;
    c->dz_max = 0.08;
    c->conf_rphi = 0.1;
    c->conf_z = 0.1;
    c->confirm = 1;
    c->reserved = 0;
}

extern "C" int tkf_find_seeds(tkf_ctx *ctx, const tkf_hit_index *idx, const tkf_seed_cuts *cuts, int32_t max_seeds,
                              int32_t *seed_hits, int32_t *seed_event, float *seed_score, int32_t *n_found,
                              tkf_stream stream)
{
    if (!ctx) return TKF_ERR_INVALID;
    if (!idx || !cuts || !n_found || max_seeds < 0 || (max_seeds > 0 && (!seed_hits || !seed_event)))
        return seed_fail(ctx, TKF_ERR_INVALID, "find_seeds: null argument or negative max_seeds");
    const tkf_config &c = ctx->cfg;
    if (c.n_layers < 4 || idx->n_layers != c.n_layers || idx->n_bins != c.n_eta_bins * c.n_phi_bins)
        return seed_fail(ctx, TKF_ERR_INVALID,
                         "find_seeds: needs an index of at least 4 layers built with this context's bins");
    for (int l = 0; l < 4; ++l)
        if (c.disk_z[l] > 0.0) return seed_fail(ctx, TKF_ERR_INVALID, "find_seeds: layers 0..3 must be cylinders");
    if (!(cuts->pt_min > 0) || !(cuts->kappa_slack >= 0) || !(cuts->z_vertex > 0) || !(cuts->d0_max > 0) ||
        !(cuts->dz_max > 0) || !(cuts->conf_rphi > 0) || !(cuts->conf_z > 0))
        return seed_fail(ctx, TKF_ERR_INVALID, "find_seeds: cuts must be positive");
    if (!(c.radius[0] > 0) || !(c.radius[1] > c.radius[0]) || !(c.radius[2] > c.radius[1]) ||
        !(c.radius[3] > c.radius[2]))
        return seed_fail(ctx, TKF_ERR_INVALID, "find_seeds: layers 0..3 must have increasing radii");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = idx->n;
    const int blocks = std::max(1, (n + kSeedThreads - 1) / kSeedThreads);
    if ((size_t)n > ctx->seed_cap || (size_t)blocks + 1 > ctx->seed_cnt_cap) {
        cudaFree(ctx->seed_b);
        cudaFree(ctx->seed_c);
        cudaFree(ctx->seed_s);
        cudaFree(ctx->seed_cnt);
        ctx->seed_b = ctx->seed_c = ctx->seed_cnt = nullptr;
        ctx->seed_s = nullptr;
        ctx->seed_cap = ctx->seed_cnt_cap = 0;
        const size_t cap = std::max(n, 1), cnt = (size_t)blocks + 1;
        cudaError_t e;
        if ((e = cudaMalloc(&ctx->seed_b, cap * sizeof(int))) != cudaSuccess ||
            (e = cudaMalloc(&ctx->seed_c, cap * sizeof(int))) != cudaSuccess ||
            (e = cudaMalloc(&ctx->seed_s, cap * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&ctx->seed_cnt, cnt * sizeof(int))) != cudaSuccess)
            return seed_cuda(ctx, e, "find_seeds: scratch");
        ctx->seed_cap = cap;
        ctx->seed_cnt_cap = cnt;
    }
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(n_found, 0, sizeof(int32_t), s);
        return e == cudaSuccess ? TKF_OK : seed_cuda(ctx, e, "find_seeds: memset");
    }
    SeedGeom g{};
    g.L = c.n_layers;
    g.n_eta = c.n_eta_bins;
    g.n_phi = c.n_phi_bins;
    g.n_bins = c.n_eta_bins * c.n_phi_bins;
    g.n_events = idx->n_events;
    for (int l = 0; l < 4; ++l) g.R[l] = (float)c.radius[l];
    g.eta_min = (float)c.eta_min;
    g.inv_eta_w = (float)(1.0 / c.eta_bin_w);
    g.phi_scale = (float)(c.n_phi_bins / (2.0 * kPi));
    g.kmax = (float)(0.00299792458 * c.bz / cuts->pt_min * (1.0 + cuts->kappa_slack));
    g.zv = (float)cuts->z_vertex;
    g.d0 = (float)cuts->d0_max;
    g.dz = (float)cuts->dz_max;
    g.w3 = (float)cuts->conf_rphi;
    g.z3 = (float)cuts->conf_z;
    g.lim01 = (float)(2.0 * (c.radius[1] - c.radius[0]));
    g.lim12 = (float)(2.0 * (c.radius[2] - c.radius[1]));
    g.lim23 = (float)(2.0 * (c.radius[3] - c.radius[2]));
    g.hit_dr = (float)c.hit_dr;
    g.confirm = cuts->confirm != 0;
    k_seed_find<<<blocks, kSeedThreads, 0, s>>>(g, idx->hxyzi, idx->bin_off, idx->bin_sub, idx->ev_off, n, ctx->seed_b,
                                                ctx->seed_c, ctx->seed_s);
    k_seed_count<<<blocks, kSeedThreads, 0, s>>>(ctx->seed_b, n, ctx->seed_cnt);
    k_seed_scan<<<1, 1024, 0, s>>>(ctx->seed_cnt, blocks, n_found);
    if (max_seeds > 0)
        k_seed_scatter<<<blocks, kSeedThreads, 0, s>>>(idx->hxyzi, idx->ev_off, idx->n_events, ctx->seed_b,
                                                       ctx->seed_c, ctx->seed_s, n, ctx->seed_cnt, max_seeds,
                                                       seed_hits, seed_event, seed_score);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TKF_OK : seed_cuda(ctx, e, "find_seeds: launch");
}
