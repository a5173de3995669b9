// Seeding from hit triplets on layers 0, 1, 2 with a confirmation hit on layer 3 (the seeding
// stage of Sec. 2, which the paper names without specifying): tkf_find_seeds.
//
// Each hit of layer 0 takes one thread, which walks the hit index: the layer-1 bins that a
// circle from the beam line through the hit can reach with |curvature| <= kappa_max and a
// z-vertex within z_vertex, then for every pair that passes the layer-2 bins around the
// pair's extrapolation, then for every triplet that passes the layer-3 bins around the
// triplet circle's crossing.  The windows only choose bins; every hit in them is tested
// against the exact cuts, so the seeds are those of a scan over all hits of the layers.  The
// thread keeps its triplet of smallest score; seeds are then compacted in the index order of
// their first hits (event by event, eta-phi bin by bin), which keeps a warp's seeds near one
// another for the building that follows.
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

// phi bins of [phi - half, phi + half]: first bin p0 (0 .. n_phi - 1) and count np (wrapping)
__device__ __forceinline__ void phi_bins(const SeedGeom &g, float phi, float half, int &p0, int &np)
{
    if (half >= 3.1f) {
        p0 = 0;
        np = g.n_phi;
        return;
    }
    const float c_lo = (phi - half + (float)kPi) * g.phi_scale, c_hi = (phi + half + (float)kPi) * g.phi_scale;
    const int k0 = (int)floorf(c_lo), k1 = (int)floorf(c_hi);
    np = min(k1 - k0 + 1, g.n_phi);
    p0 = ((k0 % g.n_phi) + g.n_phi) % g.n_phi;
}

// Calls visit(j) for every sorted position j of the hits in the window's bins of one
// (event, layer) segment.
template <class Visit>
__device__ __forceinline__ void for_window(const SeedGeom &g, const int *bin_off, int seg, int e0, int e1, int p0,
                                           int np, Visit visit)
{
    for (int eb = e0; eb <= e1; ++eb) {
        const int row = seg * g.n_bins + eb * g.n_phi;
        for (int k = 0; k < np; ++k) {
            int pb = p0 + k;
            pb -= pb >= g.n_phi ? g.n_phi : 0;
            const int j0 = __ldg(&bin_off[row + pb]), j1 = __ldg(&bin_off[row + pb + 1]);
            for (int j = j0; j < j1; ++j) visit(j);
        }
    }
}

__global__ void __launch_bounds__(kSeedThreads)
k_seed_find(const SeedGeom g, const float4 *__restrict__ hxyzi, const int *__restrict__ bin_off,
            const int *__restrict__ ev_off, int n, int *__restrict__ res_b, int *__restrict__ res_c,
            float *__restrict__ res_s)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int e = seed_find_event(ev_off, g.n_events, t);
    const int seg0 = e * g.L;
    if (t >= __ldg(&bin_off[(seg0 + 1) * g.n_bins])) {  // not on layer 0
        res_b[t] = -1;
        return;
    }
    const float4 A = hxyzi[t];
    const float ax = A.x, ay = A.y, az = A.z;
    const float ra2 = ax * ax + ay * ay, ra = sqrtf(ra2);
    if (!(ra > 1e-6f)) {  // a hit on the beam line starts no seed
        res_b[t] = -1;
        return;
    }
    const float pha = atan2f(ay, ax);
    float best_s = kInf;
    int best_b = 0x7fffffff, best_c = 0x7fffffff;
    const float zpad = 1e-3f + 1e-5f * fabsf(az);

    // layer-1 window: circles from the beam line through a with |kappa| <= kmax, z-vertex cut
    int e0, e1, p0, np;
    {
        const float R1 = g.R[1];
        const float rlo = R1 - g.hit_dr, rhi = R1 + g.hit_dr;
        const float zc_lo = fminf(az * rlo / ra - g.zv * (rlo / ra - 1.f), az * rhi / ra - g.zv * (rhi / ra - 1.f));
        const float zc_hi = fmaxf(az * rlo / ra + g.zv * (rlo / ra - 1.f), az * rhi / ra + g.zv * (rhi / ra - 1.f));
        eta_bins(g, R1, zc_lo - zpad, zc_hi + zpad, e0, e1);
        const float s1 = g.kmax * rhi * 0.5f;
        const float half = s1 >= 1.f ? 4.f : asinf(s1) - asinf(g.kmax * ra * 0.5f) + 2e-3f;
        phi_bins(g, pha, half, p0, np);
    }
    for_window(g, bin_off, seg0 + 1, e0, e1, p0, np, [&](int jb) {
        const float4 B = hxyzi[jb];
        const float bx = B.x - ax, by = B.y - ay;
        const float chord01 = sqrtf(bx * bx + by * by);
        if (!(chord01 <= g.lim01) || chord01 == 0.f) return;
        const float rb = sqrtf(B.x * B.x + B.y * B.y);
        const float k01 = 2.f * (ax * B.y - ay * B.x) / (ra * rb * chord01);
        if (!(fabsf(k01) <= g.kmax) || rb == ra) return;
        const float slope = (B.z - az) / (rb - ra);
        const float zv = az - ra * slope;
        if (!(fabsf(zv) <= g.zv)) return;
        const int b_id = __float_as_int(B.w);
        // layer-2 window: z along the r-z line of a and b, phi around the crossing of the circle
        // through the beam line, a and b, widened by the d0 cut's lever arm
        int f0, f1, q0, nq;
        {
            const float R2 = g.R[2];
            const float zc = az + slope * (R2 - ra);
            const float w = g.dz + 1e-3f + 1e-5f * fabsf(zc) + g.hit_dr * fabsf(slope);
            eta_bins(g, R2, zc - w, zc + w, f0, f1);
            // the circles through a and b that pass within d0 of the beam line differ from the one
            // through it by about d0 (R2 - ra) (R2 - rb) / (ra rb) at R2: twice that, plus slack
            const float s2 = k01 * R2 * 0.5f;
            float half = 4.f, mid = pha;
            if (fabsf(k01) * (R2 + g.hit_dr) * 0.5f < 1.f) {
                const float lever = (R2 - ra) * (R2 - rb) / (ra * rb);
                half = (2.f * g.d0 * fabsf(lever) + 0.01f + 2.f * g.hit_dr * fabsf(k01)) / (R2 - g.hit_dr) + 2e-3f;
                mid = pha + asinf(s2) - asinf(k01 * ra * 0.5f);
            }
            phi_bins(g, mid, half, q0, nq);
        }
        const float bb2 = bx * bx + by * by;
        for_window(g, bin_off, seg0 + 2, f0, f1, q0, nq, [&](int jc) {
            const float4 Cc = hxyzi[jc];
            const float d12x = Cc.x - B.x, d12y = Cc.y - B.y;
            if (!(sqrtf(d12x * d12x + d12y * d12y) <= g.lim12)) return;
            const float cx = Cc.x - ax, cy = Cc.y - ay;
            const float det = bx * cy - by * cx;
            if (det == 0.f) return;
            const float cc2 = cx * cx + cy * cy;
            const float wx = cy * bb2 - by * cc2, wy = bx * cc2 - cx * bb2;
            const float wn = sqrtf(wx * wx + wy * wy);
            const float kap = 2.f * fabsf(det) / wn;
            if (!(kap <= g.kmax)) return;
            const float sg = det > 0.f ? 1.f : -1.f;
            const float nx = sg * wx / wn, ny = sg * wy / wn;
            const float d0 = kap * ra2 * 0.5f + (ax * nx + ay * ny);
            const float rc = sqrtf(Cc.x * Cc.x + Cc.y * Cc.y);
            const float dz = Cc.z - (az + slope * (rc - ra));
            if (!(fabsf(d0) <= g.d0) || !(fabsf(dz) <= g.dz)) return;
            const float u = d0 / g.d0, v = dz / g.dz;
            const float s2 = u * u + v * v;
            if (s2 > best_s) return;  // the confirmation term only adds
            const int c_id = __float_as_int(Cc.w);
            float c3 = 0.f;
            if (g.confirm) {
                if (rc == rb) return;
                const float slope23 = (Cc.z - B.z) / (rc - rb);
                // where the circle crosses r = R3 nearest to c: centre U = a + w / (2 det); the
                // crossing lies along U at a = (R3^2 + 2 rho d0) / (2 |U|) (|U|^2 - rho^2 = 2 rho d0)
                const float rho = 1.f / kap;
                const float ux = ax + wx / (2.f * det), uy = ay + wy / (2.f * det);
                const float D = sqrtf(ux * ux + uy * uy);
                const float R3 = g.R[3];
                const float along = (R3 * R3 + 2.f * rho * d0) / (2.f * D);
                const float h2 = R3 * R3 - along * along;
                if (!(h2 >= 0.f)) return;
                const float h = sqrtf(h2), ex = ux / D, ey = uy / D;
                const float px1 = along * ex - h * ey, py1 = along * ey + h * ex;
                const float px2 = along * ex + h * ey, py2 = along * ey - h * ex;
                const bool first = (px1 - Cc.x) * (px1 - Cc.x) + (py1 - Cc.y) * (py1 - Cc.y) <=
                                   (px2 - Cc.x) * (px2 - Cc.x) + (py2 - Cc.y) * (py2 - Cc.y);
                const float ph3 = atan2f(first ? py1 : py2, first ? px1 : px2);
                const float zc3 = B.z + slope23 * (R3 - rb);
                int h0b, h1b, r0, nr;
                const float wz = g.z3 + 1e-3f + 1e-5f * fabsf(zc3) + g.hit_dr * fabsf(slope23);
                eta_bins(g, R3, zc3 - wz, zc3 + wz, h0b, h1b);
                phi_bins(g, ph3, (3.f * g.w3 + 0.02f + 2.f * g.hit_dr * kap) / (R3 - g.hit_dr) + 2e-3f, r0, nr);
                c3 = kInf;
                for_window(g, bin_off, seg0 + 3, h0b, h1b, r0, nr, [&](int je) {
                    const float4 E = hxyzi[je];
                    const float d23x = E.x - Cc.x, d23y = E.y - Cc.y;
                    if (!(sqrtf(d23x * d23x + d23y * d23y) <= g.lim23)) return;
                    const float qx = E.x - ax, qy = E.y - ay;
                    const float f3 = kap * (qx * qx + qy * qy) * 0.5f - (qx * nx + qy * ny);
                    const float re = sqrtf(E.x * E.x + E.y * E.y);
                    const float dz3 = E.z - (B.z + slope23 * (re - rb));
                    if (!(fabsf(f3) <= g.w3) || !(fabsf(dz3) <= g.z3)) return;
                    const float p = f3 / g.w3, q = dz3 / g.z3;
                    c3 = fminf(c3, p * p + q * q);
                });
                if (c3 == kInf) return;
            }
            const float s = s2 + c3;
            if (s < best_s || (s == best_s && (b_id < best_b || (b_id == best_b && c_id < best_c)))) {
                best_s = s;
                best_b = b_id;
                best_c = c_id;
            }
        });
    });
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
    if (c.n_layers < 4 || idx->n_layers != c.n_layers)
        return seed_fail(ctx, TKF_ERR_INVALID, "find_seeds: needs an index of at least 4 layers of this context");
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
    k_seed_find<<<blocks, kSeedThreads, 0, s>>>(g, idx->hxyzi, idx->bin_off, idx->ev_off, n, ctx->seed_b,
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
