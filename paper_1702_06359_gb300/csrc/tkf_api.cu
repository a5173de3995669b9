// libtkf.so: context, hit index, seed estimate and track fit kernels, and the C ABI entry
// points declared in include/tkf.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"
#include "kf_math.cuh"

using namespace tkf;

namespace {

// ------------------------------------------------------------------ error helpers

int set_err(tkf_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_err(tkf_ctx *ctx, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return set_err(ctx, e == cudaErrorMemoryAllocation ? TKF_ERR_NOMEM : TKF_ERR_CUDA, m);
}

#define TKF_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call); \
    } while (0)

// ------------------------------------------------------------------ hit index kernels

__device__ __forceinline__ int find_event(const int *off, int n_events, int i)
{  // largest e with off[e] <= i
    int lo = 0, hi = n_events;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&off[mid]) <= i) lo = mid; else hi = mid;
    }
    return lo;
}

struct IndexGeom {
    int L, n_eta, n_phi, n_bins, n_events;
    float radius[TKF_MAX_LAYERS];
    float eta_min, inv_eta_w;
    float phi_scale;     // n_phi / (2 pi), rounded once on the host
    unsigned disk_mask;  // bit l: layer l is an endcap disk (eta = asinh(z / r_hit))
};

IndexGeom index_geom(const tkf_config &c, int n_events)
{
    IndexGeom g{};
    g.L = c.n_layers;
    g.n_eta = c.n_eta_bins;
    g.n_phi = c.n_phi_bins;
    g.n_bins = c.n_eta_bins * c.n_phi_bins;
    g.n_events = n_events;
    for (int l = 0; l < c.n_layers; ++l) {
        g.radius[l] = (float)c.radius[l];
        if (c.disk_z[l] > 0.0) g.disk_mask |= 1u << l;
    }
    g.eta_min = (float)c.eta_min;
    g.inv_eta_w = (float)(1.0 / c.eta_bin_w);
    g.phi_scale = (float)(c.n_phi_bins / (2.0 * kPi));
    return g;
}

// continuous phi-bin coordinate (phi + pi) * n_phi / (2 pi); its floor is the phi bin
__device__ __forceinline__ float phi_coord(const IndexGeom &g, float x, float y)
{
    return (atan2f(y, x) + (float)kPi) * g.phi_scale;
}

// eta of a position at z on a cylinder of radius r: asinh(z / r) = sign * ln(|z/r| + sqrt((z/r)^2 + 1))
// in single precision with the fast logarithm (absolute error ~1e-6 over the eta range, far
// below the 0.1 bin width; the window search allows 1e-4 of slack at bin edges)
__device__ __forceinline__ float eta_of(float z, float r)
{
    const float t = z / r, at = fabsf(t);
    return copysignf(fast_log(at + sqrtf(at * at + 1.f)), t);
}

__device__ __forceinline__ int hit_bin(const IndexGeom &g, int l, float x, float y, float z)
{
    // on a cylinder eta of the layer's radius; on an endcap disk of the hit's own radius
    const float r = (g.disk_mask >> l) & 1u ? sqrtf(x * x + y * y) : g.radius[l];
    int eb = (int)floorf((eta_of(z, r) - g.eta_min) * g.inv_eta_w);
    eb = eb < 0 ? 0 : (eb >= g.n_eta ? g.n_eta - 1 : eb);
    int pb = (int)floorf(phi_coord(g, x, y));
    pb = pb < 0 ? 0 : (pb >= g.n_phi ? g.n_phi - 1 : pb);
    return eb * g.n_phi + pb;
}

// phi sub-bin (0..kSubBins-1) of a hit inside its phi bin pb, from the same phi coordinate
__device__ __forceinline__ int hit_sub(const IndexGeom &g, float x, float y, int pb)
{
    const int s = (int)floorf((phi_coord(g, x, y) - (float)pb) * (float)kSubBins);
    return s < 0 ? 0 : (s >= kSubBins ? kSubBins - 1 : s);
}

// key = ((event * L + layer) * n_bins + bin); counts per key.  The largest variances of each
// (event, layer) are reduced within the warp first (hits of one segment usually arrive
// together), so only one atomic per warp and segment reaches L2.
__global__ void k_hit_count(const IndexGeom g, const tkf_hits h, int *keys, int *counts, int *seg_count, int *var_max,
                            int *err)
{
    // every lane of the warp reaches the warp-wide reductions below (blockDim is a multiple of 32)
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    (void)seg_count;
    // the event of the block's first hit is searched once; a block's hits span few events
    __shared__ int s_e0;
    if (threadIdx.x == 0) s_e0 = find_event(h.event_off, g.n_events, blockIdx.x * blockDim.x);
    __syncthreads();
    const bool in = i < h.n;
    const int l = in ? h.layer[i] : 0;
    const bool ok = in && l >= 0 && l < g.L;
    int ev = s_e0;
    if (ok)
        while (ev + 1 < g.n_events && __ldg(&h.event_off[ev + 1]) <= i) ++ev;
    const int seg = ok ? ev * g.L + l : -1;
    if (ok) {
        const int key = seg * g.n_bins + hit_bin(g, l, h.x[i], h.y[i], h.z[i]);
        keys[i] = key;
        atomicAdd(&counts[key], 1);
    } else if (in) {
        keys[i] = -1;
        atomicOr(err, kErrBadLayer);
    }
    const unsigned same = __match_any_sync(0xffffffffu, seg);
    const int vu = __reduce_max_sync(same, ok ? __float_as_int(fmaxf(h.var_u[i], 0.f)) : 0);
    const int vv = __reduce_max_sync(same, ok ? __float_as_int(fmaxf(h.var_v[i], 0.f)) : 0);
    if (ok && (int)(threadIdx.x & 31) == __ffs(same) - 1) {
        atomicMax(&var_max[2 * seg + 0], vu);
        atomicMax(&var_max[2 * seg + 1], vv);
    }
}

// hits per (event, layer): sum of the segment's bin counts, one block per segment
__global__ void k_seg_total(const int *counts, int *seg_count, int n_bins)
{
    __shared__ int part[32];
    const int *c = counts + (size_t)blockIdx.x * n_bins;
    int s = 0;
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) s += c[b];
    s = __reduce_add_sync(0xffffffffu, s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int t = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0;
        t = __reduce_add_sync(0xffffffffu, t);
        if (threadIdx.x == 0) seg_count[blockIdx.x] = t;
    }
}

// exclusive scan of the (event, layer) hit counts, one block
__global__ void k_seg_scan(const int *seg_count, int *seg_base, int n)
{
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < n ? seg_count[i] : 0;
        int x = v;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int incl = x + (w > 0 ? warp_sums[w - 1] : 0) + carry;
        if (i < n) seg_base[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = incl;
        __syncthreads();
    }
}

// CSR offsets of the bins of one (event, layer) segment per block
__global__ void k_bin_scan(const int *counts, const int *seg_base, int *bin_off, int n_bins, int n_segs)
{
    __shared__ int warp_sums[32];
    __shared__ int carry;
    const int seg = blockIdx.x;
    if (threadIdx.x == 0) carry = seg_base[seg];
    __syncthreads();
    const int *c = counts + (size_t)seg * n_bins;
    int *o = bin_off + (size_t)seg * n_bins;
    for (int base = 0; base < n_bins; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < n_bins ? c[i] : 0;
        int x = v;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += t;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, s, d);
                if (lane >= d) s += t;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int incl = x + (w > 0 ? warp_sums[w - 1] : 0) + carry;
        if (i < n_bins) o[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = incl;
        __syncthreads();
    }
    if (seg == n_segs - 1 && threadIdx.x == 0) bin_off[(size_t)n_segs * n_bins] = carry;
}

// place each hit into its bin (order inside a bin fixed afterwards)
__global__ void k_hit_scatter(const IndexGeom g, const tkf_hits h, const int *keys, int *counts, const int *bin_off,
                              float4 *hxyzi, float2 *hvar, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= h.n) return;
    const int key = keys[i];
    if (key < 0) return;
    const int slot = atomicSub(&counts[key], 1) - 1;
    const int pos = bin_off[key] + slot;
    const int e = key / (g.L * g.n_bins);
    const int local = i - h.event_off[e];
    // event-local ids travel in 23-bit fields (sort keys, branch keys): a larger event is an
    // error (its ids wrap inside the event's own range, so no access leaves it)
    if (local > kMaxHitsPerEvent) atomicOr(err, kErrTooManyHits);
    hxyzi[pos] = make_float4(h.x[i], h.y[i], h.z[i], __int_as_float(local));
    hvar[pos] = make_float2(h.var_u[i], h.var_v[i]);
}

// Where sub-bins 1..15 of a bin start, packed one byte each (bytes 0..14 of bin_sub; byte 15
// zero), from the sort keys (sub-bin << 23 | id) of its hits key[a0..a1); all 0xFF when the
// bin holds more than 255 hits (a window then scans it whole).  The 16 per-sub-bin counts are
// kept as bytes of four words and prefix-summed bytewise by one multiplication per word.
template <class KeyAt>
__device__ __forceinline__ uint4 sub_starts(KeyAt key_at, int a0, int a1)
{
    const int n = a1 - a0;
    if (n <= 0) return make_uint4(0u, 0u, 0u, 0u);
    if (n > 255) return make_uint4(~0u, ~0u, ~0u, ~0u);
    unsigned h0 = 0, h1 = 0, h2 = 0, h3 = 0;
    for (int t = a0; t < a1; ++t) {
        const int sb = (key_at(t) >> 23) & (kSubBins - 1);
        const unsigned inc = 1u << (8 * (sb & 3));
        const int wd = sb >> 2;
        h0 += wd == 0 ? inc : 0u;
        h1 += wd == 1 ? inc : 0u;
        h2 += wd == 2 ? inc : 0u;
        h3 += wd == 3 ? inc : 0u;
    }
    // byte k of p = hits in sub-bins 0..k = start of sub-bin k + 1 (no byte exceeds n <= 255)
    const unsigned p0 = h0 * 0x01010101u;
    const unsigned p1 = (h1 + (p0 >> 24)) * 0x01010101u;
    const unsigned p2 = (h2 + (p1 >> 24)) * 0x01010101u;
    const unsigned p3 = ((h3 + (p2 >> 24)) * 0x01010101u) & 0x00FFFFFFu;
    return make_uint4(p0, p1, p2, p3);
}

constexpr int kSortItems = 4;                    // hits per lane held in registers
constexpr int kSortHits = 32 * kSortItems;       // hits a warp orders at once
constexpr int kSortBinsPerWarp = 64;             // consecutive bins per warp
constexpr int kSortWarps = 8;                    // warps per block

// A bin too large for one warp pass (more than kSortHits hits), ordered in place by one lane
// with an insertion sort in global memory; rare (hundreds of hits in one eta-phi bin).
__device__ void sort_bin_serial(const IndexGeom &g, int b, int i0, int i1, int base, float4 *hxyzi, float2 *hvar,
                                uint4 *bin_sub, int *pos_of_hit)
{
    const int pb = (b % g.n_bins) % g.n_phi;
    for (int i = i0; i < i1; ++i) {
        float4 q = hxyzi[i];
        q.w = __int_as_float((hit_sub(g, q.x, q.y, pb) << 23) | __float_as_int(q.w));
        hxyzi[i] = q;
    }
    for (int i = i0 + 1; i < i1; ++i) {
        const float4 k4 = hxyzi[i];
        const float2 k2 = hvar[i];
        const int key = __float_as_int(k4.w);
        int j = i - 1;
        while (j >= i0 && __float_as_int(hxyzi[j].w) > key) {
            hxyzi[j + 1] = hxyzi[j];
            hvar[j + 1] = hvar[j];
            --j;
        }
        hxyzi[j + 1] = k4;
        hvar[j + 1] = k2;
    }
    bin_sub[b] = sub_starts([&](int t) { return __float_as_int(hxyzi[t].w); }, i0, i1);
    for (int i = i0; i < i1; ++i) {
        float4 q = hxyzi[i];
        const int id = __float_as_int(q.w) & 0x7FFFFF;
        q.w = __int_as_float(id);
        hxyzi[i] = q;
        pos_of_hit[base + id] = i;
    }
}

// Orders bins [b, b_end) by (phi sub-bin, event-local hit id) -- the order a window scan
// relies on to read only the sub-bins it overlaps -- records their sub-bin starts (bin_sub)
// and fills pos_of_hit; one warp.  off(k) is the first hit of bin k (off(b_end): one past the
// last), base(k) the first hit of bin k's event, gbin(k) its index in bin_sub.  Each pass takes
// as many whole bins as hold at most kSortHits hits: it loads their hits into registers
// (coalesced), puts the sort keys in shared memory (key, lbin, off: this warp's arrays), ranks
// every hit among the keys of its bin and writes it back to its ordered slot.  All loads of a
// pass precede its stores (the warp synchronises in between), so ordering in place is safe.
template <class OffAt, class BaseAt, class GbinAt>
__device__ __forceinline__ void sort_bins_warp(const IndexGeom &g, int b, int b_end, OffAt off_at, BaseAt base_at,
                                               GbinAt gbin_at, int *key, unsigned char *lbin, int *off, float4 *hxyzi,
                                               float2 *hvar, uint4 *bin_sub, int *pos_of_hit)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    while (b < b_end) {  // warp-uniform loop
        const int nb = min(32, b_end - b);
        const int s_l = off_at(b + min(lane, nb));
        const int e_l = off_at(b + min(lane + 1, nb));
        const int o0 = __shfl_sync(full, s_l, 0);
        const bool fits = lane < nb && e_l - o0 <= kSortHits;
        const int m = __popc(__ballot_sync(full, fits));  // bins taken in this pass (a prefix)
        if (m == 0) {
            if (lane == 0) sort_bin_serial(g, gbin_at(b), s_l, e_l, base_at(b), hxyzi, hvar, bin_sub, pos_of_hit);
            __syncwarp();
            b += 1;
            continue;
        }
        const int n = __shfl_sync(full, e_l, m - 1) - o0;
        if (lane < m) {
            off[lane] = s_l - o0;
            for (int k = s_l - o0; k < e_l - o0; ++k) lbin[k] = (unsigned char)lane;
        }
        if (lane == 0) off[m] = n;
        __syncwarp();
        float4 q[kSortItems];
        float2 v[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const int k = lane + 32 * j;
            if (k < n) {
                q[j] = hxyzi[o0 + k];
                v[j] = hvar[o0 + k];
                const int pb = (gbin_at(b + lbin[k]) % g.n_bins) % g.n_phi;
                key[k] = (hit_sub(g, q[j].x, q[j].y, pb) << 23) | __float_as_int(q[j].w);
            }
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const int k = lane + 32 * j;
            if (k < n) {
                const int lb = lbin[k];
                const int a0 = off[lb], a1 = off[lb + 1];
                const int mine = key[k];
                int r = 0;
                for (int t = a0; t < a1; ++t) r += key[t] < mine;
                const int d = o0 + a0 + r;
                hxyzi[d] = q[j];  // w holds the event-local id
                hvar[d] = v[j];
                pos_of_hit[base_at(b + lb) + (mine & 0x7FFFFF)] = d;
            }
        }
        if (lane < m) bin_sub[gbin_at(b + lane)] = sub_starts([&](int t) { return key[t]; }, off[lane], off[lane + 1]);
        __syncwarp();  // shared memory is reused by the next pass
        b += m;
    }
}

// Bin order of the whole index in one launch (used when an event's bins do not fit the
// shared memory of the per-event kernel below): each warp takes kSortBinsPerWarp bins.  Held to
// 5 blocks per SM (51 registers): 1.90 ms for the 640-event index against 2.08 ms at its natural
// 64 registers and 4 blocks (6 blocks: 1.97 ms, with more spills), the same index.
#ifndef TKF_SORT_MINBLOCKS
#define TKF_SORT_MINBLOCKS 5
#endif
__global__ void __launch_bounds__(32 * kSortWarps, TKF_SORT_MINBLOCKS)
k_bin_sort(const IndexGeom g, const int *bin_off, const int *ev_off, int n_bins_total, float4 *hxyzi, float2 *hvar,
           uint4 *bin_sub, int *pos_of_hit)
{
    __shared__ int s_key[kSortWarps][kSortHits];
    __shared__ unsigned char s_bin[kSortWarps][kSortHits];
    __shared__ int s_off[kSortWarps][33];
    const int w = threadIdx.x >> 5;
    const long long first = ((long long)blockIdx.x * kSortWarps + w) * kSortBinsPerWarp;
    if (first >= n_bins_total) return;  // warp-uniform
    const int b_end = (int)min(first + kSortBinsPerWarp, (long long)n_bins_total);
    const int per_event = g.L * g.n_bins;
    sort_bins_warp(
        g, (int)first, b_end, [&](int k) { return bin_off[k]; }, [&](int k) { return ev_off[k / per_event]; },
        [](int k) { return k; }, s_key[w], s_bin[w], s_off[w], hxyzi, hvar, bin_sub, pos_of_hit);
}

// Order in which the per-event blocks below take the events: largest first (so that the
// big events of a lognormal mix start early instead of trailing the launch); the rank of
// event e counts the events larger than it, or as large with a smaller index.  Up to
// kOrderMax events (beyond that the input order is kept).
constexpr int kOrderMax = 4096;

__global__ void __launch_bounds__(1024) k_event_order(const int *ev_off, int n_events, int *perm)
{
    __shared__ int s_size[kOrderMax];
    if (n_events > kOrderMax) {
        for (int e = threadIdx.x; e < n_events; e += blockDim.x) perm[e] = e;
        return;
    }
    for (int e = threadIdx.x; e < n_events; e += blockDim.x) s_size[e] = ev_off[e + 1] - ev_off[e];
    __syncthreads();
    for (int e = threadIdx.x; e < n_events; e += blockDim.x) {
        const int se = s_size[e];
        int rank = 0;
        for (int f = 0; f < n_events; ++f) {
            const int sf = s_size[f];
            rank += sf > se || (sf == se && f < e);
        }
        perm[rank] = e;
    }
}

// Folds a thread's running variance maxima of layer l (float bits of non-negative values, so
// integer order is value order) into the block's maxima; l < 0: nothing held.
__device__ __forceinline__ void var_flush(int *s_var, int l, int mu, int mv)
{
    if (l < 0) return;
    atomicMax(&s_var[2 * l], mu);
    atomicMax(&s_var[2 * l + 1], mv);
}

// The bins of one event in one block (one block per event, events taken in the order perm),
// with the event's bin counters in shared memory: (1) count the hits per (layer, eta bin, phi
// bin) and reduce the largest variances per layer; (2) exclusive scan of the counts ->
// bin_off (the event's hits keep their place [event_off[e], event_off[e+1]) in the index);
// (3) place every hit into its bin (a shared-memory cursor per bin).  k_bin_sort then orders
// the bins.  The same bins and offsets as the multi-launch path.
// The per-event kernels take a batch of at least TKF_INDEX_EVENTS_PER_SM events per SM; smaller
// batches are spread over every SM by the multi-launch kernels.  Measured on the batched workload
// (same indices): multi-launch 0.75 / 0.86 ms at 160 / 200 events against 0.91 / 0.98 ms per event,
// per event 1.18 / 1.45 / 1.90 ms at 320 / 480 / 640 events against 1.23 / 1.85 / 2.62 ms.
#ifndef TKF_INDEX_EVENTS_PER_SM
#define TKF_INDEX_EVENTS_PER_SM 2
#endif
constexpr int kEventThreads = 1024;  // 512-thread blocks, two per SM: 2.46 ms against 1.88 ms (640 events)
constexpr int kEventWarps = kEventThreads / 32;
constexpr int kEventUnroll = 4;

__global__ void __launch_bounds__(kEventThreads)
k_index_event(const IndexGeom g, const tkf_hits h, const int *perm, int n_bins_total, float4 *hxyzi, float2 *hvar,
              int *bin_off, float2 *var_max, int *err)
{
    extern __shared__ int s_cnt[];  // [L * n_bins]: counts, then bin offsets / cursors
    __shared__ int s_var[2 * TKF_MAX_LAYERS];
    __shared__ int s_part[kEventWarps];
    const unsigned full = 0xffffffffu;
    const int e = perm[blockIdx.x], tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int cur_l = -1, mu = 0, mv = 0;  // this thread's layer and its largest variances (float bits)
    const int nb_ev = g.L * g.n_bins;
    const int h0 = h.event_off[e], h1 = h.event_off[e + 1];
    if (tid == 0 && h1 - h0 > kMaxHitsPerEvent) atomicOr(err, kErrTooManyHits);  // 23-bit local ids
    for (int k = tid; k < nb_ev; k += kEventThreads) s_cnt[k] = 0;
    if (tid < 2 * g.L) s_var[tid] = 0;
    __syncthreads();
    // (1) counts and variance maxima; kEventUnroll hits per thread and pass, loaded together
    for (int i0 = h0; i0 < h1; i0 += kEventThreads * kEventUnroll) {
        int l[kEventUnroll];
        float x[kEventUnroll], y[kEventUnroll], z[kEventUnroll], vu[kEventUnroll], vv[kEventUnroll];
#pragma unroll
        for (int u = 0; u < kEventUnroll; ++u) {
            const int i = i0 + tid + u * kEventThreads;
            const int j = i < h1 ? i : h0;  // a valid index (the event is not empty here)
            l[u] = h.layer[j];
            x[u] = h.x[j];
            y[u] = h.y[j];
            z[u] = h.z[j];
            vu[u] = h.var_u[j];
            vv[u] = h.var_v[j];
        }
#pragma unroll
        for (int u = 0; u < kEventUnroll; ++u) {
            const bool in = i0 + tid + u * kEventThreads < h1;
            const bool ok = in && l[u] >= 0 && l[u] < g.L;
            if (ok) {
                atomicAdd(&s_cnt[l[u] * g.n_bins + hit_bin(g, l[u], x[u], y[u], z[u])], 1);
                if (l[u] != cur_l) {  // hits usually come grouped by layer: rare
                    var_flush(s_var, cur_l, mu, mv);
                    cur_l = l[u];
                    mu = mv = 0;
                }
                mu = max(mu, __float_as_int(fmaxf(vu[u], 0.f)));
                mv = max(mv, __float_as_int(fmaxf(vv[u], 0.f)));
            } else if (in) {
                atomicOr(err, kErrBadLayer);
            }
        }
    }
    {  // the last running maxima, one atomic per layer and warp
        const unsigned grp = __match_any_sync(full, cur_l);
        const int ru = __reduce_max_sync(grp, (unsigned)mu), rv = __reduce_max_sync(grp, (unsigned)mv);
        if (lane == __ffs(grp) - 1) var_flush(s_var, cur_l, ru, rv);
    }
    __syncthreads();
    // (2) exclusive scan: thread t owns the contiguous chunk [t * per, (t + 1) * per)
    const int per = (nb_ev + kEventThreads - 1) / kEventThreads;
    const int c0 = min(tid * per, nb_ev), c1 = min(c0 + per, nb_ev);
    int sum = 0;
    for (int k = c0; k < c1; ++k) sum += s_cnt[k];
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_part[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = lane < kEventWarps ? s_part[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(full, x, o);
            if (lane >= o) x += t;
        }
        if (lane < kEventWarps) s_part[lane] = x;  // inclusive warp totals
    }
    __syncthreads();
    int run = incl - sum + (w > 0 ? s_part[w - 1] : 0);
    const size_t gb0 = (size_t)e * nb_ev;
    for (int k = c0; k < c1; ++k) {
        const int c = s_cnt[k];
        s_cnt[k] = run;
        bin_off[gb0 + k] = h0 + run;
        run += c;
    }
    if (e == g.n_events - 1 && tid == kEventThreads - 1) bin_off[n_bins_total] = h0 + run;
    if (tid < g.L)
        var_max[(size_t)e * g.L + tid] = make_float2(__int_as_float(s_var[2 * tid]), __int_as_float(s_var[2 * tid + 1]));
    __syncthreads();
    // (3) place the hits, kEventUnroll per thread and pass
    for (int i0 = h0; i0 < h1; i0 += kEventThreads * kEventUnroll) {
        int l[kEventUnroll];
        float x[kEventUnroll], y[kEventUnroll], z[kEventUnroll], vu[kEventUnroll], vv[kEventUnroll];
#pragma unroll
        for (int u = 0; u < kEventUnroll; ++u) {
            const int i = i0 + tid + u * kEventThreads;
            const int j = i < h1 ? i : h0;
            l[u] = h.layer[j];
            x[u] = h.x[j];
            y[u] = h.y[j];
            z[u] = h.z[j];
            vu[u] = h.var_u[j];
            vv[u] = h.var_v[j];
        }
#pragma unroll
        for (int u = 0; u < kEventUnroll; ++u) {
            const int i = i0 + tid + u * kEventThreads;
            if (i >= h1 || l[u] < 0 || l[u] >= g.L) continue;
            const int pos = h0 + atomicAdd(&s_cnt[l[u] * g.n_bins + hit_bin(g, l[u], x[u], y[u], z[u])], 1);
            hxyzi[pos] = make_float4(x[u], y[u], z[u], __int_as_float(i - h0));
            hvar[pos] = make_float2(vu[u], vv[u]);
        }
    }
}

// Dynamic shared memory of k_index_event (the event's bin counters) allowed next to its
// static arrays within one block's 227 KB; an index whose event bins need more takes the
// multi-launch path.
constexpr size_t kEventStaticSmem = (size_t)kEventWarps * 4 + 2 * TKF_MAX_LAYERS * 4;
constexpr size_t kEventMaxDynSmem = 227 * 1024 - kEventStaticSmem - 1024;

size_t index_event_smem(int n_layers, int n_bins)
{
    const size_t bytes = (size_t)n_layers * n_bins * sizeof(int);
    return bytes <= kEventMaxDynSmem ? bytes : 0;
}

// Allows k_index_event its dynamic shared memory on the current device.
cudaError_t index_event_prepare()
{
    return cudaFuncSetAttribute(k_index_event, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEventMaxDynSmem);
}

unsigned sort_blocks(size_t n_bins)
{
    const size_t per_block = (size_t)kSortWarps * kSortBinsPerWarp;
    return (unsigned)std::max<size_t>(1, (n_bins + per_block - 1) / per_block);
}

// ------------------------------------------------------------------ seed ordering for locality

// key of each seed = (event, eta bin, phi bin) of its position on layer `layer`
template <class R>
__global__ void k_seed_key(const IndexGeom g, int layer, const R *par, int stride, const int *event, int n,
                           int *keys, int *counts)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int ev = event ? event[i] : 0;
    ev = ev < 0 ? 0 : (ev >= g.n_events ? g.n_events - 1 : ev);  // bad ids are reported by the build
    const float x = (float)par[i], y = (float)par[stride + i], z = (float)par[2 * stride + i];
    const int key = ev * g.n_bins + hit_bin(g, layer, x, y, z);
    keys[i] = key;
    atomicAdd(&counts[key], 1);
}

__global__ void k_seed_place(const int *keys, int *counts, const int *off, int n, int *perm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int key = keys[i];
    perm[off[key] + atomicSub(&counts[key], 1) - 1] = i;
}

// ------------------------------------------------------------------ seed estimate and fit

template <class R> __device__ __forceinline__ R gpick(float f, double d);
template <> __device__ __forceinline__ float gpick<float>(float f, double) { return f; }
template <> __device__ __forceinline__ double gpick<double>(float, double d) { return d; }

struct FitGeom {
    int L;
    int two_step;  // hits lie off the layers' cylinders (hit_dr > 0): states go to each hit's radius
    double radius[TKF_MAX_LAYERS], xx0[TKF_MAX_LAYERS], disk_z[TKF_MAX_LAYERS];
    float radius_f[TKF_MAX_LAYERS], xx0_f[TKF_MAX_LAYERS], disk_z_f[TKF_MAX_LAYERS];
    unsigned disk_mask;  // bit l: layer l is a pair of endcap disks at z = +-disk_z[l]
    double kb, mass, prior[6];
    float kb_f, mass_f;
};

// The state's move to layer l (kDisk: the kernel serves configurations with endcap disks):
// the layer's cylinder (at target_radius), or the disk on the side of the state's z.
template <class R, bool kDisk, int kMode = kPropOut>
__device__ __forceinline__ bool to_layer(const FitGeom &g, int l, R p[6], R P[21], R radius, R kb)
{
    if (kDisk && ((g.disk_mask >> l) & 1u)) {
        const R zd = gpick<R>(g.disk_z_f[l], g.disk_z[l]);
        return propagate_plane<R>(p, P, p[2] >= R(0) ? zd : -zd, kb);
    }
    return propagate<R, kMode>(p, P, radius, kb);
}

// The Kalman update with the layer's measurement model (r-phi and z on a cylinder, r-phi and r
// on a disk).
template <class U, class R, bool kDisk>
__device__ __forceinline__ bool update_at(const FitGeom &g, int l, R p[6], R P[21], R x, R y, R z, R vu, R vv, U *c2)
{
    if (kDisk && ((g.disk_mask >> l) & 1u)) return kalman_update<U, R, true>(p, P, x, y, z, vu, vv, c2);
    return kalman_update<U, R, false>(p, P, x, y, z, vu, vv, c2);
}


// asin(x)/x, accurate near 0
template <class R> __device__ __forceinline__ R asin_over(R x)
{
    if (ab(x) < R(1e-2)) {
        const R x2 = x * x;
        return R(1) + x2 * (R(1.0 / 6) + x2 * R(3.0 / 40));
    }
    return asn(x) / x;
}

// Initial state from three hits: signed curvature 2 (P2-P1)x(P3-P2) / (|P2-P1||P3-P2||P3-P1|)
// (positive for a counter-clockwise turn), tangent at P1 = chord direction P1->P2 turned back by
// half the subtended angle, transverse arc P1->P3 = chord * asin(k c/2)/(k c/2).
template <class R>
__device__ __forceinline__ void seed_estimate(const FitGeom &g, const tkf_hits &h, int h1, int h2, int h3, R p[6],
                                              R P[21])
{
    const R x1 = h.x[h1], y1 = h.y[h1], z1 = h.z[h1];
    const R x2 = h.x[h2], y2 = h.y[h2];
    const R x3 = h.x[h3], y3 = h.y[h3], z3 = h.z[h3];
    const R ax = x2 - x1, ay = y2 - y1, bx = x3 - x2, by = y3 - y2, cx = x3 - x1, cy = y3 - y1;
    const R d12 = sq(ax * ax + ay * ay), d23 = sq(bx * bx + by * by), d13 = sq(cx * cx + cy * cy);
    const R kappa = R(2) * (ax * by - ay * bx) / (d12 * d23 * d13);
    R h12 = kappa * d12 * R(0.5), h13 = kappa * d13 * R(0.5);
    h12 = h12 > R(1) ? R(1) : (h12 < R(-1) ? R(-1) : h12);
    h13 = h13 > R(1) ? R(1) : (h13 < R(-1) ? R(-1) : h13);
    const R phi = at2(ay, ax) - asn(h12);
    const R s13 = d13 * asin_over(h13);
    const R cot = (z3 - z1) / s13;
    const R kb = gpick<R>(g.kb_f, g.kb);
    p[0] = x1;
    p[1] = y1;
    p[2] = z1;
    p[3] = -kappa / kb;
    p[4] = wrap_phi(phi);
    p[5] = at2(R(1), cot);
#pragma unroll
    for (int k = 0; k < 21; ++k) P[k] = R(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) P[sym(k, k)] = R(g.prior[k] * g.prior[k]);
    if (g.disk_mask & 1u) P[sym(2, 2)] = R(0);  // on an endcap disk z is the disk's, known exactly
}

template <class R>
__global__ void k_seed(const FitGeom g, const tkf_hits h, const int *seed_hits, tkf_tracks out, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= out.n) return;
    const int h1 = seed_hits[i], h2 = seed_hits[out.stride + i], h3 = seed_hits[2 * out.stride + i];
    if (h1 < 0 || h2 < 0 || h3 < 0 || h1 >= h.n || h2 >= h.n || h3 >= h.n) {
        atomicOr(err, kErrBadHitId);
        out.nhits[i] = TKF_TRACK_SINGULAR;
        return;
    }
    R p[6], P[21];
    seed_estimate<R>(g, h, h1, h2, h3, p, P);
    R *par = (R *)out.par, *cov = (R *)out.cov;
    const size_t st = out.stride;
#pragma unroll
    for (int k = 0; k < 6; ++k) par[k * st + i] = p[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) cov[k * st + i] = P[k];
    ((R *)out.chi2)[i] = R(0);
    out.nhits[i] = 0;
    if (out.hit_idx) {
        for (int l = 0; l < g.L; ++l) out.hit_idx[l * st + i] = l < 3 ? seed_hits[l * st + i] : -1;
    }
}

// Resident blocks of 128 threads per SM requested from the register allocator for the all-float
// fit kernels (k_fit, k_seed_fit, k_fit_backward): 7 holds them to 72 registers, their count
// before the reads were pipelined (80 otherwise, 6 blocks); measured on the 2.6 M-track fit,
// 72 registers is 4 % faster (0.575 against 0.599 ms), the backward pass 3 % (0.760 / 0.786 ms).
#ifndef TKF_FIT_MINBLOCKS_F32
#define TKF_FIT_MINBLOCKS_F32 7
#endif
constexpr int kFitThreads = 128;
template <class R, class U> struct FitMinBlocks {
    static constexpr int value = (sizeof(R) == 4 && sizeof(U) == 4) ? TKF_FIT_MINBLOCKS_F32 : 1;
};

// A hit's position and variances read from the hit planes (zeros for an id outside 0..n-1).
template <class R> struct HitRec {
    R x, y, z, vu, vv;
};
template <class R> __device__ __forceinline__ HitRec<R> load_hit(const tkf_hits &h, int hid)
{
    HitRec<R> r{R(0), R(0), R(0), R(0), R(0)};
    if (hid >= 0 && hid < h.n) {
        r.x = R(__ldg(&h.x[hid]));
        r.y = R(__ldg(&h.y[hid]));
        r.z = R(__ldg(&h.z[hid]));
        r.vu = R(__ldg(&h.var_u[hid]));
        r.vv = R(__ldg(&h.var_v[hid]));
    }
    return r;
}

// The cylinder a layer's state is taken to: the hit's own radius (c, read by load_hit) when hits
// lie off the layers' cylinders (the two-step geometry of Sec. 2.2) and the layer has a valid
// hit, else the layer's radius.
template <class R>
__device__ __forceinline__ R target_radius(const FitGeom &g, const tkf_hits &h, int l, int hid, const HitRec<R> &c)
{
    return (g.two_step && hid >= 0 && hid < h.n) ? sq(c.x * c.x + c.y * c.y) : gpick<R>(g.radius_f[l], g.radius[l]);
}

// The Kalman fit over layers first..last of a state in registers: propagate (on the first
// layer only when prop_first: the state then lies on the layer before), update with the
// layer's hit (hit_at(l), -1 = none) and add the layer's scattering (all but the outermost
// layer of the detector).  status: 0, or the track status that stopped the fit.
// The reads are software-pipelined: while a layer is processed, the next layer's hit and the
// id of the one after are already on their way, so the loads' latency hides behind a layer's
// arithmetic instead of stalling each step.
template <class R, class U, bool kDisk, class HitAt>
__device__ __forceinline__ void fit_layers(const FitGeom &g, const tkf_hits &h, HitAt hit_at, int first, int last,
                                           bool prop_first, R p[6], R P[21], R &chi2, int &nh, int &status, int *err)
{
    const R kb = gpick<R>(g.kb_f, g.kb), mass = gpick<R>(g.mass_f, g.mass);
    int hid = first <= last ? hit_at(first) : -1;
    int hid1 = first + 1 <= last ? hit_at(first + 1) : -1;
    HitRec<R> cur = load_hit<R>(h, hid);
    for (int l = first; l <= last && status == 0; ++l) {
        const HitRec<R> nxt = load_hit<R>(h, hid1);
        const int hid2 = l + 2 <= last ? hit_at(l + 2) : -1;
        if ((l > first || prop_first) && !to_layer<R, kDisk>(g, l, p, P, target_radius<R>(g, h, l, hid, cur), kb)) {
            status = TKF_TRACK_NOREACH;
            break;
        }
        if (hid >= h.n) {
            atomicOr(err, kErrBadHitId);
            status = TKF_TRACK_SINGULAR;
            break;
        }
        if (hid >= 0) {
            U dc2;
            if (!update_at<U, R, kDisk>(g, l, p, P, cur.x, cur.y, cur.z, cur.vu, cur.vv, &dc2)) {
                status = TKF_TRACK_SINGULAR;
                break;
            }
            chi2 += R(dc2);
            nh += 1;
        }
        if (l < g.L - 1)
            scatter<R>(p, P, gpick<R>(g.xx0_f[l], g.xx0[l]), mass, kDisk && ((g.disk_mask >> l) & 1u));
        cur = nxt;
        hid = hid1;
        hid1 = hid2;
    }
}

template <class R> __device__ __forceinline__ void store_fit(const tkf_tracks &out, int i, const R p[6], const R P[21],
                                                             R chi2, int nhits)
{
    R *op = (R *)out.par, *oc = (R *)out.cov;
    const size_t so = out.stride;
#pragma unroll
    for (int k = 0; k < 6; ++k) op[k * so + i] = p[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) oc[k * so + i] = P[k];
    ((R *)out.chi2)[i] = chi2;
    out.nhits[i] = nhits;
}

// prop_first = 0: the input state lies on layer `first` (its first step is the update there);
// 1: it lies on the layer before (the fit continues a fit of the earlier layers).
template <class R, class U, bool kDisk>
__global__ void __launch_bounds__(kFitThreads, (FitMinBlocks<R, U>::value)) k_fit(const FitGeom g, const tkf_hits h, const tkf_tracks in, const int *hit_idx, int first, int last,
                      int prop_first, tkf_tracks out, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= in.n) return;
    const size_t si = in.stride, so = out.stride;
    R p[6], P[21];
    const R *ip = (const R *)in.par, *ic = (const R *)in.cov;
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = ip[k * si + i];
#pragma unroll
    for (int k = 0; k < 21; ++k) P[k] = ic[k * si + i];
    R chi2 = ((const R *)in.chi2)[i];
    int nh = in.nhits[i];
    int status = nh < 0 ? nh : 0;
    fit_layers<R, U, kDisk>(
        g, h, [&](int l) { return hit_idx[l * si + i]; }, first, last, prop_first != 0, p, P, chi2, nh, status, err);
    store_fit<R>(out, i, p, P, chi2, status ? status : nh);
    if (out.hit_idx && out.hit_idx != hit_idx)
        for (int l = 0; l < g.L; ++l) out.hit_idx[l * so + i] = hit_idx[l * si + i];
}

// Seed estimate and its fit over layers 0..last in one pass (the first two steps of the
// batched pipeline): the same values as k_seed followed by k_fit, without storing the estimate.
template <class R, class U, bool kDisk>
__global__ void __launch_bounds__(kFitThreads, (FitMinBlocks<R, U>::value)) k_seed_fit(const FitGeom g, const tkf_hits h, const int *seed_hits, int last, tkf_tracks out, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= out.n) return;
    const size_t st = out.stride;
    const int h1 = seed_hits[i], h2 = seed_hits[st + i], h3 = seed_hits[2 * st + i];
    R p[6], P[21], chi2 = R(0);
    int nh = 0, status = 0;
    if (h1 < 0 || h2 < 0 || h3 < 0 || h1 >= h.n || h2 >= h.n || h3 >= h.n) {
        atomicOr(err, kErrBadHitId);
        status = TKF_TRACK_SINGULAR;
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] = R(0);
#pragma unroll
        for (int k = 0; k < 21; ++k) P[k] = R(0);
    } else {
        seed_estimate<R>(g, h, h1, h2, h3, p, P);
        fit_layers<R, U, kDisk>(
            g, h, [&](int l) { return l < 3 ? seed_hits[l * st + i] : -1; }, 0, last, false, p, P, chi2, nh, status,
            err);
    }
    store_fit<R>(out, i, p, P, chi2, status ? status : nh);
    if (out.hit_idx)
        for (int l = 0; l < g.L; ++l) out.hit_idx[l * st + i] = l < 3 ? seed_hits[l * st + i] : -1;
}

// The reversed description of a track: (x, y, z, q/pT, phi, theta) -> (x, y, z, -q/pT, phi + pi,
// pi - theta) is the same helix run backwards (transverse path s -> -s), so outward
// propagation of the reversed state reaches the previous (inner) crossing.  The map is its own
// inverse with Jacobian diag(1, 1, 1, -1, 1, -1): covariance elements pairing one of q/pT,
// theta with one of x, y, z, phi change sign.  `scale` multiplies the covariance.
template <class R> __device__ __forceinline__ void reverse_track(R p[6], R P[21], R scale)
{
    p[3] = -p[3];
    p[4] = p[4] > R(0) ? p[4] - R(kPi) : p[4] + R(kPi);
    p[5] = R(kPi) - p[5];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            const bool odd = ((i == 3 || i == 5) != (j == 3 || j == 5));
            P[sym(i, j)] = (odd ? -scale : scale) * P[sym(i, j)];
        }
}

// Backward (inward) pass over a fitted track's hits, layers last..first: the state on layer
// `last` with its covariance times `scale`, then per layer from `last` inward the update with
// the layer's hit, the layer's material, the propagation to the next smaller cylinder (as the
// outward propagation of the reversed track).  The result lies on layer `first` after its
// update and material; chi2 and nhits are the pass's own.
template <class R, class U, bool kDisk>
__global__ void __launch_bounds__(kFitThreads, (FitMinBlocks<R, U>::value)) k_fit_backward(const FitGeom g, const tkf_hits h, const tkf_tracks in, const int *hit_idx, int last,
                               int first, R scale, tkf_tracks out, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= in.n) return;
    const size_t si = in.stride, so = out.stride;
    R p[6], P[21];
    const R *ip = (const R *)in.par, *ic = (const R *)in.cov;
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = ip[k * si + i];
#pragma unroll
    for (int k = 0; k < 21; ++k) P[k] = ic[k * si + i];
    const int nh_in = in.nhits[i];
    int status = nh_in < 0 ? nh_in : 0, nh = 0;
    R chi2 = R(0);
    const R kb = gpick<R>(g.kb_f, g.kb), mass = gpick<R>(g.mass_f, g.mass);
    reverse_track<R>(p, P, scale);
    // reads pipelined as in fit_layers: the next (inner) layer's hit is loaded during this one
    int hid = last >= first ? hit_idx[last * si + i] : -1;
    int hid1 = last - 1 >= first ? hit_idx[(last - 1) * si + i] : -1;
    HitRec<R> cur = load_hit<R>(h, hid);
    for (int l = last; l >= first && status == 0; --l) {
        const HitRec<R> nxt = load_hit<R>(h, hid1);
        const int hid2 = l - 2 >= first ? hit_idx[(l - 2) * si + i] : -1;
        if (l < last && !to_layer<R, kDisk, kPropIn>(g, l, p, P, target_radius<R>(g, h, l, hid, cur), kb)) {
            status = TKF_TRACK_NOREACH;
            break;
        }
        if (hid >= h.n) {
            atomicOr(err, kErrBadHitId);
            status = TKF_TRACK_SINGULAR;
            break;
        }
        if (hid >= 0) {
            U dc2;
            if (!update_at<U, R, kDisk>(g, l, p, P, cur.x, cur.y, cur.z, cur.vu, cur.vv, &dc2)) {
                status = TKF_TRACK_SINGULAR;
                break;
            }
            chi2 += R(dc2);
            nh += 1;
        }
        scatter<R>(p, P, gpick<R>(g.xx0_f[l], g.xx0[l]), mass, kDisk && ((g.disk_mask >> l) & 1u));
        cur = nxt;
        hid = hid1;
        hid1 = hid2;
    }
    reverse_track<R>(p, P, R(1));
    store_fit<R>(out, i, p, P, chi2, status ? status : nh);
    if (out.hit_idx && out.hit_idx != hit_idx)
        for (int l = 0; l < g.L; ++l) out.hit_idx[l * so + i] = hit_idx[l * si + i];
}

FitGeom fit_geom(const tkf_ctx *ctx)
{
    FitGeom g{};
    const tkf_config &c = ctx->cfg;
    g.L = c.n_layers;
    g.two_step = c.hit_dr > 0.0;
    for (int l = 0; l < c.n_layers; ++l) {
        g.radius[l] = c.radius[l];
        g.xx0[l] = c.x_over_x0[l];
        g.radius_f[l] = (float)c.radius[l];
        g.xx0_f[l] = (float)c.x_over_x0[l];
        g.disk_z[l] = c.disk_z[l];
        g.disk_z_f[l] = (float)c.disk_z[l];
        if (c.disk_z[l] > 0.0) g.disk_mask |= 1u << l;
    }
    g.kb = kCurv * c.bz;
    g.kb_f = (float)g.kb;
    g.mass = c.mass;
    g.mass_f = (float)c.mass;
    for (int k = 0; k < 6; ++k) g.prior[k] = c.prior_sigma[k];
    return g;
}

int check_tracks(tkf_ctx *ctx, const tkf_tracks *t, bool need_hits, const char *name)
{
    if (!t) return set_err(ctx, TKF_ERR_INVALID, std::string(name) + " is null");
    if (t->n < 0 || t->stride < t->n) return set_err(ctx, TKF_ERR_INVALID, std::string(name) + ": need 0 <= n <= stride");
    if (t->n > 0 && (!t->par || !t->cov || !t->chi2 || !t->nhits))
        return set_err(ctx, TKF_ERR_INVALID, std::string(name) + ": par, cov, chi2 and nhits are required");
    if (need_hits && t->n > 0 && !t->hit_idx) return set_err(ctx, TKF_ERR_INVALID, std::string(name) + ": hit_idx is required");
    return TKF_OK;
}

int check_hits(tkf_ctx *ctx, const tkf_hits *h)
{
    if (!h) return set_err(ctx, TKF_ERR_INVALID, "hits is null");
    if (h->n < 0 || h->n_events < 1) return set_err(ctx, TKF_ERR_INVALID, "hits: need n >= 0 and n_events >= 1");
    if (!h->event_off) return set_err(ctx, TKF_ERR_INVALID, "hits: event_off is required");
    if (h->n > 0 && (!h->x || !h->y || !h->z || !h->var_u || !h->var_v || !h->layer))
        return set_err(ctx, TKF_ERR_INVALID, "hits: x, y, z, var_u, var_v and layer are required");
    return TKF_OK;
}

template <class T> int grow(tkf_ctx *ctx, T **p, size_t n)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_err(ctx, e, "cudaMalloc (hit index)");
    }
    return TKF_OK;
}

}  // namespace

namespace tkf {

int hit_index_reserve(tkf_ctx *ctx, tkf_hit_index **out, size_t max_hits, size_t max_events)
{
    const tkf_config &c = ctx->cfg;
    const size_t n_segs = max_events * (size_t)c.n_layers;
    const size_t n_bins = n_segs * (size_t)c.n_eta_bins * c.n_phi_bins;
    if (n_bins >= (size_t)1 << 31) return set_err(ctx, TKF_ERR_INVALID, "hit index: too many events for the bin table");
    tkf_hit_index *idx = *out;
    if (!idx) {
        idx = new (std::nothrow) tkf_hit_index();
        if (!idx) return set_err(ctx, TKF_ERR_NOMEM, "hit index: host allocation failed");
        idx->ctx = ctx;
        *out = idx;
    }
    int st = TKF_OK;
    if (max_hits > idx->cap_hits || !idx->hxyzi) {
        const size_t cap = std::max<size_t>(max_hits, 1);
        if ((st = grow(ctx, &idx->hxyzi, cap)) || (st = grow(ctx, &idx->hvar, cap)) ||
            (st = grow(ctx, &idx->pos_of_hit, cap)) || (st = grow(ctx, &idx->keys, cap)))
            return st;
        idx->cap_hits = cap;
    }
    if (n_bins > idx->cap_bins || !idx->bin_off) {
        if ((st = grow(ctx, &idx->bin_off, n_bins + 1)) || (st = grow(ctx, &idx->counts, n_bins)) ||
            (st = grow(ctx, &idx->bin_sub, n_bins)))
            return st;
        idx->cap_bins = n_bins;
    }
    if (n_segs > idx->cap_segs || !idx->seg_count) {
        if ((st = grow(ctx, &idx->seg_count, n_segs)) || (st = grow(ctx, &idx->seg_base, n_segs)) ||
            (st = grow(ctx, &idx->var_max, n_segs)) || (st = grow(ctx, &idx->ev_off, n_segs + 1)))
            return st;
        idx->cap_segs = n_segs;
    }
    return TKF_OK;
}

int seed_order_reserve(tkf_ctx *ctx, size_t max_seeds, size_t max_events)
{
    const size_t nb = max_events * (size_t)ctx->cfg.n_eta_bins * ctx->cfg.n_phi_bins;
    int st = TKF_OK;
    if (max_seeds > ctx->ord_cap_seeds || !ctx->ord_key) {
        if ((st = grow(ctx, &ctx->ord_key, max_seeds)) || (st = grow(ctx, &ctx->ord_perm, max_seeds))) return st;
        ctx->ord_cap_seeds = max_seeds;
    }
    if (nb > ctx->ord_cap_bins || !ctx->ord_counts) {
        if ((st = grow(ctx, &ctx->ord_counts, nb)) || (st = grow(ctx, &ctx->ord_off, nb + 1))) return st;
        if (cudaMemset(ctx->ord_counts, 0, nb * sizeof(int)) != cudaSuccess)
            return set_err(ctx, TKF_ERR_CUDA, "cudaMemset (seed order)");
        ctx->ord_cap_bins = nb;
    }
    if (max_events > ctx->ord_cap_events || !ctx->ord_seg_count) {
        if ((st = grow(ctx, &ctx->ord_seg_count, max_events)) || (st = grow(ctx, &ctx->ord_seg_base, max_events)))
            return st;
        ctx->ord_cap_events = max_events;
    }
    return TKF_OK;
}

#ifndef TKF_BUILD_FIRST_PASS
#define TKF_BUILD_FIRST_PASS 1
#endif
int first_list_reserve(tkf_ctx *ctx, size_t max_seeds)
{
    const size_t n = max_seeds * (size_t)build_nmax(ctx->cfg.n_cand);
    if (n <= ctx->first_cap && ctx->first_key) return TKF_OK;
    int st = grow(ctx, &ctx->first_key, n);
    if (!st) st = grow(ctx, &ctx->first_hit, n);
    ctx->first_cap = st ? 0 : n;
    return st;
}

}  // namespace tkf

// ====================================================================== C ABI

extern "C" {

void tkf_default_config(tkf_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->n_layers = 10;
    for (int l = 0; l < 10; ++l) {
        cfg->radius[l] = 4.0 * (l + 1);
        cfg->x_over_x0[l] = 0.03;
    }
    cfg->bz = 3.8;
    cfg->mass = 0.13957;
    const double prior[6] = {0.1, 0.1, 1.0, 0.5, 0.05, 0.05};
    for (int k = 0; k < 6; ++k) cfg->prior_sigma[k] = prior[k];
    cfg->eta_min = -2.0;
    cfg->eta_bin_w = 0.1;
    cfg->n_eta_bins = 40;
    cfg->n_phi_bins = 63;
    cfg->chi2_cut = 30.0;
    cfg->window_margin = 1e-3;
    cfg->n_cand = 6;
    cfg->first_build_layer = 3;
    cfg->precision = TKF_FP32;
    cfg->seeds_per_block = 0;
    cfg->seed_order = 0;
}

const char *tkf_status_string(int status)
{
    switch (status) {
    case TKF_OK: return "ok";
    case TKF_ERR_INVALID: return "invalid argument";
    case TKF_ERR_CUDA: return "CUDA error";
    case TKF_ERR_NOMEM: return "out of device memory";
    case TKF_ERR_AGAIN: return "busy, try again";
    case TKF_ERR_TIMEOUT: return "timed out";
    case TKF_ERR_NOTREADY: return "not ready";
    case TKF_ERR_KERNEL: return "kernel reported an error";
    case TKF_ERR_TOO_LARGE: return "input exceeds the fixed capacity of the allocation-free entry point";
    default: return "unknown status";
    }
}

int tkf_create(const tkf_config *cfg, tkf_ctx **out)
{
    if (!cfg || !out) return TKF_ERR_INVALID;
    *out = nullptr;
    const tkf_config &c = *cfg;
    if (c.n_layers < 4 || c.n_layers > TKF_MAX_LAYERS || c.n_cand < 1 || c.n_cand > TKF_MAX_CAND ||
        c.first_build_layer < 3 || c.first_build_layer > c.n_layers || c.n_eta_bins < 1 || c.n_phi_bins < 1 ||
        c.n_eta_bins * c.n_phi_bins > 1 << 20 || !(c.eta_bin_w > 0) || !(c.chi2_cut > 0) || !(c.bz != 0) ||
        c.precision < TKF_FP32 || c.precision > TKF_FP64 || c.seeds_per_block < 0 || c.window_margin < 0 ||
        !(c.hit_dr >= 0.0) || !(c.hit_dr < c.radius[0]))
        return TKF_ERR_INVALID;
    bool any_disk = false;
    for (int l = 0; l < c.n_layers; ++l) {
        if (!(c.disk_z[l] >= 0.0) || !(c.disk_z[l] < 1e6)) return TKF_ERR_INVALID;
        any_disk |= c.disk_z[l] > 0.0;
    }
    if (any_disk && c.hit_dr > 0.0) return TKF_ERR_INVALID;
    for (int l = 0; l < c.n_layers; ++l) {
        if (!(c.radius[l] > 0) || c.x_over_x0[l] < 0) return TKF_ERR_INVALID;
        if (l == 0) continue;
        const bool d0 = c.disk_z[l - 1] > 0.0, d1 = c.disk_z[l] > 0.0;
        if (!d0 && !d1 && (!(c.radius[l] > c.radius[l - 1]) || !(2.0 * c.hit_dr < c.radius[l] - c.radius[l - 1])))
            return TKF_ERR_INVALID;
        if (d0 && d1 && !(c.disk_z[l] > c.disk_z[l - 1])) return TKF_ERR_INVALID;
    }
    tkf_ctx *ctx = new (std::nothrow) tkf_ctx();
    if (!ctx) return TKF_ERR_NOMEM;
    ctx->cfg = c;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_tile, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_err, sizeof(int));
    if (e == cudaSuccess) e = index_event_prepare();
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        if (ctx->d_tile) cudaFree(ctx->d_tile);
        if (ctx->d_err) cudaFree(ctx->d_err);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? TKF_ERR_NOMEM : TKF_ERR_CUDA;
    }
    *out = ctx;
    return TKF_OK;
}

int tkf_destroy(tkf_ctx *ctx)
{
    if (!ctx) return TKF_ERR_INVALID;
    cudaFree(ctx->d_tile);
    cudaFree(ctx->d_err);
    for (int *p : {ctx->ord_key, ctx->ord_perm, ctx->ord_counts, ctx->ord_off, ctx->ord_seg_count, ctx->ord_seg_base,
                   (int *)ctx->first_key, ctx->first_hit, ctx->seed_b, ctx->seed_c, ctx->seed_cnt, (int *)ctx->seed_s})
        cudaFree(p);
    delete ctx;
    return TKF_OK;
}

const char *tkf_last_error(const tkf_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tkf_get_config(const tkf_ctx *ctx, tkf_config *out)
{
    if (!ctx || !out) return TKF_ERR_INVALID;
    *out = ctx->cfg;
    return TKF_OK;
}

int tkf_build_hit_index(tkf_ctx *ctx, const tkf_hits *hits, tkf_hit_index **out, tkf_stream stream)
{
    if (!ctx || !out) return TKF_ERR_INVALID;
    int st = check_hits(ctx, hits);
    if (st) return st;
    const tkf_config &c = ctx->cfg;
    const int L = c.n_layers, NB = c.n_eta_bins * c.n_phi_bins;
    const size_t n_segs = (size_t)hits->n_events * L;
    const size_t n_bins = n_segs * NB;
    if (n_bins >= (size_t)1 << 31 || n_segs > (1 << 22))
        return set_err(ctx, TKF_ERR_INVALID, "hit index: too many events for the bin table");
    tkf_hit_index *idx = *out;
    const bool fresh = idx == nullptr;
    if (fresh) {
        idx = new (std::nothrow) tkf_hit_index();
        if (!idx) return set_err(ctx, TKF_ERR_NOMEM, "hit index: host allocation failed");
        idx->ctx = ctx;
    }
    const size_t nh = (size_t)hits->n;
    if (nh > idx->cap_hits || fresh) {
        const size_t cap = std::max<size_t>(nh, 1);
        if ((st = grow(ctx, &idx->hxyzi, cap)) || (st = grow(ctx, &idx->hvar, cap)) ||
            (st = grow(ctx, &idx->pos_of_hit, cap)) || (st = grow(ctx, &idx->keys, cap)))
            goto fail;
        idx->cap_hits = cap;
    }
    if (n_bins > idx->cap_bins || fresh) {
        if ((st = grow(ctx, &idx->bin_off, n_bins + 1)) || (st = grow(ctx, &idx->counts, n_bins)) ||
            (st = grow(ctx, &idx->bin_sub, n_bins)))
            goto fail;
        idx->cap_bins = n_bins;
    }
    if (n_segs > idx->cap_segs || (size_t)hits->n_events + 1 > idx->cap_segs + 1 || fresh) {
        if ((st = grow(ctx, &idx->seg_count, n_segs)) || (st = grow(ctx, &idx->seg_base, n_segs)) ||
            (st = grow(ctx, &idx->var_max, n_segs)) || (st = grow(ctx, &idx->ev_off, n_segs + 1)))
            goto fail;
        idx->cap_segs = n_segs;
    }
    {
        idx->n = hits->n;
        idx->n_events = hits->n_events;
        idx->n_layers = L;
        idx->n_bins = NB;
        cudaStream_t s = (cudaStream_t)stream;
        const IndexGeom g = index_geom(c, hits->n_events);
        TKF_CUDA(ctx, cudaMemcpyAsync(idx->ev_off, hits->event_off, (hits->n_events + 1) * sizeof(int),
                                      cudaMemcpyDeviceToDevice, s));
        // one block per event when the batch has enough events to fill the GPU twice and their
        // bins fit a block's shared memory (set up by tkf_create); otherwise counts in global
        // memory and every block on the hits of a few events
        const size_t ev_smem = hits->n_events >= TKF_INDEX_EVENTS_PER_SM * ctx->sm_count ? index_event_smem(L, NB) : 0;
        if (ev_smem) {
            int *perm = idx->seg_base;  // >= n_events entries
            k_event_order<<<1, 1024, 0, s>>>(hits->event_off, hits->n_events, perm);
            k_index_event<<<(unsigned)hits->n_events, kEventThreads, ev_smem, s>>>(
                g, *hits, perm, (int)n_bins, idx->hxyzi, idx->hvar, idx->bin_off, idx->var_max, ctx->d_err);
            k_bin_sort<<<sort_blocks(n_bins), 32 * kSortWarps, 0, s>>>(g, idx->bin_off, idx->ev_off, (int)n_bins,
                                                                       idx->hxyzi, idx->hvar, idx->bin_sub,
                                                                       idx->pos_of_hit);
            TKF_CUDA(ctx, cudaGetLastError());
            *out = idx;
            return TKF_OK;
        }
        TKF_CUDA(ctx, cudaMemsetAsync(idx->counts, 0, n_bins * sizeof(int), s));
        TKF_CUDA(ctx, cudaMemsetAsync(idx->var_max, 0, n_segs * sizeof(float2), s));
        if (hits->n > 0) {
            const int nb = (hits->n + 255) / 256;
            k_hit_count<<<nb, 256, 0, s>>>(g, *hits, idx->keys, idx->counts, idx->seg_count, (int *)idx->var_max,
                                           ctx->d_err);
        }
        k_seg_total<<<(unsigned)n_segs, 256, 0, s>>>(idx->counts, idx->seg_count, NB);
        k_seg_scan<<<1, 1024, 0, s>>>(idx->seg_count, idx->seg_base, (int)n_segs);
        k_bin_scan<<<(unsigned)n_segs, 256, 0, s>>>(idx->counts, idx->seg_base, idx->bin_off, NB, (int)n_segs);
        if (hits->n > 0) {
            const int nb = (hits->n + 255) / 256;
            k_hit_scatter<<<nb, 256, 0, s>>>(g, *hits, idx->keys, idx->counts, idx->bin_off, idx->hxyzi, idx->hvar,
                                              ctx->d_err);
        }
        k_bin_sort<<<sort_blocks(n_bins), 32 * kSortWarps, 0, s>>>(g, idx->bin_off, idx->ev_off, (int)n_bins,
                                                                   idx->hxyzi, idx->hvar, idx->bin_sub, idx->pos_of_hit);
        TKF_CUDA(ctx, cudaGetLastError());
    }
    *out = idx;
    return TKF_OK;
fail:
    if (fresh) {
        tkf_hit_index_free(idx);
    }
    return st;
}

int tkf_hit_index_free(tkf_hit_index *idx)
{
    if (!idx) return TKF_ERR_INVALID;
    cudaFree(idx->hxyzi);
    cudaFree(idx->hvar);
    cudaFree(idx->pos_of_hit);
    cudaFree(idx->bin_sub);
    cudaFree(idx->keys);
    cudaFree(idx->bin_off);
    cudaFree(idx->counts);
    cudaFree(idx->seg_count);
    cudaFree(idx->seg_base);
    cudaFree(idx->var_max);
    cudaFree(idx->ev_off);
    delete idx;
    return TKF_OK;
}

int tkf_hit_index_get_view(const tkf_hit_index *idx, tkf_hit_index_view *v)
{
    if (!idx || !v) return TKF_ERR_INVALID;
    v->hit_xyzi = (const float *)idx->hxyzi;
    v->hit_var = (const float *)idx->hvar;
    v->bin_sub = (const uint32_t *)idx->bin_sub;
    v->pos_of_hit = idx->pos_of_hit;
    v->bin_off = idx->bin_off;
    v->var_max = (const float *)idx->var_max;
    v->event_off = idx->ev_off;
    v->n = idx->n;
    v->n_events = idx->n_events;
    v->n_layers = idx->n_layers;
    v->n_bins = idx->n_bins;
    return TKF_OK;
}

int tkf_seed_state(tkf_ctx *ctx, const tkf_hits *hits, const int32_t *seed_hits, tkf_tracks *out, tkf_stream stream)
{
    if (!ctx) return TKF_ERR_INVALID;
    int st = check_hits(ctx, hits);
    if (st || (st = check_tracks(ctx, out, false, "out"))) return st;
    if (out->n > 0 && !seed_hits) return set_err(ctx, TKF_ERR_INVALID, "seed_hits is null");
    if (out->n == 0) return TKF_OK;
    const FitGeom g = fit_geom(ctx);
    const int nb = (out->n + 127) / 128;
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->cfg.precision == TKF_FP64)
        k_seed<double><<<nb, 128, 0, s>>>(g, *hits, seed_hits, *out, ctx->d_err);
    else
        k_seed<float><<<nb, 128, 0, s>>>(g, *hits, seed_hits, *out, ctx->d_err);
    TKF_CUDA(ctx, cudaGetLastError());
    return TKF_OK;
}

int tkf_fit(tkf_ctx *ctx, const tkf_hits *hits, const tkf_tracks *init, const int32_t *hit_idx, int32_t first_layer,
            int32_t last_layer, tkf_tracks *out, tkf_stream stream)
{
    return tkf::fit_tracks(ctx, hits, init, hit_idx, first_layer, last_layer, out, stream, false);
}

int tkf_fit_continue(tkf_ctx *ctx, const tkf_hits *hits, const tkf_tracks *init, const int32_t *hit_idx,
                     int32_t first_layer, int32_t last_layer, tkf_tracks *out, tkf_stream stream)
{
    return tkf::fit_tracks(ctx, hits, init, hit_idx, first_layer, last_layer, out, stream, true);
}

int tkf_seed_fit(tkf_ctx *ctx, const tkf_hits *hits, const int32_t *seed_hits, int32_t last_layer, tkf_tracks *out,
                 tkf_stream stream)
{
    return tkf::seed_and_fit(ctx, hits, seed_hits, last_layer, out, stream);
}

int tkf_fit_backward(tkf_ctx *ctx, const tkf_hits *hits, const tkf_tracks *init, const int32_t *hit_idx,
                     int32_t last_layer, int32_t first_layer, double cov_scale, tkf_tracks *out, tkf_stream stream)
{
    return tkf::fit_backward(ctx, hits, init, hit_idx, last_layer, first_layer, cov_scale, out, stream);
}

}  // extern "C"

int tkf::fit_tracks(tkf_ctx *ctx, const tkf_hits *hits, const tkf_tracks *init, const int32_t *hit_idx,
                    int32_t first_layer, int32_t last_layer, tkf_tracks *out, tkf_stream stream, bool continue_fit)
{
    if (!ctx) return TKF_ERR_INVALID;
    if (continue_fit && first_layer < 1) return set_err(ctx, TKF_ERR_INVALID, "a continued fit starts at layer >= 1");
    int st = check_hits(ctx, hits);
    if (st || (st = check_tracks(ctx, init, hit_idx == nullptr, "init")) || (st = check_tracks(ctx, out, false, "out")))
        return st;
    if (out->n != init->n) return set_err(ctx, TKF_ERR_INVALID, "out->n must equal init->n");
    if (first_layer < 0 || last_layer < first_layer || last_layer >= ctx->cfg.n_layers)
        return set_err(ctx, TKF_ERR_INVALID, "need 0 <= first_layer <= last_layer < n_layers");
    if (init->n == 0) return TKF_OK;
    const int32_t *hidx = hit_idx ? hit_idx : init->hit_idx;
    const FitGeom g = fit_geom(ctx);
    const int nb = (init->n + 127) / 128;
    cudaStream_t s = (cudaStream_t)stream;
    const int pf = continue_fit ? 1 : 0;
    auto go = [&](auto kern) {
        kern<<<nb, kFitThreads, 0, s>>>(g, *hits, *init, hidx, first_layer, last_layer, pf, *out, ctx->d_err);
    };
    const bool dk = g.disk_mask != 0;
    switch (ctx->cfg.precision) {
    case TKF_FP32: dk ? go(k_fit<float, float, true>) : go(k_fit<float, float, false>); break;
    case TKF_MIXED: dk ? go(k_fit<float, double, true>) : go(k_fit<float, double, false>); break;
    default: dk ? go(k_fit<double, double, true>) : go(k_fit<double, double, false>); break;
    }
    TKF_CUDA(ctx, cudaGetLastError());
    return TKF_OK;
}

int tkf::fit_backward(tkf_ctx *ctx, const tkf_hits *hits, const tkf_tracks *init, const int32_t *hit_idx,
                      int32_t last_layer, int32_t first_layer, double cov_scale, tkf_tracks *out, tkf_stream stream)
{
    if (!ctx) return TKF_ERR_INVALID;
    int st = check_hits(ctx, hits);
    if (st || (st = check_tracks(ctx, init, hit_idx == nullptr, "init")) || (st = check_tracks(ctx, out, false, "out")))
        return st;
    if (out->n != init->n) return set_err(ctx, TKF_ERR_INVALID, "out->n must equal init->n");
    if (first_layer < 0 || last_layer < first_layer || last_layer >= ctx->cfg.n_layers)
        return set_err(ctx, TKF_ERR_INVALID, "need 0 <= first_layer <= last_layer < n_layers");
    if (!(cov_scale > 0.0) || !std::isfinite(cov_scale))
        return set_err(ctx, TKF_ERR_INVALID, "cov_scale must be positive and finite");
    if (init->n == 0) return TKF_OK;
    const int32_t *hidx = hit_idx ? hit_idx : init->hit_idx;
    const FitGeom g = fit_geom(ctx);
    const int nb = (init->n + 127) / 128;
    cudaStream_t s = (cudaStream_t)stream;
    auto go = [&](auto kern, auto scale) {
        kern<<<nb, kFitThreads, 0, s>>>(g, *hits, *init, hidx, last_layer, first_layer, scale, *out, ctx->d_err);
    };
    const bool dk = g.disk_mask != 0;
    const float sf = (float)cov_scale;
    switch (ctx->cfg.precision) {
    case TKF_FP32: dk ? go(k_fit_backward<float, float, true>, sf) : go(k_fit_backward<float, float, false>, sf); break;
    case TKF_MIXED:
        dk ? go(k_fit_backward<float, double, true>, sf) : go(k_fit_backward<float, double, false>, sf);
        break;
    default:
        dk ? go(k_fit_backward<double, double, true>, cov_scale) : go(k_fit_backward<double, double, false>, cov_scale);
        break;
    }
    TKF_CUDA(ctx, cudaGetLastError());
    return TKF_OK;
}

int tkf::seed_and_fit(tkf_ctx *ctx, const tkf_hits *hits, const int32_t *seed_hits, int32_t last_layer,
                      tkf_tracks *out, tkf_stream stream)
{
    if (!ctx) return TKF_ERR_INVALID;
    int st = check_hits(ctx, hits);
    if (st || (st = check_tracks(ctx, out, false, "out"))) return st;
    if (out->n > 0 && !seed_hits) return set_err(ctx, TKF_ERR_INVALID, "seed_hits is null");
    if (last_layer < 0 || last_layer >= ctx->cfg.n_layers)
        return set_err(ctx, TKF_ERR_INVALID, "need 0 <= last_layer < n_layers");
    if (out->n == 0) return TKF_OK;
    const FitGeom g = fit_geom(ctx);
    const int nb = (out->n + 127) / 128;
    cudaStream_t s = (cudaStream_t)stream;
    auto go = [&](auto kern) { kern<<<nb, kFitThreads, 0, s>>>(g, *hits, seed_hits, last_layer, *out, ctx->d_err); };
    const bool dk = g.disk_mask != 0;
    switch (ctx->cfg.precision) {
    case TKF_FP32: dk ? go(k_seed_fit<float, float, true>) : go(k_seed_fit<float, float, false>); break;
    case TKF_MIXED: dk ? go(k_seed_fit<float, double, true>) : go(k_seed_fit<float, double, false>); break;
    default: dk ? go(k_seed_fit<double, double, true>) : go(k_seed_fit<double, double, false>); break;
    }
    TKF_CUDA(ctx, cudaGetLastError());
    return TKF_OK;
}

extern "C" {

int tkf_build_tracks(tkf_ctx *ctx, const tkf_hit_index *idx, const tkf_tracks *seeds, tkf_tracks *out,
                     tkf_tracks *out_all, int32_t *n_cand_out, tkf_stream stream)
{
    if (!ctx) return TKF_ERR_INVALID;
    if (!idx) return set_err(ctx, TKF_ERR_INVALID, "hit index is null");
    const tkf_config &c = ctx->cfg;
    int st = check_tracks(ctx, seeds, false, "seeds");
    if (st || (st = check_tracks(ctx, out, false, "out"))) return st;
    if (out->stride < seeds->n) return set_err(ctx, TKF_ERR_INVALID, "out->stride < seeds->n");
    if (out_all && ((st = check_tracks(ctx, out_all, false, "out_all")) ||
                    (size_t)out_all->stride < (size_t)seeds->n * c.n_cand))
        return st ? st : set_err(ctx, TKF_ERR_INVALID, "out_all->stride < seeds->n * n_cand");
    if (idx->n_layers != c.n_layers || idx->n_bins != c.n_eta_bins * c.n_phi_bins)
        return set_err(ctx, TKF_ERR_INVALID, "hit index built with another geometry");
    if (seeds->n == 0) return TKF_OK;
    BuildArgs a{};
    a.L = c.n_layers;
    a.first = c.first_build_layer;
    a.ncand = c.n_cand;
    a.n_eta = c.n_eta_bins;
    a.n_phi = c.n_phi_bins;
    a.n_bins = c.n_eta_bins * c.n_phi_bins;
    // default work tile: two groups of seeds per warp (small tiles keep every warp busy when
    // a launch holds a single event)
    a.seeds_per_block = c.seeds_per_block > 0 ? c.seeds_per_block : 2 * (32 / c.n_cand);
    a.n_seeds = seeds->n;
    a.n_events = idx->n_events;
    for (int l = 0; l < c.n_layers; ++l) {
        a.radius[l] = c.radius[l];
        a.xx0[l] = c.x_over_x0[l];
        a.radius_f[l] = (float)c.radius[l];
        a.xx0_f[l] = (float)c.x_over_x0[l];
    }
    a.kb = kCurv * c.bz;
    a.mass = c.mass;
    a.eta_min = c.eta_min;
    a.inv_eta_w = 1.0 / c.eta_bin_w;
    a.cut = c.chi2_cut;
    a.margin = c.window_margin;
    a.hit_dr = c.hit_dr;
    a.hit_dr_f = (float)c.hit_dr;
    for (int l = 0; l < c.n_layers; ++l) {
        a.disk_z[l] = c.disk_z[l];
        a.disk_z_f[l] = (float)c.disk_z[l];
        if (c.disk_z[l] > 0.0) a.disk_mask |= 1u << l;
    }
    a.kb_f = (float)a.kb;
    a.mass_f = (float)a.mass;
    a.eta_min_f = (float)a.eta_min;
    a.inv_eta_w_f = (float)a.inv_eta_w;
    a.cut_f = (float)a.cut;
    a.margin_f = (float)a.margin;
    a.hxyzi = idx->hxyzi;
    a.hvar = idx->hvar;
    a.bin_sub = idx->bin_sub;
    a.pos_of_hit = idx->pos_of_hit;
    a.bin_off = idx->bin_off;
    a.var_max = idx->var_max;
    a.ev_off = idx->ev_off;
    a.s_par = seeds->par;
    a.s_cov = seeds->cov;
    a.s_chi2 = seeds->chi2;
    a.s_nhits = seeds->nhits;
    a.s_hit = seeds->hit_idx;
    a.s_event = seeds->event;
    a.s_stride = seeds->stride;
    a.o_par = out->par;
    a.o_cov = out->cov;
    a.o_chi2 = out->chi2;
    a.o_nhits = out->nhits;
    a.o_hit = out->hit_idx;
    a.o_stride = out->stride;
    if (out_all) {
        a.a_par = out_all->par;
        a.a_cov = out_all->cov;
        a.a_chi2 = out_all->chi2;
        a.a_nhits = out_all->nhits;
        a.a_hit = out_all->hit_idx;
        a.a_stride = out_all->stride;
    }
    a.n_cand_out = n_cand_out;
    a.tile_counter = ctx->d_tile;
    a.err = ctx->d_err;
    cudaStream_t s = (cudaStream_t)stream;
    if (c.seed_order) {
        // counting sort of the seeds by (event, eta bin, phi bin) on the last seeding layer
        if ((st = tkf::seed_order_reserve(ctx, (size_t)seeds->n, (size_t)idx->n_events))) return st;
        const IndexGeom g = index_geom(c, idx->n_events);
        const int nb = (seeds->n + 255) / 256, layer = c.first_build_layer - 1;
        if (c.precision == TKF_FP64)
            k_seed_key<double><<<nb, 256, 0, s>>>(g, layer, (const double *)seeds->par, seeds->stride, seeds->event,
                                                  seeds->n, ctx->ord_key, ctx->ord_counts);
        else
            k_seed_key<float><<<nb, 256, 0, s>>>(g, layer, (const float *)seeds->par, seeds->stride, seeds->event,
                                                 seeds->n, ctx->ord_key, ctx->ord_counts);
        k_seg_total<<<(unsigned)idx->n_events, 256, 0, s>>>(ctx->ord_counts, ctx->ord_seg_count, g.n_bins);
        k_seg_scan<<<1, 1024, 0, s>>>(ctx->ord_seg_count, ctx->ord_seg_base, idx->n_events);
        k_bin_scan<<<(unsigned)idx->n_events, 256, 0, s>>>(ctx->ord_counts, ctx->ord_seg_base, ctx->ord_off, g.n_bins,
                                                           idx->n_events);
        k_seed_place<<<nb, 256, 0, s>>>(ctx->ord_key, ctx->ord_counts, ctx->ord_off, seeds->n, ctx->ord_perm);
        a.s_perm = ctx->ord_perm;  // counts are back to zero after k_seed_place
    }
    const int nmax = build_nmax(c.n_cand);
    if (TKF_BUILD_FIRST_PASS && c.first_build_layer < c.n_layers && seeds->n > 0) {
        if ((st = tkf::first_list_reserve(ctx, (size_t)seeds->n))) return st;
        a.f_key = ctx->first_key;
        a.f_hit = ctx->first_hit;
    }
    auto launch = a.disk_mask    ? (c.precision == TKF_FP32    ? launch_build3_fp32
                                    : c.precision == TKF_MIXED ? launch_build3_mixed
                                                               : launch_build3_fp64)
                  : c.hit_dr > 0.0 ? (c.precision == TKF_FP32    ? launch_build2_fp32
                                    : c.precision == TKF_MIXED ? launch_build2_mixed
                                                               : launch_build2_fp64)
                                   : (c.precision == TKF_FP32    ? launch_build_fp32
                                    : c.precision == TKF_MIXED ? launch_build_mixed
                                                               : launch_build_fp64);
    int occ = 0;
    TKF_CUDA(ctx, launch(a, nmax, 0, nullptr, &occ));
    const long long tiles = ((long long)seeds->n + a.seeds_per_block - 1) / a.seeds_per_block;
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)std::max(occ, 1) * ctx->sm_count));
    TKF_CUDA(ctx, cudaMemsetAsync(ctx->d_tile, 0, sizeof(int), s));
    TKF_CUDA(ctx, launch(a, nmax, grid, s, nullptr));
    TKF_CUDA(ctx, cudaGetLastError());
    return TKF_OK;
}

int tkf_sync_status(tkf_ctx *ctx, tkf_stream stream)
{
    if (!ctx) return TKF_ERR_INVALID;
    TKF_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)stream));
    int e = 0;
    TKF_CUDA(ctx, cudaMemcpy(&e, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        TKF_CUDA(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
        char buf[160];
        std::snprintf(buf, sizeof buf, "kernel error bits 0x%x (1: hit layer out of range, 2: hit id out of range, 4: more than 8388606 hits "
                      "in one event, 8: seed event out of range)", e);
        return set_err(ctx, TKF_ERR_KERNEL, buf);
    }
    return TKF_OK;
}

// ---------------------------------------------------------------- allocation-free hit index
//
// Scratch of tkf_build_hit_index_noalloc: per-hit bin keys, per-bin counters, per-segment
// totals and bases, and one error word, in a fixed array of the library's device memory.

}  // extern "C"

namespace {

constexpr size_t kNoallocWords =
    (size_t)TKF_NOALLOC_MAX_HITS + TKF_NOALLOC_MAX_BINS + 2 * (size_t)TKF_NOALLOC_MAX_SEGMENTS + 64;
static __device__ __align__(256) int g_noalloc_scratch[kNoallocWords];

// Device address of g_noalloc_scratch per device, looked up once with that device current.
std::mutex g_noalloc_mutex;
int *g_noalloc_addr[64] = {};

int g_noalloc_sms[64] = {};

int noalloc_scratch(int **out, int *sm_count)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TKF_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        int *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, g_noalloc_scratch) != cudaSuccess || !p) return TKF_ERR_CUDA;
        if (index_event_prepare() != cudaSuccess) return TKF_ERR_CUDA;
        if (cudaDeviceGetAttribute(&g_noalloc_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return TKF_ERR_CUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    *sm_count = g_noalloc_sms[dev];
    return TKF_OK;
}

}  // namespace

extern "C" int tkf_build_hit_index_noalloc(const tkf_config *cfg, const tkf_hits *hits, const tkf_hit_index_out *out,
                                           tkf_stream stream)
{
    if (!cfg || !hits || !out) return TKF_ERR_INVALID;
    const tkf_config &c = *cfg;
    if (c.n_layers < 1 || c.n_layers > TKF_MAX_LAYERS || c.n_eta_bins < 1 || c.n_phi_bins < 1 ||
        !(c.eta_bin_w > 0))
        return TKF_ERR_INVALID;
    for (int l = 0; l < c.n_layers; ++l)
        if (!(c.radius[l] > 0)) return TKF_ERR_INVALID;
    if (hits->n < 0 || hits->n_events < 1 || !hits->event_off) return TKF_ERR_INVALID;
    if (hits->n > 0 && (!hits->x || !hits->y || !hits->z || !hits->var_u || !hits->var_v || !hits->layer))
        return TKF_ERR_INVALID;
    if (!out->hit_xyzi || !out->hit_var || !out->bin_sub || !out->pos_of_hit || !out->bin_off || !out->var_max ||
        !out->event_off)
        return TKF_ERR_INVALID;
    const int L = c.n_layers, NB = c.n_eta_bins * c.n_phi_bins;
    const size_t n_segs = (size_t)hits->n_events * L;
    const size_t n_bins = n_segs * NB;
    if ((size_t)hits->n > TKF_NOALLOC_MAX_HITS || n_bins > TKF_NOALLOC_MAX_BINS || n_segs > TKF_NOALLOC_MAX_SEGMENTS)
        return TKF_ERR_TOO_LARGE;
    int *scratch = nullptr, n_sm = 0;
    int st = noalloc_scratch(&scratch, &n_sm);
    if (st) return st;
    int *keys = scratch;
    int *counts = keys + TKF_NOALLOC_MAX_HITS;
    int *seg_count = counts + TKF_NOALLOC_MAX_BINS;
    int *seg_base = seg_count + TKF_NOALLOC_MAX_SEGMENTS;
    int *err = seg_base + TKF_NOALLOC_MAX_SEGMENTS;
    const IndexGeom g = index_geom(c, hits->n_events);
    cudaStream_t s = (cudaStream_t)stream;
    float4 *hxyzi = (float4 *)out->hit_xyzi;
    float2 *hvar = (float2 *)out->hit_var;
    if (cudaMemcpyAsync(out->event_off, hits->event_off, (hits->n_events + 1) * sizeof(int), cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
        return TKF_ERR_CUDA;
    if (const size_t ev_smem = hits->n_events >= TKF_INDEX_EVENTS_PER_SM * n_sm ? index_event_smem(L, NB) : 0) {
        // one block per event
        k_event_order<<<1, 1024, 0, s>>>(hits->event_off, hits->n_events, seg_base);
        k_index_event<<<(unsigned)hits->n_events, kEventThreads, ev_smem, s>>>(
            g, *hits, seg_base, (int)n_bins, hxyzi, hvar, out->bin_off, (float2 *)out->var_max, err);
        k_bin_sort<<<sort_blocks(n_bins), 32 * kSortWarps, 0, s>>>(g, out->bin_off, out->event_off, (int)n_bins, hxyzi,
                                                                   hvar, (uint4 *)out->bin_sub, out->pos_of_hit);
        return cudaGetLastError() == cudaSuccess ? TKF_OK : TKF_ERR_CUDA;
    }
    if (cudaMemsetAsync(counts, 0, n_bins * sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(out->var_max, 0, n_segs * 2 * sizeof(float), s) != cudaSuccess)
        return TKF_ERR_CUDA;
    if (hits->n > 0)
        k_hit_count<<<(hits->n + 255) / 256, 256, 0, s>>>(g, *hits, keys, counts, seg_count, (int *)out->var_max, err);
    k_seg_total<<<(unsigned)n_segs, 256, 0, s>>>(counts, seg_count, NB);
    k_seg_scan<<<1, 1024, 0, s>>>(seg_count, seg_base, (int)n_segs);
    k_bin_scan<<<(unsigned)n_segs, 256, 0, s>>>(counts, seg_base, out->bin_off, NB, (int)n_segs);
    if (hits->n > 0)
        k_hit_scatter<<<(hits->n + 255) / 256, 256, 0, s>>>(g, *hits, keys, counts, out->bin_off, hxyzi, hvar, err);
    k_bin_sort<<<sort_blocks(n_bins), 32 * kSortWarps, 0, s>>>(g, out->bin_off, out->event_off, (int)n_bins, hxyzi,
                                                               hvar, (uint4 *)out->bin_sub, out->pos_of_hit);
    return cudaGetLastError() == cudaSuccess ? TKF_OK : TKF_ERR_CUDA;
}
