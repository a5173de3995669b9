// Host-side internals shared by the translation units of libtkf.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "tkf.h"

namespace tkf {

constexpr int kBuildThreads = 128;  // 4 warps per block
constexpr int kHoleId = 0x7FFFFF;   // event-local hit id field value of a hole branch
constexpr int kMaxHitsPerEvent = 0x7FFFFF - 1;
constexpr int kSubBins = 16;        // phi sub-bins per phi bin recorded by the hit index

// error bits raised by kernels (atomicOr into the context's error word)
enum : int { kErrBadLayer = 1, kErrBadHitId = 2, kErrTooManyHits = 4, kErrBadEvent = 8 };

struct BuildArgs {
    int L, first, ncand, n_eta, n_phi, n_bins, seeds_per_block, n_seeds, n_events;
    float radius_f[TKF_MAX_LAYERS], xx0_f[TKF_MAX_LAYERS];
    double radius[TKF_MAX_LAYERS], xx0[TKF_MAX_LAYERS];
    float kb_f, mass_f, eta_min_f, inv_eta_w_f, cut_f, margin_f, hit_dr_f;
    double kb, mass, eta_min, inv_eta_w, cut, margin, hit_dr;
    float disk_z_f[TKF_MAX_LAYERS];
    double disk_z[TKF_MAX_LAYERS];
    unsigned disk_mask;  // bit l: layer l is a pair of endcap disks at z = +-disk_z[l]
    // hit index
    const float4 *hxyzi;
    const float2 *hvar;
    const uint4 *bin_sub;
    const int *pos_of_hit;
    const int *bin_off;
    const float2 *var_max;
    const int *ev_off;
    // seeds
    const void *s_par, *s_cov, *s_chi2;
    const int *s_nhits, *s_hit, *s_event;
    const int *s_perm;  // processing order of the seeds (null: input order)
    int s_stride;
    // best candidate per seed
    void *o_par, *o_cov, *o_chi2;
    int *o_nhits, *o_hit;
    int o_stride;
    // every final candidate (optional)
    void *a_par, *a_cov, *a_chi2;
    int *a_nhits, *a_hit;
    int a_stride;
    int *n_cand_out;
    // branch lists of the first building layer, [NMAX][n_seeds] by seed (written by k_first_scan
    // before k_build; null: k_build scans that layer itself)
    unsigned *f_key;
    int *f_hit;
    int *tile_counter;
    int *err;
};

// Launchers of the build kernel, one translation unit per precision.  `nmax` is the
// compile-time candidate capacity (1, 4, 6, 10 or 16) >= a.ncand.  `occupancy` (if not
// null) receives the resident blocks per SM of that instantiation instead of launching.
cudaError_t launch_build_fp32(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy);
cudaError_t launch_build_mixed(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy);
cudaError_t launch_build_fp64(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy);
// The same for hits off the layers' cylinders (a.hit_dr > 0): the two-step building of Sec. 2.2.
cudaError_t launch_build2_fp32(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy);
cudaError_t launch_build2_mixed(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy);
cudaError_t launch_build2_fp64(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy);
// The same for configurations with endcap disks (a.disk_mask != 0; the "endcap z" of Sec. 2.2).
cudaError_t launch_build3_fp32(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy);
cudaError_t launch_build3_mixed(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy);
cudaError_t launch_build3_fp64(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy);

// tkf_fit, and its continued form (continue_fit: `init` lies on layer first_layer - 1, as a
// fit of the earlier layers leaves it; the fit propagates before its first update).
int fit_tracks(tkf_ctx *ctx, const tkf_hits *hits, const tkf_tracks *init, const int32_t *hit_idx, int32_t first_layer,
               int32_t last_layer, tkf_tracks *out, tkf_stream stream, bool continue_fit);

// tkf_seed_state followed by tkf_fit over layers 0..last_layer in one kernel (the estimate is not
// stored): the seed fit of the batched pipeline.
int seed_and_fit(tkf_ctx *ctx, const tkf_hits *hits, const int32_t *seed_hits, int32_t last_layer, tkf_tracks *out,
                 tkf_stream stream);

// tkf_fit_backward: the inward pass over layers last_layer..first_layer.
int fit_backward(tkf_ctx *ctx, const tkf_hits *hits, const tkf_tracks *init, const int32_t *hit_idx,
                 int32_t last_layer, int32_t first_layer, double cov_scale, tkf_tracks *out, tkf_stream stream);

// Allocates (or grows) `*idx` so that batches of up to max_hits hits and max_events events
// need no further allocation (used before capturing the pipeline into a CUDA graph).
int hit_index_reserve(tkf_ctx *ctx, tkf_hit_index **idx, size_t max_hits, size_t max_events);

// Scratch of the seed ordering in tkf_build_tracks, sized for max_seeds seeds of max_events
// events (grown on demand outside graph capture; reserved by the pipeline).
int seed_order_reserve(tkf_ctx *ctx, size_t max_seeds, size_t max_events);

// Branch lists of the first building layer (k_first_scan) for max_seeds seeds of the
// configuration's candidate capacity (grown on demand outside graph capture; reserved by the
// pipeline).
int first_list_reserve(tkf_ctx *ctx, size_t max_seeds);

inline int build_nmax(int n)
{
    return n <= 1 ? 1 : n <= 4 ? 4 : n <= 6 ? 6 : n <= 10 ? 10 : 16;
}

}  // namespace tkf

struct tkf_ctx {
    tkf_config cfg;
    int device = 0;
    int sm_count = 0;
    std::string err;
    int *d_tile = nullptr;  // work-tile counter of the persistent build kernel
    int *d_err = nullptr;   // error bits raised by kernels
    // seed ordering scratch: key and permutation per seed, counts and offsets per (event, bin)
    int *ord_key = nullptr, *ord_perm = nullptr, *ord_counts = nullptr, *ord_off = nullptr;
    int *ord_seg_count = nullptr, *ord_seg_base = nullptr;
    size_t ord_cap_seeds = 0, ord_cap_bins = 0, ord_cap_events = 0;
    // first-layer branch lists: key and hit id planes of first_cap entries each
    unsigned *first_key = nullptr;
    int *first_hit = nullptr;
    size_t first_cap = 0;
    // seeding scratch: best layer-1 / layer-2 hit and score per sorted hit position, seeds per block
    int *seed_b = nullptr, *seed_c = nullptr, *seed_cnt = nullptr;
    float *seed_s = nullptr;
    size_t seed_cap = 0, seed_cnt_cap = 0;
};

struct tkf_hit_index {
    tkf_ctx *ctx = nullptr;
    int n = 0, n_events = 0, n_layers = 0, n_bins = 0;
    size_t cap_hits = 0, cap_bins = 0, cap_segs = 0;
    float4 *hxyzi = nullptr;
    float2 *hvar = nullptr;
    uint4 *bin_sub = nullptr;  // cap_bins
    int *pos_of_hit = nullptr;
    int *keys = nullptr;
    int *bin_off = nullptr;   // cap_bins + 1
    int *counts = nullptr;    // cap_bins
    int *seg_count = nullptr; // cap_segs
    int *seg_base = nullptr;  // cap_segs
    float2 *var_max = nullptr;
    int *ev_off = nullptr;    // cap_segs + 1 (>= n_events + 1)
};
