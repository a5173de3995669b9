/*
 * tkf -- Kalman-filter track building and fitting on one GB300 (sm_103a).
 *
 * C ABI of the library libtkf.so.  The method is the Kalman-filter (KF) tracking of
 * Cerati et al., "Kalman filter tracking on parallel architectures" (arXiv:1702.06359):
 * seeding, combinatorial track building and a final KF fit (Sec. 2), in the hybrid
 * coordinates of Sec. 2.2 (global Cartesian position, polar momentum) on the ideal barrel of
 * Sec. 2.2 (thin cylinders, uniform solenoid field Bz), with the KF update on the plane
 * tangent to the cylinder at the hit (Sec. 2.2).
 *
 * Conventions for every call:
 *  - Return value: TKF_OK (0) or a TKF_ERR_* code; no C++ exception crosses the ABI.  The
 *    text of the last error of a context is given by tkf_last_error().
 *  - Array arguments named "device" are CUDA device pointers owned by the caller (for
 *    example PyTorch tensors); they must stay valid until the work queued on `stream` has
 *    completed.  Host structs passed by pointer are read during the call only.
 *  - Work is queued asynchronously on `stream` (NULL = the legacy default stream); a call
 *    returning TKF_OK means the work was queued, not that it finished.  Errors found while
 *    the kernels run are reported per track (see tkf_tracks.nhits) and by tkf_sync_status().
 *  - Track state p = (x, y, z, q/pT, phi, theta) in cm, GeV^-1, rad; covariances are the 21
 *    elements of the lower triangle in row order: (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) ...
 *  - Layers are numbered from 0 (innermost).  Hit ids are indices into the caller's hit
 *    arrays (tkf_hits); -1 means "no hit on this layer" (a hole).
 */
#ifndef TKF_H
#define TKF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TKF_MAX_LAYERS 16
#define TKF_MAX_CAND 16

typedef struct CUstream_st *tkf_stream; /* a cudaStream_t */

enum tkf_status_code {
    TKF_OK = 0,
    TKF_ERR_INVALID = 1,  /* bad argument or configuration; nothing was queued */
    TKF_ERR_CUDA = 2,     /* a CUDA runtime call failed (text in tkf_last_error) */
    TKF_ERR_NOMEM = 3,    /* device allocation failed */
    TKF_ERR_AGAIN = 4,    /* queue or device-memory budget full: retry later */
    TKF_ERR_TIMEOUT = 5,  /* a bounded wait ran out */
    TKF_ERR_NOTREADY = 6, /* result not available yet */
    TKF_ERR_KERNEL = 7,   /* a kernel reported an internal error word */
    TKF_ERR_TOO_LARGE = 8 /* input exceeds the fixed capacity of tkf_build_hit_index_noalloc */
};

/* Arithmetic of the KF steps (Sec. 3.2: the update's numerical stability).  FP32: everything
 * in float.  MIXED: float, except the innovation covariance, its inverse, the gain and the
 * Joseph-form covariance update, done in double and rounded back (the state update applies
 * the rounded gain in float).  FP64: everything in double (track arrays hold double). */
enum tkf_precision { TKF_FP32 = 0, TKF_MIXED = 1, TKF_FP64 = 2 };

/* Per-track status written to tkf_tracks.nhits when a track fails (nhits < 0). */
enum tkf_track_status { TKF_TRACK_NOREACH = -1, TKF_TRACK_SINGULAR = -2, TKF_TRACK_LOST = -3 };

typedef struct {
    int32_t n_layers;                 /* barrel cylinders, <= TKF_MAX_LAYERS */
    double radius[TKF_MAX_LAYERS];    /* cm, increasing */
    double x_over_x0[TKF_MAX_LAYERS]; /* thin-scatterer thickness of each layer (0 = none) */
    double bz;                        /* T, uniform field along z */
    double mass;                      /* GeV, mass hypothesis for the scattering width */
    double prior_sigma[6];            /* seed prior (cm, cm, cm, GeV^-1, rad, rad) */
    double eta_min, eta_bin_w;        /* hit index: eta bins of width eta_bin_w from eta_min */
    int32_t n_eta_bins, n_phi_bins;   /* phi bins cover [-pi, pi) */
    double chi2_cut;                  /* a hit is compatible when chi2 < chi2_cut (2 dof) */
    double window_margin;             /* relative widening of the chi2 bounding box */
    int32_t n_cand;                   /* candidates kept per seed while building, 1..16 */
    int32_t first_build_layer;        /* seeds are states on layer first_build_layer - 1 */
    int32_t precision;                /* enum tkf_precision */
    int32_t seeds_per_block;          /* seeds per work tile of the build kernel (one warp takes a
                                         tile at a time); 0 = default */
    int32_t seed_order;               /* 1: build seeds grouped by (event, eta bin, phi bin) so that a
                                         warp's seeds share hit-index cache lines (results do not
                                         depend on it); 0: in input order */
    double hit_dr;                    /* cm, largest |hit radius - radius[layer]|.  0: hits lie on
                                         the cylinders.  > 0 (hits on modules off the average
                                         cylinder, the simplified CMS geometry of Sec. 2.2): fits
                                         take each layer's state to its hit's own radius; building
                                         propagates to the layer's radius, opens the window there
                                         widened by the track's travel over hit_dr, and takes each
                                         candidate hit's chi2 after a second propagation to the
                                         hit's radius.  Must satisfy 0 <= hit_dr < radius[0] and
                                         2 hit_dr < the gap between consecutive radii. */
    double disk_z[TKF_MAX_LAYERS];    /* cm.  0: layer l is the cylinder of radius[l].  > 0: layer l
                                         is a pair of endcap disks at z = +-disk_z[l] (the "endcap
                                         z" of Sec. 2.2; radius[l] is then the disk's outer
                                         radius): a state goes to the disk on the side of its z by
                                         the exact helix/plane crossing, a hit there is measured in
                                         r-phi (var_u) and r (var_v), its eta bin is
                                         asinh(z / r_hit), and the seed's z on a first-layer disk
                                         is exact (zero prior variance).  Consecutive disk layers
                                         need increasing disk_z; disks exclude hit_dr > 0. */
} tkf_config;

/* Hits of one or more events (device arrays of length n, caller-owned).  The hits of event e
 * are [event_off[e], event_off[e+1]); at most 8388606 hits per event.  layer in
 * [0, n_layers).  var_u / var_v: measurement variances along the cylinder's tangent (r-phi)
 * and along z (cm^2). */
typedef struct {
    const float *x, *y, *z, *var_u, *var_v;
    const int32_t *layer;
    const int32_t *event_off; /* device, n_events + 1 entries */
    int32_t n, n_events;
} tkf_hits;

/* Track structure-of-arrays, track-major planes of `stride` elements (caller-owned device
 * memory).  Element type of par/cov/chi2 is float, or double when precision == TKF_FP64.
 *   par     [6][stride]   cov [21][stride]   chi2 [stride]
 *   nhits   [stride]  hits used (< 0: enum tkf_track_status)
 *   hit_idx [n_layers][stride]  hit id per layer, -1 = none (may be NULL where unused)
 *   event   [stride]  event index of each track (may be NULL: every track in event 0) */
typedef struct {
    void *par, *cov, *chi2;
    int32_t *nhits, *hit_idx, *event;
    int32_t n, stride;
} tkf_tracks;

typedef struct tkf_ctx tkf_ctx;
typedef struct tkf_hit_index tkf_hit_index;

/* Device view of a hit index (pointers owned by the index). */
typedef struct {
    const float *hit_xyzi;   /* [n][4] sorted hits: x, y, z, event-local hit id (bits of an int32) */
    const float *hit_var;    /* [n][2] sorted hits: var_u, var_v */
    const uint32_t *bin_sub; /* [n_events * n_layers * n_bins][4]: bytes 0..14 = start of phi
                                sixteenths 1..15 of each bin relative to its first hit (all bytes
                                0xFF: the bin holds more than 255 hits) */
    const int32_t *pos_of_hit; /* [n] sorted position of hit id i */
    const int32_t *bin_off;  /* [n_events * n_layers * n_bins + 1] CSR offsets into the sorted hits;
                                bin (e, l, b) is [off[(e*L+l)*n_bins+b], off[(e*L+l)*n_bins+b+1]) */
    const float *var_max;    /* [n_events][n_layers][2] largest var_u, var_v of the layer */
    const int32_t *event_off; /* [n_events + 1] copy of the hits' event offsets */
    int32_t n, n_events, n_layers, n_bins;
} tkf_hit_index_view;

/* ---------------------------------------------------------------- context */

/* Fills `cfg` with the plain-building workload of the toy barrel: 10 cylinders at
 * 4, 8, ..., 40 cm, Bz = 3.8 T, x/X0 = 0.03 per layer, pion mass, 40 x 0.1 eta bins from
 * -2, 63 phi bins, chi2 < 30, 6 candidates, building from layer 3, FP32, seeds in input order. */
void tkf_default_config(tkf_config *cfg);

/* Creates a context on the current CUDA device.  The context owns its scratch memory. */
int tkf_create(const tkf_config *cfg, tkf_ctx **out);
int tkf_destroy(tkf_ctx *ctx);
const char *tkf_last_error(const tkf_ctx *ctx);
const char *tkf_status_string(int status);
/* Copies the context's configuration (with the autotuned seeds_per_block, if any). */
int tkf_get_config(const tkf_ctx *ctx, tkf_config *out);

/* ---------------------------------------------------------------- hot path */

/* Hit index (the hit-candidate data structure of Sec. 3.2.1): every hit is binned by
 * (event, layer, eta bin, phi bin), eta = asinh(z / radius[layer]) clamped to the bin range;
 * hits are reordered by (event, layer, eta bin, phi bin) into float4/float2 planes with CSR
 * bin offsets; inside a bin they are ordered by (phi sixteenth of the bin, hit id), and the
 * start of each sixteenth is recorded, so that a search window reads only the sixteenths it
 * overlaps.  *out: NULL to allocate a new index, or an index from an earlier call
 * whose storage is reused (grown if too small).  Library-owned until tkf_hit_index_free.
 * Errors: TKF_ERR_INVALID (bad sizes), TKF_ERR_NOMEM. */
int tkf_build_hit_index(tkf_ctx *ctx, const tkf_hits *hits, tkf_hit_index **out, tkf_stream stream);
int tkf_hit_index_free(tkf_hit_index *idx);
int tkf_hit_index_get_view(const tkf_hit_index *idx, tkf_hit_index_view *view);

/* Seed estimate (the seeding stage of Sec. 2): for each track, the state on layer 0 from its
 * hits on layers 0, 1, 2: curvature and charge from the circle through the three (x, y)
 * points, phi = tangent at the first hit, cot(theta) = dz / transverse arc, position = first
 * hit; covariance = diag(prior_sigma^2); chi2 = 0, nhits = 0; hit_idx rows 0..2 copied,
 * others -1 (when out->hit_idx is not NULL).
 *   seed_hits: device int32 [3][stride_in] hit ids, stride_in = out->stride.
 * Errors: TKF_ERR_INVALID. */
int tkf_seed_state(tkf_ctx *ctx, const tkf_hits *hits, const int32_t *seed_hits, tkf_tracks *out,
                   tkf_stream stream);

/* Track fit (Sec. 2: the KF applied without branching over a known hit list): each track
 * starts from `init` (a state on layer first_layer), gets the KF update with its hit on
 * first_layer, then for each layer up to last_layer: exact helix propagation to the cylinder
 * (with transport Jacobian), KF update with the hit (if any) in Joseph form, and the layer's
 * scattering noise (Highland width) unless the layer is the outermost one.  chi2 and nhits of
 * `init` are accumulated.  hit_idx: device int32 [n_layers][init->stride] (NULL: init->hit_idx).
 * `out` may alias `init`.  Failed tracks get nhits < 0 (enum tkf_track_status).
 * Errors: TKF_ERR_INVALID. */
int tkf_fit(tkf_ctx *ctx, const tkf_hits *hits, const tkf_tracks *init, const int32_t *hit_idx,
            int32_t first_layer, int32_t last_layer, tkf_tracks *out, tkf_stream stream);

/* The track fit of Sec. 2 continued: `init` lies on layer first_layer - 1 (as tkf_fit or tkf_seed_fit
 * leave it after that layer), so each track is propagated to first_layer before its first
 * update.  Fitting layers 0..k and then continuing over k+1..last gives the same result as one
 * fit over 0..last.  Errors: TKF_ERR_INVALID (also first_layer < 1). */
int tkf_fit_continue(tkf_ctx *ctx, const tkf_hits *hits, const tkf_tracks *init, const int32_t *hit_idx,
                     int32_t first_layer, int32_t last_layer, tkf_tracks *out, tkf_stream stream);

/* Seeding and fitting (Sec. 2): tkf_seed_state followed by tkf_fit over layers 0..last_layer
 * with the seed hits (rows 0..2 of seed_hits, no hit on later layers) in one kernel, without
 * storing the estimate: the seed fit of the batched pipeline.  seed_hits: device int32 [3][out->stride].  out gets the fitted
 * state, chi2, nhits and hit_idx (rows 0..2 the seed hits, others -1).  Seeds with a hit id out
 * of range get nhits = TKF_TRACK_SINGULAR and a zero state (and the kernel error bit).
 * Errors: TKF_ERR_INVALID. */
int tkf_seed_fit(tkf_ctx *ctx, const tkf_hits *hits, const int32_t *seed_hits, int32_t last_layer, tkf_tracks *out,
                 tkf_stream stream);

/* Cuts of the seeding from hit triplets (tkf_find_seeds); lengths in cm.  Defaults
 * (tkf_default_seed_cuts): pt_min 0.5 GeV, kappa_slack 0.15, z_vertex 4, d0_max 0.08,
 * dz_max 0.08, conf_rphi 0.1, conf_z 0.1, confirm 1. */
typedef struct {
    double pt_min;      /* curvature limit kappa_max = 0.00299792458 * bz / pt_min * (1 + kappa_slack) */
    double kappa_slack;
    double z_vertex;    /* |z at r = 0| of the r-z line through the layer-0 and layer-1 hits */
    double d0_max;      /* |power of the beam line point (x = y = 0) / diameter| of the triplet circle */
    double dz_max;      /* |z of the layer-2 hit - the r-z line through the first two, at its r| */
    double conf_rphi;   /* |signed distance of the layer-3 hit from the triplet circle| */
    double conf_z;      /* |z of the layer-3 hit - the r-z line through the layer-1 and layer-2 hits| */
    int32_t confirm;    /* 1: a seed needs a confirmation hit on layer 3 */
    int32_t reserved;
} tkf_seed_cuts;

void tkf_default_seed_cuts(tkf_seed_cuts *cuts);

/* Seeding from hit triplets (the seeding stage of Sec. 2, which the paper names without
 * specifying it): for every hit a of layer 0, the triplet (a, b, c) of hits on layers 0, 1, 2 of
 * smallest score that passes every cut -- transverse chords |b - a| <= 2 (R1 - R0) and
 * |c - b| <= 2 (R2 - R1) (outward, not a looping circle's far crossing); |curvature| <= kappa_max
 * for the circle through the beam line point, a and b, and for the circle through a, b, c; the
 * z-vertex, d0 and dz cuts of tkf_seed_cuts -- and, with confirm, a layer-3 hit e with
 * |e - c| <= 2 (R3 - R2) inside the conf_rphi / conf_z cuts.  Score = (d0 / d0_max)^2 +
 * (dz / dz_max)^2 + the smallest (f / conf_rphi)^2 + (dz3 / conf_z)^2 of its confirming hits;
 * equal scores keep the smallest event-local hit ids (b first).  r of a hit is its transverse
 * radius.  Layers 0..3 must be cylinders of increasing radius.  The search walks the index's
 * eta-phi bins around each pair's and triplet's extrapolation and applies the exact cuts to
 * every hit there, so the result equals a scan over all hits of the layers (up to the FP32
 * evaluation of quantities within about 1e-4 of a cut).
 *   idx: a hit index of this context (tkf_build_hit_index).
 *   seed_hits: device int32 [3][max_seeds]: global hit ids (into the indexed tkf_hits) of a, b, c,
 *              the layout tkf_seed_fit and tkf_pipeline_run take.
 *   seed_event: device int32 [max_seeds], the event of each seed.
 *   seed_score: device float [max_seeds] or NULL.
 *   n_found: device int32 [1]: the number of seeds found, which may exceed max_seeds (then only
 *            the first max_seeds are written).
 * Seeds are ordered by event, then by the index position of their layer-0 hit (eta bin, phi
 * bin, phi sixteenth, hit id).  Scratch (12 bytes per indexed hit) is held by the context.
 * Errors: TKF_ERR_INVALID (null pointers, cuts not positive, fewer than 4 layers, a disk among
 * layers 0..3, an index binned by another configuration), TKF_ERR_NOMEM, TKF_ERR_CUDA. */
int tkf_find_seeds(tkf_ctx *ctx, const tkf_hit_index *idx, const tkf_seed_cuts *cuts, int32_t max_seeds,
                   int32_t *seed_hits, int32_t *seed_event, float *seed_score, int32_t *n_found, tkf_stream stream);

/* Backward pass of the final fit (Sec. 2: the final fit gives the best estimate of the track's
 * parameters; this pass carries that estimate to the production point): an inward Kalman
 * filter over each track's hits from layer last_layer down to first_layer.  `init` holds the
 * states on layer last_layer (typically tkf_fit's output over 0..last_layer); their covariance
 * is multiplied by cov_scale (> 0; a large factor such as 1e4 discounts the forward fit's
 * information, so the pass is nearly an independent fit in the opposite direction).  Then, per
 * layer from last_layer inward: the Kalman update with the layer's hit (hit_idx as for tkf_fit;
 * -1 = none), the layer's scattering material, and the propagation to the next smaller
 * cylinder (the outward propagation of the reversed track: same helix, opposite direction).
 * `out` receives the states on first_layer after its update and material -- on layer 0, the
 * track as it left the production region -- with this pass's chi2 and hit count (nhits < 0:
 * enum tkf_track_status, also for inputs with nhits < 0).  hit_idx null: init->hit_idx.
 * Errors: TKF_ERR_INVALID (also last_layer < first_layer, cov_scale not positive or finite). */
int tkf_fit_backward(tkf_ctx *ctx, const tkf_hits *hits, const tkf_tracks *init, const int32_t *hit_idx,
                     int32_t last_layer, int32_t first_layer, double cov_scale, tkf_tracks *out, tkf_stream stream);

/* Combinatorial track building (Sec. 2, Sec. 3.2): each seed (a state on layer
 * first_build_layer - 1, with chi2, nhits and the hit ids of the seeding layers) is extended
 * outward layer by layer: every candidate is propagated to the next cylinder, every hit of
 * the eta-phi window around it with chi2 < chi2_cut (on the same half of the cylinder) makes
 * a branch, a candidate without any makes one hole branch, the branches of the seed are
 * ranked by (nHits desc, chi2 asc, parent rank asc, hit id asc) and the best n_cand are kept,
 * updated by the KF and given the layer's scattering noise.  One persistent launch over all
 * seeds of all events (tiles of seeds_per_block seeds pulled from an atomic counter), after a
 * launch that scans the first building layer one lane per seed (every seed enters it with a
 * single candidate) into branch lists held in the context (2 x 4 bytes per seed and candidate
 * slot, allocated on first use and grown when a call has more seeds; a pipeline reserves them).
 *   out: best candidate per seed (out->stride >= seeds->n).
 *   out_all: NULL, or every final candidate: candidate r of seed s at s * n_cand + r
 *            (stride >= seeds->n * n_cand); n_cand_out (device int32 [seeds->n], may be NULL)
 *            receives the number of candidates of each seed.
 * Errors: TKF_ERR_INVALID; per seed nhits = TKF_TRACK_LOST (state, covariance, chi2 zero) when
 * every candidate was lost or the seed's event is out of range. */
int tkf_build_tracks(tkf_ctx *ctx, const tkf_hit_index *idx, const tkf_tracks *seeds, tkf_tracks *out,
                     tkf_tracks *out_all, int32_t *n_cand_out, tkf_stream stream);

/* Waits for `stream` and reports errors raised by kernels of this context since the last
 * call (TKF_ERR_KERNEL with text in tkf_last_error), or a CUDA error (TKF_ERR_CUDA). */
int tkf_sync_status(tkf_ctx *ctx, tkf_stream stream);

/* ---------------------------------------------------------------- batched pipeline */

typedef struct tkf_pipeline tkf_pipeline;

/* A reusable pipeline for batches of up to max_hits hits, max_events events and max_tracks
 * seeds: the whole chain of Sec. 2 -- hit index, seed estimate, KF fit of the seeding layers,
 * combinatorial building, final KF fit of the built hit lists -- over every event of a batch
 * at once (the multi-event packing of Sec. 4, with the building kernel's dynamic work tiles
 * standing for the TBB work stealing of Sec. 2.3).  All buffers (hit index, the track sets)
 * are allocated here or by tkf_pipeline_set_backward, so a run allocates nothing.  With
 * use_graph != 0 the first run with a given input signature (hit pointers and sizes, seed pointers, n_tracks) is captured into a
 * CUDA graph on the pipeline's own stream and replayed by every later run with the same
 * signature (one cudaGraphLaunch); another signature re-captures.
 * Errors: TKF_ERR_INVALID, TKF_ERR_NOMEM, TKF_ERR_CUDA. */
int tkf_pipeline_create(tkf_ctx *ctx, int32_t max_hits, int32_t max_events, int32_t max_tracks, int32_t use_graph,
                        tkf_pipeline **out);
int tkf_pipeline_destroy(tkf_pipeline *p);

/* One pass over a batch, queued on `stream`.  seed_hits: device int32 [3][max_tracks] hit ids
 * of each seed on layers 0..2; seed_event: device int32 [n_tracks] event of each seed.  The
 * results stay in pipeline-owned track sets (tkf_pipeline_outputs), valid until the next run.
 * Errors: TKF_ERR_INVALID (batch larger than the creation sizes), TKF_ERR_CUDA. */
int tkf_pipeline_run(tkf_pipeline *p, const tkf_hits *hits, const int32_t *seed_hits, const int32_t *seed_event,
                     int32_t n_tracks, tkf_stream stream);

/* Views of the pipeline's track sets of the last run (stride = max_tracks; any may be NULL):
 * `seeds` = states after the seeding layers (with their event ids), `built` = best candidate
 * per seed after building, `fitted` = its final fit (hit_idx = the built hit list). */
int tkf_pipeline_outputs(const tkf_pipeline *p, tkf_tracks *seeds, tkf_tracks *built, tkf_tracks *fitted);

/* Adds (cov_scale > 0) or removes (0) a last stage to every following run: the backward pass
 * of the final fit (tkf_fit_backward from the fitted states on the outermost layer to layer 0,
 * with this covariance scale) into a fifth, pipeline-owned track set; the next run captures
 * its graph again.  The first enabling call allocates that set.
 * Errors: TKF_ERR_INVALID (cov_scale negative or not finite), TKF_ERR_NOMEM, TKF_ERR_CUDA. */
int tkf_pipeline_set_backward(tkf_pipeline *p, double cov_scale);

/* View of the backward pass's track set of the last run (states on layer 0; hit_idx = the
 * built hit list).  Errors: TKF_ERR_INVALID (no backward stage set). */
int tkf_pipeline_backward_outputs(const tkf_pipeline *p, tkf_tracks *out);

/* Number of graph captures so far (replays do not count); -1 for a null pipeline. */
int tkf_pipeline_captures(const tkf_pipeline *p);

/* The pipeline's hit index (valid after a run; owned by the pipeline). */
const tkf_hit_index *tkf_pipeline_index(const tkf_pipeline *p);

/* Milliseconds between CUDA events recorded just before and after tkf_build_tracks in the last
 * run (the seed ordering, the first-layer scan and the building kernel; event-record nodes
 * inside the graph); waits for the second event only.
 * Errors: TKF_ERR_INVALID (no run yet), TKF_ERR_CUDA. */
int tkf_pipeline_build_ms(tkf_pipeline *p, float *ms);

/* Work-tile autotuner of the building kernel (the paper tunes its TBB task size against tail
 * effects, Sec. 2.3): times `repeats` launches of tkf_build_tracks for each tile size in
 * tiles[0..n_tiles) (seeds pulled per warp), writes the mean milliseconds to ms_out (may be
 * NULL), keeps the fastest in the context's seeds_per_block and returns it in *best.
 * Synchronises `stream`.  Errors: TKF_ERR_INVALID, TKF_ERR_CUDA. */
int tkf_autotune_build(tkf_ctx *ctx, const tkf_hit_index *idx, const tkf_tracks *seeds, tkf_tracks *out,
                       const int32_t *tiles, int32_t n_tiles, int32_t repeats, float *ms_out, int32_t *best,
                       tkf_stream stream);

/* ---------------------------------------------------------------- serving loop */

/* A trigger-like request loop over the pipeline (the paper's GPU port found host set-up
 * copies dominating, Sec. 5; here events stream in while earlier ones run).  Events are
 * submitted one at a time and wait in a host queue bounded by queue_bytes; a worker thread
 * packs every queued event that fits into the next free slot and launches it while other
 * slots still run (continuous batching).  Each slot owns a context, a pipeline and device
 * buffers for max_batch_events / max_batch_hits / max_batch_tracks, allocated at creation, so
 * the device memory in use is fixed by those limits (events are admitted into a batch only if
 * they fit its buffers).  Results land in pinned host buffers drawn from a pool bounded by
 * result_bytes; while unreleased results hold all of it, no new batch starts (the queue then
 * fills and submissions get TKF_ERR_AGAIN), so callers release results promptly.  The pool
 * starts with one full-size buffer per slot, made at creation (pinned allocation can wait for
 * the device); a batch takes the smallest free buffer that holds it, and new buffers are made
 * only while more results are held than the pool has buffers.  Results of
 * an event do not depend on the batch it ran in. */
typedef struct tkf_server tkf_server;

typedef struct {
    int32_t n_slots;          /* batches in flight at once */
    int32_t max_batch_events; /* events per batch */
    int32_t max_batch_hits;   /* hits per batch (also the largest event accepted) */
    int32_t max_batch_tracks; /* seeds per batch (also the largest event accepted) */
    size_t queue_bytes;       /* host bytes of submitted, not yet launched events */
    size_t result_bytes;      /* pinned host bytes for results; at least one full batch,
                                 max_batch_tracks * (29 + n_layers) * 4 */
} tkf_server_options;

/* One event in host memory: hit planes of length n_hits and seed_hits [3][n_seeds], the
 * event-local hit ids of each seed on layers 0, 1, 2.  borrow = 0: tkf_submit_event copies the
 * arrays (the caller may free them on return).  borrow = 1: the server reads them in place --
 * the hit planes straight into device memory, fastest from pinned memory -- so the caller
 * keeps them alive and unchanged until tkf_poll reports the event done (for an event released
 * before that, until tkf_server_destroy returns). */
typedef struct {
    const float *x, *y, *z, *var_u, *var_v;
    const int32_t *layer;
    int32_t n_hits;
    const int32_t *seed_hits;
    int32_t n_seeds;
    int32_t borrow;
} tkf_event;

/* Result of one event (pinned host memory owned by the server, valid until tkf_release): the
 * final fit of the best built candidate of every seed -- par [6][stride], cov [21][stride],
 * chi2, nhits, first n_tracks columns -- and its hit ids [n_layers][stride] (event-local,
 * -1 = hole); timestamps (steady clock, ns) of submission, batch launch and completion; and
 * the device interval of the event's batch, from before its first input copy to after its
 * last result copy on the slot's stream (CUDA event times in ms since the server's creation,
 * -1 if unavailable): two batches whose intervals intersect were in flight on the GPU at once. */
typedef struct {
    int32_t status, n_tracks, stride;
    const float *par, *cov, *chi2;
    const int32_t *nhits, *hit_idx;
    int64_t t_submit_ns, t_start_ns, t_done_ns;
    float gpu_start_ms, gpu_done_ms;
    float gpu_inputs_ms, gpu_results_ms; /* same clock: inputs copied in; kernels done (results start back) */
} tkf_result;

typedef struct {
    int64_t submitted, rejected, events_done, tracks_done, batches, max_batch_events;
    int64_t result_allocs; /* pinned result buffers allocated so far (each takes milliseconds) */
} tkf_server_stats;

/* Defaults: 3 slots, 64 events, 4 Mi hits and 256 Ki seeds per batch, 1 GiB host queue,
 * 1 GiB of pinned result memory. */
void tkf_server_default_options(tkf_server_options *opt);

/* Creates the server on the current device (precision FP32 or MIXED) and starts its worker.
 * Errors: TKF_ERR_INVALID (bad options, result_bytes below one batch), TKF_ERR_NOMEM,
 * TKF_ERR_CUDA. */
int tkf_server_create(const tkf_config *cfg, const tkf_server_options *opt, tkf_server **out);
/* Stops the worker after the batches in flight finish, and frees everything (results not yet
 * released included).  No other call on this server may overlap or follow it. */
int tkf_server_destroy(tkf_server *server);

/* Non-blocking submission.  Errors: TKF_ERR_AGAIN (host queue full: retry later),
 * TKF_ERR_INVALID (malformed event, or larger than a batch), a worker's earlier error. */
int tkf_submit_event(tkf_server *server, const tkf_event *event, uint64_t *ticket);

/* Result of `ticket`: waits up to timeout_us microseconds (0: do not wait).
 * Errors: TKF_ERR_NOTREADY (timeout_us = 0 and not done), TKF_ERR_TIMEOUT, TKF_ERR_INVALID
 * (unknown or released ticket). */
int tkf_poll(tkf_server *server, uint64_t ticket, tkf_result *result, int64_t timeout_us);

/* Frees the result of `ticket` (its pointers become invalid; its share of the result memory
 * returns to the pool once every event of its batch is released). */
int tkf_release(tkf_server *server, uint64_t ticket);

int tkf_server_get_stats(tkf_server *server, tkf_server_stats *out);

/* Batch forms for clients that move many events per call.  tkf_submit_events submits
 * events[0..n) in order, each as its own arrival (the worker may start a batch with the first
 * events while the rest are queued), and stops at the first refusal: returns that status
 * (TKF_ERR_AGAIN: queue full; TKF_ERR_INVALID: a malformed event) with *n_accepted events
 * accepted and their tickets in tickets[0..*n_accepted).  tkf_wait_all fills results[k] for tickets[k], waiting up to
 * timeout_us in total (0: do not wait); it returns the first error (TKF_ERR_TIMEOUT,
 * TKF_ERR_NOTREADY, TKF_ERR_INVALID), the results before it being filled.  tkf_release_many
 * releases every ticket given and returns the first error. */
int tkf_submit_events(tkf_server *server, const tkf_event *events, int32_t n, uint64_t *tickets,
                      int32_t *n_accepted);
int tkf_wait_all(tkf_server *server, const uint64_t *tickets, int32_t n, tkf_result *results, int64_t timeout_us);
int tkf_release_many(tkf_server *server, const uint64_t *tickets, int32_t n);

/* ---------------------------------------------------------------- allocation-free variant */

/* Caller-owned output arrays of tkf_build_hit_index_noalloc (device memory), laid out as in
 * tkf_hit_index_view: hit_xyzi [n][4], hit_var [n][2], bin_sub [n_events * n_layers * n_bins][4],
 * pos_of_hit [n],
 * bin_off [n_events * n_layers * n_bins + 1], var_max [n_events * n_layers][2],
 * event_off [n_events + 1], with n_bins = n_eta_bins * n_phi_bins. */
typedef struct {
    float *hit_xyzi, *hit_var;
    uint32_t *bin_sub;
    int32_t *pos_of_hit, *bin_off;
    float *var_max;
    int32_t *event_off;
} tkf_hit_index_out;

/* Capacity of the fixed scratch of tkf_build_hit_index_noalloc. */
#define TKF_NOALLOC_MAX_HITS (1 << 20)      /* hits per call */
#define TKF_NOALLOC_MAX_BINS (1 << 18)      /* n_events * n_layers * n_eta_bins * n_phi_bins */
#define TKF_NOALLOC_MAX_SEGMENTS 4096       /* n_events * n_layers */

/* The same hit index as tkf_build_hit_index, written into caller-owned arrays, for callers
 * that cannot allocate device memory: code running where cudaMalloc is not allowed or not
 * wanted (inside another framework's memory pool, in a process whose device memory is fully
 * reserved up front, or where an allocation could block or fail in the middle of a time-
 * critical trigger path).  The paper has no counterpart; this is an interface addition.
 *
 * It allocates nothing: no cudaMalloc, cudaFree or allocating library call, and it needs no
 * tkf_ctx.  Its temporary work space is one fixed array in the library's own device memory
 * (TKF_NOALLOC_MAX_HITS + TKF_NOALLOC_MAX_BINS + 2 * TKF_NOALLOC_MAX_SEGMENTS int32, about
 * 5 MB), which every GPU that loads libtkf.so keeps until the process exits.  Inputs larger
 * than that capacity are rejected with TKF_ERR_TOO_LARGE before any work is queued.
 *
 * The first call on a device looks up the device address of that array (with that device
 * current) and keeps it for the life of the process; make that first call before capturing a
 * stream into a CUDA graph.  The kept address belongs to the device's primary context: after
 * cudaDeviceReset (or any reset of that context) it no longer points at the array, so a
 * process that resets a device must not call this function on it again.  All calls share the
 * one array and each call clears the counters that must start at zero, so calls may follow
 * each other freely on one stream, but calls whose work overlaps on the GPU (other streams,
 * other host threads) race on it and must be serialised by the caller.  The array also holds
 * an error word that the kernels set (a hit layer out of range) but that is never cleared nor
 * read: kernel-side errors are not reported, so validate inputs beforehand.
 * Errors: TKF_ERR_INVALID (bad configuration or arguments), TKF_ERR_TOO_LARGE, TKF_ERR_CUDA. */
int tkf_build_hit_index_noalloc(const tkf_config *cfg, const tkf_hits *hits, const tkf_hit_index_out *out,
                                tkf_stream stream);

/* ---------------------------------------------------------------- diagnostics */

/* Measures the arithmetic throughput of the current device's SMs, the denominators of the
 * rooflines of the ALU-bound kernels: FP32 and FP64 fused multiply-add (TFLOP/s, 2 per FMA) and
 * the special-function unit (__sinf, tera-operations/s).  Each probe runs independent
 * dependency chains in 2048 threads per SM for about a millisecond; the best of three timed
 * launches (after an untimed one) on `stream` is reported.  Synchronous: it returns after the
 * last probe.  Errors: TKF_ERR_INVALID (a null output), TKF_ERR_NOMEM, TKF_ERR_CUDA. */
int tkf_probe_alu(tkf_stream stream, double *fp32_tflops, double *fp64_tflops, double *sfu_tops);

#ifdef __cplusplus
}
#endif
#endif
