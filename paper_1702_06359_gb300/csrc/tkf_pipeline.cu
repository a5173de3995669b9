// tkf_pipeline: the whole hot path on a batch of events (Sec. 2: seeding, building, final fit)
// as one reusable object -- buffers sized once for the largest batch, the sequence of kernels
// captured into a CUDA graph and replayed -- and the work-tile autotuner of the build kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace {

struct Buf {
    void *par = nullptr, *cov = nullptr, *chi2 = nullptr;
    int *nhits = nullptr, *hit_idx = nullptr, *event = nullptr;
};

void free_buf(Buf &b)
{
    cudaFree(b.par);
    cudaFree(b.cov);
    cudaFree(b.chi2);
    cudaFree(b.nhits);
    cudaFree(b.hit_idx);
    cudaFree(b.event);
    b = Buf();
}

cudaError_t alloc_buf(Buf &b, int n, int L, size_t es)
{
    cudaError_t e;
    const size_t nn = std::max(n, 1);
    if ((e = cudaMalloc(&b.par, 6 * nn * es)) || (e = cudaMalloc(&b.cov, 21 * nn * es)) ||
        (e = cudaMalloc(&b.chi2, nn * es)) || (e = cudaMalloc((void **)&b.nhits, nn * sizeof(int))) ||
        (e = cudaMalloc((void **)&b.hit_idx, L * nn * sizeof(int))) || (e = cudaMalloc((void **)&b.event, nn * sizeof(int))))
        return e;
    return cudaMemset(b.hit_idx, 0xff, L * nn * sizeof(int));
}

tkf_tracks view(const Buf &b, int n, int stride)
{
    tkf_tracks t;
    t.par = b.par;
    t.cov = b.cov;
    t.chi2 = b.chi2;
    t.nhits = b.nhits;
    t.hit_idx = b.hit_idx;
    t.event = b.event;
    t.n = n;
    t.stride = stride;
    return t;
}

struct Signature {
    tkf_hits hits;
    const int32_t *seed_hits, *seed_event;
    int32_t n_tracks, tile;
    double back_scale;
    bool operator==(const Signature &o) const { return std::memcmp(this, &o, sizeof *this) == 0; }
};

}  // namespace

struct tkf_pipeline {
    tkf_ctx *ctx = nullptr;
    int max_hits = 0, max_events = 0, max_tracks = 0, use_graph = 1;
    tkf_hit_index *idx = nullptr;
    Buf seeds, built, final_, back;
    double back_scale = 0.0;  // > 0: the step ends with the backward pass (covariance scale)
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Signature sig{};
    bool have_sig = false;
    int captures = 0;
    cudaEvent_t build_ev[2] = {nullptr, nullptr};  // around the building kernel of the last run
    bool timed = false;
};

namespace {

int fail(tkf_ctx *ctx, int code, const std::string &m)
{
    ctx->err = m;
    return code;
}

// the step: index -> seed estimate and seed fit (layers 0..first-1, one kernel) -> build ->
// final fit (layers first..L-1, continuing the seed fit)
int issue(tkf_pipeline *p, const tkf_hits *hits, const int32_t *seed_hits, const int32_t *seed_event, int n,
          cudaStream_t s, bool capturing)
{
    tkf_ctx *ctx = p->ctx;
    const int L = ctx->cfg.n_layers, first = ctx->cfg.first_build_layer, stride = p->max_tracks;
    int st = tkf_build_hit_index(ctx, hits, &p->idx, (tkf_stream)s);
    if (st) return st;
    tkf_tracks seeds = view(p->seeds, n, stride), built = view(p->built, n, stride),
               fin = view(p->final_, n, stride);
    seeds.event = const_cast<int32_t *>(seed_event);
    if ((st = tkf::seed_and_fit(ctx, hits, seed_hits, first - 1, &seeds, (tkf_stream)s))) return st;
    // events around the building kernel (event-record nodes when captured into the graph)
    const unsigned flag = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (cudaEventRecordWithFlags(p->build_ev[0], s, flag) != cudaSuccess)
        return fail(ctx, TKF_ERR_CUDA, "pipeline: cudaEventRecord");
    if ((st = tkf_build_tracks(ctx, p->idx, &seeds, &built, nullptr, nullptr, (tkf_stream)s))) return st;
    if (cudaEventRecordWithFlags(p->build_ev[1], s, flag) != cudaSuccess)
        return fail(ctx, TKF_ERR_CUDA, "pipeline: cudaEventRecord");
    // final fit of the built hit list: layers 0..first-1 carry the seed's hits, so the seed fit
    // already holds its state there (bit for bit); the fit continues from it on layer first
    if ((st = tkf::fit_tracks(ctx, hits, &seeds, built.hit_idx, first, L - 1, &fin, (tkf_stream)s, true))) return st;
    if (!(p->back_scale > 0.0)) return TKF_OK;
    // optional: the final fit's backward pass to the innermost layer
    tkf_tracks bk = view(p->back, n, stride);
    return tkf::fit_backward(ctx, hits, &fin, built.hit_idx, L - 1, 0, p->back_scale, &bk, (tkf_stream)s);
}

}  // namespace

extern "C" {

int tkf_pipeline_create(tkf_ctx *ctx, int32_t max_hits, int32_t max_events, int32_t max_tracks, int32_t use_graph,
                        tkf_pipeline **out)
{
    if (!ctx || !out || max_hits < 1 || max_events < 1 || max_tracks < 1) return TKF_ERR_INVALID;
    *out = nullptr;
    tkf_pipeline *p = new (std::nothrow) tkf_pipeline();
    if (!p) return TKF_ERR_NOMEM;
    p->ctx = ctx;
    p->max_hits = max_hits;
    p->max_events = max_events;
    p->max_tracks = max_tracks;
    p->use_graph = use_graph ? 1 : 0;
    const int L = ctx->cfg.n_layers;
    const size_t es = ctx->cfg.precision == TKF_FP64 ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaSuccess;
    for (Buf *b : {&p->seeds, &p->built, &p->final_})
        if (e == cudaSuccess) e = alloc_buf(*b, max_tracks, L, es);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&p->build_ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&p->build_ev[1]);
    int st = e == cudaSuccess ? TKF_OK : (e == cudaErrorMemoryAllocation ? TKF_ERR_NOMEM : TKF_ERR_CUDA);
    if (!st) st = tkf::hit_index_reserve(ctx, &p->idx, (size_t)max_hits, (size_t)max_events);  // no later allocation
    if (!st && ctx->cfg.seed_order) st = tkf::seed_order_reserve(ctx, (size_t)max_tracks, (size_t)max_events);
    if (!st) st = tkf::first_list_reserve(ctx, (size_t)max_tracks);
    if (st) {
        tkf_pipeline_destroy(p);
        return st;
    }
    *out = p;
    return TKF_OK;
}

int tkf_pipeline_destroy(tkf_pipeline *p)
{
    if (!p) return TKF_ERR_INVALID;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->capture) cudaStreamDestroy(p->capture);
    for (cudaEvent_t ev : p->build_ev)
        if (ev) cudaEventDestroy(ev);
    if (p->idx) tkf_hit_index_free(p->idx);
    for (Buf *b : {&p->seeds, &p->built, &p->final_, &p->back}) free_buf(*b);
    delete p;
    return TKF_OK;
}

int tkf_pipeline_run(tkf_pipeline *p, const tkf_hits *hits, const int32_t *seed_hits, const int32_t *seed_event,
                     int32_t n_tracks, tkf_stream stream)
{
    if (!p || !hits || (n_tracks > 0 && (!seed_hits || !seed_event))) return TKF_ERR_INVALID;
    tkf_ctx *ctx = p->ctx;
    if (n_tracks < 0 || n_tracks > p->max_tracks || hits->n > p->max_hits || hits->n_events > p->max_events)
        return fail(ctx, TKF_ERR_INVALID, "pipeline: batch larger than the sizes given at creation");
    cudaStream_t s = (cudaStream_t)stream;
    p->timed = true;
    if (!p->use_graph) return issue(p, hits, seed_hits, seed_event, n_tracks, s, false);
    Signature sig{};
    sig.hits = *hits;
    sig.seed_hits = seed_hits;
    sig.seed_event = seed_event;
    sig.n_tracks = n_tracks;
    sig.tile = ctx->cfg.seeds_per_block;
    sig.back_scale = p->back_scale;
    if (!p->have_sig || !(sig == p->sig)) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        p->exec = nullptr;
        p->graph = nullptr;
        p->have_sig = false;
        // capture on the pipeline's own stream (the caller's may be the legacy default stream)
        if (cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fail(ctx, TKF_ERR_CUDA, "pipeline: cudaStreamBeginCapture failed");
        const int st = issue(p, hits, seed_hits, seed_event, n_tracks, p->capture, true);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p->capture, &g);
        if (st || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return st ? st : fail(ctx, TKF_ERR_CUDA, std::string("pipeline: capture failed: ") + cudaGetErrorString(e));
        }
        if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            return fail(ctx, TKF_ERR_CUDA, "pipeline: cudaGraphInstantiate failed");
        }
        p->graph = g;
        p->sig = sig;
        p->have_sig = true;
        p->captures += 1;
    }
    const cudaError_t e = cudaGraphLaunch(p->exec, s);
    if (e != cudaSuccess) return fail(ctx, TKF_ERR_CUDA, std::string("pipeline: cudaGraphLaunch: ") + cudaGetErrorString(e));
    return TKF_OK;
}

int tkf_pipeline_outputs(const tkf_pipeline *p, tkf_tracks *seeds, tkf_tracks *built, tkf_tracks *fitted)
{
    if (!p) return TKF_ERR_INVALID;
    const int n = p->have_sig ? p->sig.n_tracks : p->max_tracks;
    if (seeds) {
        *seeds = view(p->seeds, n, p->max_tracks);
        if (p->have_sig) seeds->event = const_cast<int32_t *>(p->sig.seed_event);
    }
    if (built) *built = view(p->built, n, p->max_tracks);
    if (fitted) {
        *fitted = view(p->final_, n, p->max_tracks);
        fitted->hit_idx = p->built.hit_idx;  // the final fit uses the built hit list
    }
    return TKF_OK;
}

int tkf_pipeline_set_backward(tkf_pipeline *p, double cov_scale)
{
    if (!p) return TKF_ERR_INVALID;
    if (!(cov_scale >= 0.0) || !std::isfinite(cov_scale))
        return fail(p->ctx, TKF_ERR_INVALID, "pipeline: cov_scale must be >= 0 and finite");
    if (cov_scale > 0.0 && !p->back.par) {
        const size_t es = p->ctx->cfg.precision == TKF_FP64 ? sizeof(double) : sizeof(float);
        const cudaError_t e = alloc_buf(p->back, p->max_tracks, p->ctx->cfg.n_layers, es);
        if (e != cudaSuccess) {
            free_buf(p->back);
            return fail(p->ctx, e == cudaErrorMemoryAllocation ? TKF_ERR_NOMEM : TKF_ERR_CUDA,
                        "pipeline: backward buffers");
        }
    }
    p->back_scale = cov_scale;  // a graph captured with another setting is captured again
    return TKF_OK;
}

int tkf_pipeline_backward_outputs(const tkf_pipeline *p, tkf_tracks *out)
{
    if (!p || !out || !(p->back_scale > 0.0)) return TKF_ERR_INVALID;
    const int n = p->have_sig ? p->sig.n_tracks : p->max_tracks;
    *out = view(p->back, n, p->max_tracks);
    out->hit_idx = p->built.hit_idx;
    return TKF_OK;
}

int tkf_pipeline_captures(const tkf_pipeline *p) { return p ? p->captures : -1; }

const tkf_hit_index *tkf_pipeline_index(const tkf_pipeline *p) { return p ? p->idx : nullptr; }

int tkf_pipeline_build_ms(tkf_pipeline *p, float *ms)
{
    if (!p || !ms || !p->timed) return TKF_ERR_INVALID;
    if (cudaEventSynchronize(p->build_ev[1]) != cudaSuccess) return fail(p->ctx, TKF_ERR_CUDA, "pipeline: event sync");
    if (cudaEventElapsedTime(ms, p->build_ev[0], p->build_ev[1]) != cudaSuccess)
        return fail(p->ctx, TKF_ERR_CUDA, "pipeline: cudaEventElapsedTime");
    return TKF_OK;
}

int tkf_autotune_build(tkf_ctx *ctx, const tkf_hit_index *idx, const tkf_tracks *seeds, tkf_tracks *out,
                       const int32_t *tiles, int32_t n_tiles, int32_t repeats, float *ms_out, int32_t *best,
                       tkf_stream stream)
{
    if (!ctx || !idx || !seeds || !out || !tiles || n_tiles < 1 || repeats < 1) return TKF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return fail(ctx, TKF_ERR_CUDA, "autotune: cudaEventCreate");
    const int saved = ctx->cfg.seeds_per_block;
    float best_ms = 0.f;
    int best_tile = -1, st = TKF_OK;
    for (int k = 0; k < n_tiles && !st; ++k) {
        if (tiles[k] < 1) { st = fail(ctx, TKF_ERR_INVALID, "autotune: tile sizes must be positive"); break; }
        ctx->cfg.seeds_per_block = tiles[k];
        st = tkf_build_tracks(ctx, idx, seeds, out, nullptr, nullptr, stream);  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < repeats && !st; ++r) st = tkf_build_tracks(ctx, idx, seeds, out, nullptr, nullptr, stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(ctx, TKF_ERR_CUDA, "autotune: event sync"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= repeats;
        if (ms_out) ms_out[k] = ms;
        if (best_tile < 0 || ms < best_ms) {
            best_ms = ms;
            best_tile = tiles[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->cfg.seeds_per_block = st ? saved : best_tile;
    if (best) *best = st ? saved : best_tile;
    return st;
}

}  // extern "C"
