// tkf_server: a trigger-like serving loop over the tracking pipeline.  Events arrive one at a
// time (tkf_submit_event), wait in a bounded host queue, and a worker thread packs every
// queued event that fits into the next free slot -- a slot owns a context, a pipeline and
// device buffers sized at creation, so device memory is bounded up front -- and launches it
// on the slot's stream while other slots are still running (continuous batching: arrivals
// join the next batch as soon as a slot frees up).  Completion is observed with CUDA events;
// each event's tracks are copied out with its submit/start/done timestamps (tkf_poll).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Pending {
    uint64_t ticket;
    std::vector<float> x, y, z, vu, vv;  // owned copies (borrow = 0)
    std::vector<int> layer, seeds;       // seeds: [3][n_seeds] event-local hit ids
    const float *bx = nullptr, *by = nullptr, *bz = nullptr, *bvu = nullptr, *bvv = nullptr;
    const int *blayer = nullptr, *bseeds = nullptr;  // the caller's arrays (borrow = 1)
    bool borrowed = false;
    int n_hits, n_seeds;
    int64_t t_submit;
    size_t bytes;
    const float *px() const { return borrowed ? bx : x.data(); }
    const float *py() const { return borrowed ? by : y.data(); }
    const float *pz() const { return borrowed ? bz : z.data(); }
    const float *pvu() const { return borrowed ? bvu : vu.data(); }
    const float *pvv() const { return borrowed ? bvv : vv.data(); }
    const int *player() const { return borrowed ? blayer : layer.data(); }
    const int *pseeds() const { return borrowed ? bseeds : seeds.data(); }
};

// Pinned host memory receiving one batch's results (planes of `cap` tracks), shared by that
// batch's events until the last of them is released, then reused by a later batch.
struct OutBuf {
    float *par = nullptr, *cov = nullptr, *chi2 = nullptr;
    int *nhits = nullptr, *hit = nullptr;
    int cap = 0;
    size_t bytes = 0;
    int refs = 0;
};

struct Done {
    OutBuf *buf = nullptr;  // results at column trk0 of the batch's planes (stride buf->cap)
    int trk0 = 0;
    int64_t t_submit = 0, t_start = 0, t_done = 0;
    float gpu_start_ms = 0.f, gpu_done_ms = 0.f;  // the batch's device interval (server clock)
    float gpu_inputs_ms = 0.f, gpu_results_ms = 0.f;  // inputs on the device; results start back
    int status = TKF_OK;
    int n = 0;
    bool done = false;
};

template <class T> struct Pinned {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count)
    {
        n = count;
        return cudaMallocHost((void **)&p, std::max<size_t>(count, 1) * sizeof(T));
    }
    void free()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
    }
};

struct EvInfo {
    uint64_t ticket;
    int hit0, n_hits, trk0, n_tracks;
    int64_t t_submit;
};

struct Slot {
    tkf_ctx *ctx = nullptr;
    tkf_pipeline *pipe = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t t_begin = nullptr, t_end = nullptr;  // timed: the batch's first and last device work
    cudaEvent_t t_in = nullptr, t_out = nullptr;     // timed: inputs copied; kernels done
    // host staging (pinned) for copied events, and the per-batch event offsets
    Pinned<float> hx, hy, hz, hvu, hvv;
    Pinned<int> hlayer, hraw, hoff, htoff;
    // device inputs: hit planes, the events' seed blocks as submitted ([3][n] event-local ids
    // per event, back to back), hit and seed offsets of the events; seed ids of the batch
    // ([3][T], batch hit ids) and seed events made from them on the device; event-local hit
    // ids of the built tracks ([L][T])
    float *dx = nullptr, *dy = nullptr, *dz = nullptr, *dvu = nullptr, *dvv = nullptr;
    int *dlayer = nullptr, *draw = nullptr, *doff = nullptr, *dtoff = nullptr, *dseeds = nullptr, *dsev = nullptr;
    int *dlocal = nullptr;
    OutBuf *out = nullptr;  // result buffer of the running batch
    bool busy = false;
    int64_t t_start = 0;
    int n_tracks = 0;
    std::vector<EvInfo> evs;
};

}  // namespace

struct tkf_server {
    tkf_config cfg{};
    tkf_server_options opt{};
    int device = 0;
    std::vector<Slot> slots;
    std::deque<Pending> queue;
    size_t queued_bytes = 0;
    std::unordered_map<uint64_t, Done> results;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    tkf_server_stats stats{};
    int worker_error = TKF_OK;
    std::vector<OutBuf *> free_bufs;  // result buffers no event holds
    size_t result_bytes = 0;          // pinned bytes of all result buffers, free or held
    cudaEvent_t t_ref = nullptr;      // device time zero of the batches' intervals
};

namespace {

void free_slot(Slot &s)
{
    if (s.pipe) tkf_pipeline_destroy(s.pipe);
    if (s.ctx) tkf_destroy(s.ctx);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.done) cudaEventDestroy(s.done);
    if (s.t_begin) cudaEventDestroy(s.t_begin);
    if (s.t_end) cudaEventDestroy(s.t_end);
    if (s.t_in) cudaEventDestroy(s.t_in);
    if (s.t_out) cudaEventDestroy(s.t_out);
    for (void *p : {(void *)s.dx, (void *)s.dy, (void *)s.dz, (void *)s.dvu, (void *)s.dvv, (void *)s.dlayer,
                    (void *)s.draw, (void *)s.doff, (void *)s.dtoff, (void *)s.dseeds, (void *)s.dsev, (void *)s.dlocal})
        cudaFree(p);
    s.hx.free(); s.hy.free(); s.hz.free(); s.hvu.free(); s.hvv.free();
    s.hlayer.free(); s.hraw.free(); s.hoff.free(); s.htoff.free();
}

size_t outbuf_bytes(const tkf_server *sv, int cap) { return (size_t)cap * (29 + sv->cfg.n_layers) * 4; }

void free_outbuf(tkf_server *sv, OutBuf *b)
{
    for (void *p : {(void *)b->par, (void *)b->cov, (void *)b->chi2, (void *)b->nhits, (void *)b->hit})
        if (p) cudaFreeHost(p);
    sv->result_bytes -= b->bytes;
    delete b;
}

// A new pinned result buffer of `cap` tracks within the budget (nullptr if it does not fit or the
// allocation fails).  cudaMallocHost can wait for the device, so the server makes n_slots of them
// when it is created and allocates more only when results held by the client exceed them.
OutBuf *new_outbuf(tkf_server *sv, int cap)
{
    const size_t bytes = outbuf_bytes(sv, cap);
    if (sv->result_bytes + bytes > sv->opt.result_bytes) return nullptr;
    OutBuf *b = new (std::nothrow) OutBuf();
    if (!b) return nullptr;
    b->cap = cap;
    b->bytes = bytes;
    sv->result_bytes += bytes;
    const size_t T = cap, L = sv->cfg.n_layers;
    if (cudaMallocHost((void **)&b->par, 6 * T * 4) || cudaMallocHost((void **)&b->cov, 21 * T * 4) ||
        cudaMallocHost((void **)&b->chi2, T * 4) || cudaMallocHost((void **)&b->nhits, T * 4) ||
        cudaMallocHost((void **)&b->hit, L * T * 4)) {
        free_outbuf(sv, b);
        return nullptr;
    }
    sv->stats.result_allocs += 1;
    return b;
}

// A result buffer for a batch of `trk` tracks (called with the lock held): the smallest free one
// that holds it, else a new one within the pinned-memory budget opt.result_bytes: of the largest
// batch (max_batch_tracks) while the budget has room for it, so that it can serve any later
// batch and the pool stops growing (no cudaMallocHost on the serving path once it holds as many
// buffers as batches are held at once), else of the batch's size class (the next power of two
// from 1024), freeing idle buffers first -- a client holding the results of many small batches
// then still fits.  nullptr when the budget is held by unreleased results (the batch waits).
OutBuf *get_outbuf(tkf_server *sv, int trk)
{
    int cap = 1024;
    while (cap < trk) cap *= 2;
    cap = std::min(cap, std::max(sv->opt.max_batch_tracks, trk));
    // the smallest free buffer that holds the batch (of its size class or larger): the slots'
    // buffers made at creation serve every batch while the client releases results promptly, so
    // nothing is allocated (cudaMallocHost) or freed (cudaFreeHost) on the serving path
    size_t best = sv->free_bufs.size();
    for (size_t k = 0; k < sv->free_bufs.size(); ++k)
        if (sv->free_bufs[k]->cap >= trk && (best == sv->free_bufs.size() || sv->free_bufs[k]->cap < sv->free_bufs[best]->cap))
            best = k;
    if (best < sv->free_bufs.size()) {
        OutBuf *b = sv->free_bufs[best];
        sv->free_bufs.erase(sv->free_bufs.begin() + best);
        return b;
    }
    const int cap_max = std::max(sv->opt.max_batch_tracks, trk);
    if (sv->result_bytes + outbuf_bytes(sv, cap_max) <= sv->opt.result_bytes) cap = cap_max;
    const size_t bytes = outbuf_bytes(sv, cap);
    while (sv->result_bytes + bytes > sv->opt.result_bytes && !sv->free_bufs.empty()) {
        free_outbuf(sv, sv->free_bufs.back());
        sv->free_bufs.pop_back();
    }
    return new_outbuf(sv, cap);
}

void unref(tkf_server *sv, OutBuf *b)
{
    if (b && --b->refs == 0) sv->free_bufs.push_back(b);
}

int init_slot(tkf_server *sv, Slot &s)
{
    const tkf_server_options &o = sv->opt;
    const size_t H = o.max_batch_hits, T = o.max_batch_tracks, E = o.max_batch_events;
    int st = tkf_create(&sv->cfg, &s.ctx);
    if (st) return st;
    if ((st = tkf_pipeline_create(s.ctx, (int)H, (int)E, (int)T, 0, &s.pipe))) return st;
    cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    if (!e) e = cudaEventCreate(&s.t_begin);
    if (!e) e = cudaEventCreate(&s.t_end);
    if (!e) e = cudaEventCreate(&s.t_in);
    if (!e) e = cudaEventCreate(&s.t_out);
    if (!e) e = s.hx.alloc(H); if (!e) e = s.hy.alloc(H); if (!e) e = s.hz.alloc(H);
    if (!e) e = s.hvu.alloc(H); if (!e) e = s.hvv.alloc(H); if (!e) e = s.hlayer.alloc(H);
    if (!e) e = s.hraw.alloc(3 * T); if (!e) e = s.hoff.alloc(E + 1); if (!e) e = s.htoff.alloc(E + 1);
    const size_t h1 = std::max<size_t>(H, 1), t1 = std::max<size_t>(T, 1), L = sv->cfg.n_layers;
    if (!e) e = cudaMalloc((void **)&s.dx, h1 * 4); if (!e) e = cudaMalloc((void **)&s.dy, h1 * 4);
    if (!e) e = cudaMalloc((void **)&s.dz, h1 * 4); if (!e) e = cudaMalloc((void **)&s.dvu, h1 * 4);
    if (!e) e = cudaMalloc((void **)&s.dvv, h1 * 4); if (!e) e = cudaMalloc((void **)&s.dlayer, h1 * 4);
    if (!e) e = cudaMalloc((void **)&s.draw, 3 * t1 * 4); if (!e) e = cudaMalloc((void **)&s.doff, (E + 1) * 4);
    if (!e) e = cudaMalloc((void **)&s.dtoff, (E + 1) * 4); if (!e) e = cudaMalloc((void **)&s.dseeds, 3 * t1 * 4);
    if (!e) e = cudaMalloc((void **)&s.dsev, t1 * 4); if (!e) e = cudaMalloc((void **)&s.dlocal, L * t1 * 4);
    if (e) return e == cudaErrorMemoryAllocation ? TKF_ERR_NOMEM : TKF_ERR_CUDA;
    return TKF_OK;
}

// Seed ids of the batch from the events' seed blocks: seed t of event e (its tl-th) reads
// raw[3 * toff[e] + j * n_e + tl] and adds the event's first hit; its event is e.
__global__ void k_prep_seeds(const int *raw, const int *toff, const int *hoff, int n_events, int n_tracks, int stride,
                             int *seeds, int *sev)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tracks) return;
    int lo = 0, hi = n_events;  // largest e with toff[e] <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (toff[mid] <= t) lo = mid; else hi = mid;
    }
    const int t0 = toff[lo], n_e = toff[lo + 1] - t0, h0 = hoff[lo];
    const int *r = raw + 3 * (size_t)t0 + (t - t0);
    seeds[t] = r[0] + h0;
    seeds[stride + t] = r[n_e] + h0;
    seeds[2 * (size_t)stride + t] = r[2 * n_e] + h0;
    sev[t] = lo;
}

// Event-local hit ids of the built tracks ([L][stride] in, [L][out_stride] out; -1 = hole).
__global__ void k_local_hits(const int *hit_idx, int stride, const int *sev, const int *hoff, int n_tracks, int L,
                             int out_stride, int *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tracks) return;
    const int h0 = hoff[sev[t]];
    for (int l = 0; l < L; ++l) {
        const int h = hit_idx[(size_t)l * stride + t];
        out[(size_t)l * out_stride + t] = h >= 0 ? h - h0 : -1;
    }
}

// Host-to-device copies of a batch, merged while consecutive pieces are adjacent on both sides
// (events lent from one host buffer, or staged back to back, move in one copy per array).
struct CopyRun {
    const char *src = nullptr;
    char *dst = nullptr;
    size_t bytes = 0;
    cudaError_t add(const void *s, void *d, size_t n, cudaStream_t st)
    {
        if (!n) return cudaSuccess;
        if (bytes && (const char *)s == src + bytes && (char *)d == dst + bytes) {
            bytes += n;
            return cudaSuccess;
        }
        const cudaError_t e = flush(st);
        src = (const char *)s;
        dst = (char *)d;
        bytes = n;
        return e;
    }
    cudaError_t flush(cudaStream_t st)
    {
        cudaError_t e = cudaSuccess;
        if (bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
        bytes = 0;
        return e;
    }
};

// Packs `evs` into slot `s` and queues, on its stream: the input copies (lent arrays straight
// from the caller's memory, copied events from the slot's pinned staging), the seed and
// event-id preparation, the pipeline, the event-local hit ids and the result copies.
int launch_batch(tkf_server *sv, Slot &s, std::vector<Pending> &evs)
{
    const int L = sv->cfg.n_layers;
    const size_t T = sv->opt.max_batch_tracks;
    cudaStream_t st = s.stream;
    cudaError_t e = cudaSuccess;
    CopyRun run[7];
    int hit = 0, trk = 0;
    s.evs.clear();
    if (cudaEventRecord(s.t_begin, st) != cudaSuccess) return TKF_ERR_CUDA;
    for (size_t k = 0; k < evs.size(); ++k) {
        Pending &p = evs[k];
        const size_t nb = (size_t)p.n_hits * 4, sb = (size_t)p.n_seeds * 12;
        s.hoff.p[k] = hit;
        s.htoff.p[k] = trk;
        const void *src[7];
        if (p.borrowed) {
            src[0] = p.bx; src[1] = p.by; src[2] = p.bz; src[3] = p.bvu; src[4] = p.bvv; src[5] = p.blayer;
            src[6] = p.bseeds;
        } else {
            std::memcpy(s.hx.p + hit, p.px(), nb);
            std::memcpy(s.hy.p + hit, p.py(), nb);
            std::memcpy(s.hz.p + hit, p.pz(), nb);
            std::memcpy(s.hvu.p + hit, p.pvu(), nb);
            std::memcpy(s.hvv.p + hit, p.pvv(), nb);
            std::memcpy(s.hlayer.p + hit, p.player(), nb);
            std::memcpy(s.hraw.p + 3 * (size_t)trk, p.pseeds(), sb);
            src[0] = s.hx.p + hit; src[1] = s.hy.p + hit; src[2] = s.hz.p + hit; src[3] = s.hvu.p + hit;
            src[4] = s.hvv.p + hit; src[5] = s.hlayer.p + hit; src[6] = s.hraw.p + 3 * (size_t)trk;
        }
        void *dst[7] = {s.dx + hit, s.dy + hit, s.dz + hit, s.dvu + hit, s.dvv + hit, s.dlayer + hit,
                        s.draw + 3 * (size_t)trk};
        for (int j = 0; j < 7 && !e; ++j) e = run[j].add(src[j], dst[j], j < 6 ? nb : sb, st);
        s.evs.push_back({p.ticket, hit, p.n_hits, trk, p.n_seeds, p.t_submit});
        hit += p.n_hits;
        trk += p.n_seeds;
    }
    for (int j = 0; j < 7 && !e; ++j) e = run[j].flush(st);
    const int E = (int)evs.size();
    s.hoff.p[E] = hit;
    s.htoff.p[E] = trk;
    s.n_tracks = trk;
    if (!e) e = cudaMemcpyAsync(s.doff, s.hoff.p, (E + 1) * 4, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(s.dtoff, s.htoff.p, (E + 1) * 4, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaEventRecord(s.t_in, st);
    if (!e && trk) {
        k_prep_seeds<<<(trk + 255) / 256, 256, 0, st>>>(s.draw, s.dtoff, s.doff, E, trk, (int)T, s.dseeds, s.dsev);
        e = cudaGetLastError();
    }
    if (e) return TKF_ERR_CUDA;
    tkf_hits h{};
    h.x = s.dx; h.y = s.dy; h.z = s.dz; h.var_u = s.dvu; h.var_v = s.dvv; h.layer = s.dlayer;
    h.event_off = s.doff;
    h.n = hit;
    h.n_events = E;
    int rc = tkf_pipeline_run(s.pipe, &h, s.dseeds, s.dsev, trk, (tkf_stream)st);
    if (rc) return rc;
    tkf_tracks built, fitted;
    tkf_pipeline_outputs(s.pipe, nullptr, &built, &fitted);
    const size_t es = sizeof(float), dp = (size_t)fitted.stride * es;
    OutBuf *o = s.out;
    const size_t hp = (size_t)o->cap * es;  // host pitch
    if (trk) {
        k_local_hits<<<(trk + 255) / 256, 256, 0, st>>>(built.hit_idx, built.stride, s.dsev, s.doff, trk, L, (int)T,
                                                        s.dlocal);
        e = cudaGetLastError();
        if (!e) e = cudaEventRecord(s.t_out, st);
        if (!e) e = cudaMemcpy2DAsync(o->par, hp, fitted.par, dp, trk * es, 6, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaMemcpy2DAsync(o->cov, hp, fitted.cov, dp, trk * es, 21, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaMemcpyAsync(o->chi2, fitted.chi2, trk * es, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaMemcpyAsync(o->nhits, fitted.nhits, trk * 4, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaMemcpy2DAsync(o->hit, hp, s.dlocal, T * 4, trk * 4, L, cudaMemcpyDeviceToHost, st);
    }
    if (!e && !trk) e = cudaEventRecord(s.t_out, st);
    if (!e) e = cudaEventRecord(s.t_end, st);
    if (!e) e = cudaEventRecord(s.done, st);
    if (e) return TKF_ERR_CUDA;
    s.t_start = now_ns();
    return TKF_OK;
}

// Hands each finished event its columns of the batch's result buffer (called with the lock
// held).
void harvest(tkf_server *sv, Slot &s)
{
    const int64_t t_done = now_ns();
    float g0 = 0.f, g1 = 0.f, gi = 0.f, go = 0.f;  // the batch's device times against the server's time zero
    if (cudaEventElapsedTime(&g0, sv->t_ref, s.t_begin) != cudaSuccess ||
        cudaEventElapsedTime(&g1, sv->t_ref, s.t_end) != cudaSuccess ||
        cudaEventElapsedTime(&gi, sv->t_ref, s.t_in) != cudaSuccess ||
        cudaEventElapsedTime(&go, sv->t_ref, s.t_out) != cudaSuccess)
        g0 = g1 = gi = go = -1.f;
    OutBuf *o = s.out;
    o->refs = 1;  // held by this function until the end
    for (const EvInfo &ev : s.evs) {
        auto it = sv->results.find(ev.ticket);
        if (it == sv->results.end()) continue;  // released before completion
        Done &d = it->second;
        d.buf = o;
        o->refs += 1;
        d.trk0 = ev.trk0;
        d.n = ev.n_tracks;
        d.t_submit = ev.t_submit;
        d.t_start = s.t_start;
        d.t_done = t_done;
        d.gpu_start_ms = g0;
        d.gpu_done_ms = g1;
        d.gpu_inputs_ms = gi;
        d.gpu_results_ms = go;
        d.status = TKF_OK;
        d.done = true;
        sv->stats.events_done += 1;
        sv->stats.tracks_done += ev.n_tracks;
    }
    unref(sv, o);
    s.out = nullptr;
    sv->stats.batches += 1;
    sv->stats.max_batch_events = std::max<int64_t>(sv->stats.max_batch_events, (int64_t)s.evs.size());
    s.busy = false;
    s.evs.clear();
}

void worker_loop(tkf_server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        // completed batches
        for (Slot &s : sv->slots)
            if (s.busy && cudaEventQuery(s.done) == cudaSuccess) harvest(sv, s);
        sv->cv_done.notify_all();
        if (sv->stop) break;
        // new batches on free slots: every queued event that fits
        bool launched = false;
        for (Slot &s : sv->slots) {
            if (s.busy || sv->queue.empty()) continue;
            std::vector<Pending> batch;
            size_t hits = 0, trks = 0;
            while (!sv->queue.empty() && (int)batch.size() < sv->opt.max_batch_events) {
                Pending &p = sv->queue.front();
                if (hits + p.n_hits > (size_t)sv->opt.max_batch_hits || trks + p.n_seeds > (size_t)sv->opt.max_batch_tracks)
                    break;
                hits += p.n_hits;
                trks += p.n_seeds;
                sv->queued_bytes -= p.bytes;
                batch.push_back(std::move(p));
                sv->queue.pop_front();
            }
            if (batch.empty()) continue;
            s.out = get_outbuf(sv, (int)trks);
            if (!s.out) {  // result memory held by unreleased results: put the batch back, wait
                for (auto it = batch.rbegin(); it != batch.rend(); ++it) {
                    sv->queued_bytes += it->bytes;
                    sv->queue.push_front(std::move(*it));
                }
                break;
            }
            s.busy = true;  // owned by this thread from here; submitters only touch the queue
            lk.unlock();
            const int rc = launch_batch(sv, s, batch);
            lk.lock();
            if (rc) {
                s.busy = false;
                sv->free_bufs.push_back(s.out);
                s.out = nullptr;
                sv->worker_error = rc;
                for (Pending &p : batch) {
                    auto it = sv->results.find(p.ticket);
                    if (it != sv->results.end()) {
                        it->second.done = true;
                        it->second.status = rc;
                    }
                }
            }
            launched = true;
        }
        bool any_busy = false;
        for (Slot &s : sv->slots) any_busy |= s.busy;
        if (!launched && !any_busy && !sv->queue.empty()) {
            // the queue waits for result memory: sleep until a release (or stop)
            sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        } else if (!launched) {
            // wait for a submission, or poll the running batches every 20 microseconds
            if (any_busy)
                sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(5),
                                     [sv] { return sv->stop || !sv->queue.empty(); });
        }
    }
    // drain: wait for running batches so that their buffers can be freed
    for (Slot &s : sv->slots)
        if (s.busy) {
            lk.unlock();
            cudaEventSynchronize(s.done);
            lk.lock();
            harvest(sv, s);
        }
    sv->cv_done.notify_all();
}

}  // namespace

extern "C" {

void tkf_server_default_options(tkf_server_options *o)
{
    if (!o) return;
    o->n_slots = 3;
    o->max_batch_events = 64;
    o->max_batch_hits = 1 << 22;
    o->max_batch_tracks = 1 << 18;
    o->queue_bytes = (size_t)1 << 30;
    o->result_bytes = (size_t)1 << 30;
}

int tkf_server_create(const tkf_config *cfg, const tkf_server_options *opt, tkf_server **out)
{
    if (!cfg || !opt || !out) return TKF_ERR_INVALID;
    *out = nullptr;
    if (opt->n_slots < 1 || opt->max_batch_events < 1 || opt->max_batch_hits < 1 || opt->max_batch_tracks < 1 ||
        cfg->precision == TKF_FP64 || cfg->n_layers < 1 ||
        opt->result_bytes < (size_t)opt->max_batch_tracks * (29 + cfg->n_layers) * 4)
        return TKF_ERR_INVALID;
    tkf_server *sv = new (std::nothrow) tkf_server();
    if (!sv) return TKF_ERR_NOMEM;
    sv->cfg = *cfg;
    sv->opt = *opt;
    if (cudaGetDevice(&sv->device) != cudaSuccess) {
        delete sv;
        return TKF_ERR_CUDA;
    }
    sv->slots.resize(opt->n_slots);
    for (Slot &s : sv->slots) {
        const int st = init_slot(sv, s);
        if (st) {
            for (Slot &t : sv->slots) free_slot(t);
            delete sv;
            return st;
        }
    }
    // one full-size result buffer per slot (as many as the budget holds), made before any batch runs
    for (int k = 0; k < opt->n_slots; ++k) {
        OutBuf *b = new_outbuf(sv, opt->max_batch_tracks);
        if (!b) break;
        sv->free_bufs.push_back(b);
    }
    if (cudaEventCreate(&sv->t_ref) != cudaSuccess || cudaEventRecord(sv->t_ref, sv->slots[0].stream) != cudaSuccess ||
        cudaEventSynchronize(sv->t_ref) != cudaSuccess) {
        for (Slot &t : sv->slots) free_slot(t);
        for (OutBuf *b : sv->free_bufs) free_outbuf(sv, b);
        if (sv->t_ref) cudaEventDestroy(sv->t_ref);
        delete sv;
        return TKF_ERR_CUDA;
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return TKF_OK;
}

int tkf_server_destroy(tkf_server *sv)
{
    if (!sv) return TKF_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot &s : sv->slots) free_slot(s);
    std::vector<OutBuf *> held;
    for (auto &kv : sv->results)
        if (kv.second.buf && std::find(held.begin(), held.end(), kv.second.buf) == held.end())
            held.push_back(kv.second.buf);
    for (OutBuf *b : held) free_outbuf(sv, b);
    for (OutBuf *b : sv->free_bufs) free_outbuf(sv, b);
    if (sv->t_ref) cudaEventDestroy(sv->t_ref);
    delete sv;
    return TKF_OK;
}

}  // extern "C"

namespace {

// Checks one event; TKF_OK or TKF_ERR_INVALID.
int check_event(const tkf_server *sv, const tkf_event *ev)
{
    if (!ev || ev->n_hits < 0 || ev->n_seeds < 0) return TKF_ERR_INVALID;
    if (ev->n_hits > 0 && (!ev->x || !ev->y || !ev->z || !ev->var_u || !ev->var_v || !ev->layer)) return TKF_ERR_INVALID;
    if (ev->n_seeds > 0 && !ev->seed_hits) return TKF_ERR_INVALID;
    if (ev->n_hits > sv->opt.max_batch_hits || ev->n_seeds > sv->opt.max_batch_tracks) return TKF_ERR_INVALID;
    int lo = 0, hi = 0;
    for (int t = 0; t < 3 * ev->n_seeds; ++t) {
        lo = std::min(lo, ev->seed_hits[t]);
        hi = std::max(hi, ev->seed_hits[t]);
    }
    if (lo < 0 || (ev->n_seeds > 0 && hi >= ev->n_hits)) return TKF_ERR_INVALID;
    return TKF_OK;
}

size_t event_bytes(const tkf_event *ev)
{
    return ev->borrow ? 64 : (size_t)ev->n_hits * 24 + (size_t)ev->n_seeds * 12;
}

// The queue entry of a checked event (copies its arrays unless it is lent).
Pending make_pending(const tkf_event *ev, int64_t t_submit)
{
    Pending p;
    p.n_hits = ev->n_hits;
    p.n_seeds = ev->n_seeds;
    if (ev->borrow) {
        p.borrowed = true;
        p.bx = ev->x; p.by = ev->y; p.bz = ev->z; p.bvu = ev->var_u; p.bvv = ev->var_v;
        p.blayer = ev->layer;
        p.bseeds = ev->seed_hits;
    } else {
        p.x.assign(ev->x, ev->x + ev->n_hits);
        p.y.assign(ev->y, ev->y + ev->n_hits);
        p.z.assign(ev->z, ev->z + ev->n_hits);
        p.vu.assign(ev->var_u, ev->var_u + ev->n_hits);
        p.vv.assign(ev->var_v, ev->var_v + ev->n_hits);
        p.layer.assign(ev->layer, ev->layer + ev->n_hits);
        p.seeds.assign(ev->seed_hits, ev->seed_hits + 3 * ev->n_seeds);
    }
    p.bytes = event_bytes(ev);
    p.t_submit = t_submit;
    return p;
}

// Submits events[0..n): the checked prefix that fits the queue budget is reserved, copied
// outside the lock, then queued in one piece with one wake-up of the worker (n = 1: one
// arrival).
int submit_some(tkf_server *sv, const tkf_event *events, int32_t n, uint64_t *tickets, int32_t *n_accepted)
{
    const int64_t t_submit = now_ns();
    *n_accepted = 0;
    int32_t m = 0;
    int first_err = TKF_OK;
    while (m < n && (first_err = check_event(sv, &events[m])) == TKF_OK) ++m;
    int32_t k = 0;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->worker_error) return sv->worker_error;
        while (k < m && sv->queued_bytes + bytes + event_bytes(&events[k]) <= sv->opt.queue_bytes) {
            bytes += event_bytes(&events[k]);
            ++k;
        }
        if (k < m) {
            sv->stats.rejected += 1;
            first_err = TKF_ERR_AGAIN;
        }
        sv->queued_bytes += bytes;  // reserved before copying outside the lock
    }
    std::vector<Pending> ps;
    ps.reserve(k);
    for (int32_t i = 0; i < k; ++i) ps.push_back(make_pending(&events[i], t_submit));
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (int32_t i = 0; i < k; ++i) {
            ps[i].ticket = sv->next_ticket++;
            tickets[i] = ps[i].ticket;
            sv->results.emplace(ps[i].ticket, Done());
            sv->queue.push_back(std::move(ps[i]));
            sv->stats.submitted += 1;
        }
    }
    if (k) sv->cv_work.notify_one();
    *n_accepted = k;
    return first_err;
}

}  // namespace

extern "C" {

int tkf_submit_event(tkf_server *sv, const tkf_event *ev, uint64_t *ticket)
{
    if (!sv || !ev || !ticket) return TKF_ERR_INVALID;
    int32_t n_acc = 0;
    return submit_some(sv, ev, 1, ticket, &n_acc);
}

int tkf_poll(tkf_server *sv, uint64_t ticket, tkf_result *r, int64_t timeout_us)
{
    if (!sv || !r) return TKF_ERR_INVALID;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) return TKF_ERR_INVALID;
    if (!it->second.done) {
        if (timeout_us == 0) return TKF_ERR_NOTREADY;
        const bool ok = sv->cv_done.wait_for(lk, std::chrono::microseconds(std::max<int64_t>(timeout_us, 1)), [&] {
            auto jt = sv->results.find(ticket);
            return jt == sv->results.end() || jt->second.done;
        });
        it = sv->results.find(ticket);
        if (it == sv->results.end()) return TKF_ERR_INVALID;
        if (!ok || !it->second.done) return TKF_ERR_TIMEOUT;
    }
    const Done &d = it->second;
    r->status = d.status;
    r->n_tracks = d.n;
    const OutBuf *o = d.buf;
    r->stride = o ? o->cap : 0;
    r->par = o ? o->par + d.trk0 : nullptr;
    r->cov = o ? o->cov + d.trk0 : nullptr;
    r->chi2 = o ? o->chi2 + d.trk0 : nullptr;
    r->nhits = o ? o->nhits + d.trk0 : nullptr;
    r->hit_idx = o ? o->hit + d.trk0 : nullptr;
    r->t_submit_ns = d.t_submit;
    r->t_start_ns = d.t_start;
    r->t_done_ns = d.t_done;
    r->gpu_start_ms = d.gpu_start_ms;
    r->gpu_done_ms = d.gpu_done_ms;
    r->gpu_inputs_ms = d.gpu_inputs_ms;
    r->gpu_results_ms = d.gpu_results_ms;
    return TKF_OK;
}

int tkf_release(tkf_server *sv, uint64_t ticket)
{
    if (!sv) return TKF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) return TKF_ERR_INVALID;
    unref(sv, it->second.buf);
    sv->results.erase(it);
    sv->cv_work.notify_one();  // a batch may be waiting for result memory
    return TKF_OK;
}

int tkf_submit_events(tkf_server *sv, const tkf_event *events, int32_t n, uint64_t *tickets, int32_t *n_accepted)
{
    if (!sv || (n > 0 && (!events || !tickets)) || n < 0 || !n_accepted) return TKF_ERR_INVALID;
    *n_accepted = 0;
    // one event at a time, as separate arrivals: the worker starts a batch with the first events
    // while the rest are still being queued, so the first copies and kernels overlap the
    // submission of the burst and the batches that follow grow to max_batch_events
    for (int32_t k = 0; k < n; ++k) {
        int32_t one = 0;
        const int st = submit_some(sv, &events[k], 1, &tickets[k], &one);
        if (st) return st;
        *n_accepted = k + 1;
    }
    return TKF_OK;
}

int tkf_wait_all(tkf_server *sv, const uint64_t *tickets, int32_t n, tkf_result *results, int64_t timeout_us)
{
    if (!sv || n < 0 || (n > 0 && (!tickets || !results))) return TKF_ERR_INVALID;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max<int64_t>(timeout_us, 0));
    for (int32_t k = 0; k < n; ++k) {
        const int64_t left = std::chrono::duration_cast<std::chrono::microseconds>(
                                 deadline - std::chrono::steady_clock::now()).count();
        const int st = tkf_poll(sv, tickets[k], &results[k], timeout_us == 0 ? 0 : std::max<int64_t>(left, 1));
        if (st) return st;
    }
    return TKF_OK;
}

int tkf_release_many(tkf_server *sv, const uint64_t *tickets, int32_t n)
{
    if (!sv || n < 0 || (n > 0 && !tickets)) return TKF_ERR_INVALID;
    int first = TKF_OK;
    for (int32_t k = 0; k < n; ++k) {
        const int st = tkf_release(sv, tickets[k]);
        if (st && !first) first = st;
    }
    return first;
}

int tkf_server_get_stats(tkf_server *sv, tkf_server_stats *out)
{
    if (!sv || !out) return TKF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    return TKF_OK;
}

}  // extern "C"
