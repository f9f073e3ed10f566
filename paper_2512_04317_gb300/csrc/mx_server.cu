// Request server with continuous batching over the ragged batch executor.
//
// Requests (host buffers) enter a FIFO queue.  A worker thread admits them in
// arrival order whenever an execution slot (a stream with its own engine) is
// free and the device memory budget allows: all queued requests that fit form
// one batch, which is copied in, transformed in place by one engine run and
// copied out on that slot while batches admitted earlier still run on other
// slots.  Each request's copy out ends with its own host callback, which
// completes that request; the last one returns the slot and its memory.  No kernel waits on the host: the device-side part
// of a request is the engine's launches, the host side only enqueues.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "mx_plan.h"

using namespace mxfft;

namespace {

double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

struct SReq {
    mxfft_request r;
    size_t bytes;          // complex data on the device
    size_t rss_bytes;      // RSS images on the device
    double t_submit, t_admit;
};

struct DoneCtx {
    struct ::mxfft_server_s* srv;
    int slot, req;
};

struct Finished {
    int slot, req;
    double t;
};

struct Slot {
    cudaStream_t stream = nullptr;
    mxfft_engine_t eng = nullptr;
    bool busy = false;
    std::vector<SReq> reqs;
    std::vector<DoneCtx> ctx;         // one per request, stable while the batch runs
    int n_done = 0;
    int first_slice = 0;              // running slice offset while retiring
    size_t bytes = 0;
    uint32_t* h_flags = nullptr;      // pinned: per slice, non-finite input magnitude
    int flags_cap = 0;
    int status = MXFFT_OK;
};

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

}  // namespace

struct mxfft_server_s {
    mxfft_server_config cfg;
    int device = -1;
    std::mutex mu;
    std::condition_variable cv;        // worker: submissions, finished slots, stop
    std::condition_variable cv_done;   // waiters: completions
    std::deque<SReq> pending;
    std::deque<mxfft_completion> done;
    std::vector<Slot> slots;
    std::vector<Finished> finished;
    size_t budget = 0, inflight = 0, peak = 0;
    uint64_t submitted = 0, completed = 0, batches = 0;
    bool stop = false;
    std::thread worker;
};

namespace {

void CUDART_CB request_done(void* arg) {
    DoneCtx* c = static_cast<DoneCtx*>(arg);
    const double t = now_us();
    std::lock_guard<std::mutex> lk(c->srv->mu);
    c->srv->finished.push_back(Finished{c->slot, c->req, t});
    c->srv->cv.notify_all();
}

// Enqueue a batch on its slot: copies in, one engine run, the flags, then per
// request its copy out and a host callback.  Returns the number of requests
// whose callback was enqueued (the caller completes the rest itself).
int launch_batch(mxfft_server_s* S, int i) {
    Slot& sl = S->slots[i];
    cudaStream_t s = sl.stream;
    int slices = 0;
    for (const SReq& q : sl.reqs) slices += q.r.slices;
    sl.status = MXFFT_OK;
    if (slices > sl.flags_cap) {
        if (sl.h_flags) cudaFreeHost(sl.h_flags);
        sl.h_flags = nullptr;
        sl.flags_cap = 0;
        int cap = 64;
        while (cap < slices) cap *= 2;
        if (cudaMallocHost(&sl.h_flags, cap * sizeof(uint32_t)) != cudaSuccess) {
            sl.status = MXFFT_ERR_NOMEM;
            return 0;
        }
        sl.flags_cap = cap;
    }
    char* d = nullptr;
    cudaError_t err = cudaMallocAsync((void**)&d, sl.bytes, s);
    if (err != cudaSuccess) {
        sl.status = cuda_status(err);
        return 0;
    }
    // layout of the batch buffer: each request's data, then its RSS images
    std::vector<mxfft_item> items;
    std::vector<size_t> offs;
    size_t off = 0;
    for (const SReq& q : sl.reqs) {
        if (err == cudaSuccess) err = cudaMemcpyAsync(d + off, q.r.host_in, q.bytes, cudaMemcpyHostToDevice, s);
        void* rss = q.rss_bytes ? d + off + q.bytes : nullptr;
        items.push_back(mxfft_item{q.r.n0, q.r.n1, q.r.format, q.r.k, q.r.op, q.r.slices, d + off, d + off,
                                   q.r.coils, 0, rss});
        offs.push_back(off);
        off += q.bytes + q.rss_bytes;
    }
    int rc = err == cudaSuccess ? MXFFT_OK : cuda_status(err);
    if (rc == MXFFT_OK) rc = mxfft_engine_run(sl.eng, items.data(), (int)items.size(), s);
    if (rc == MXFFT_OK) rc = cuda_status(engine_flags_async(sl.eng, sl.h_flags, s));
    sl.status = rc;
    if (rc != MXFFT_OK) std::fill(sl.h_flags, sl.h_flags + slices, 0u);
    sl.ctx.assign(sl.reqs.size(), DoneCtx{S, i, 0});
    int queued = 0;
    for (size_t j = 0; j < sl.reqs.size(); j++) {
        const SReq& q = sl.reqs[j];
        if (rc == MXFFT_OK && q.r.host_out)
            rc = cuda_status(cudaMemcpyAsync(q.r.host_out, d + offs[j], q.bytes, cudaMemcpyDeviceToHost, s));
        if (rc == MXFFT_OK && q.rss_bytes)
            rc = cuda_status(cudaMemcpyAsync(q.r.host_rss, d + offs[j] + q.bytes, q.rss_bytes,
                                             cudaMemcpyDeviceToHost, s));
        if (rc != MXFFT_OK) sl.status = rc;
        sl.ctx[j].req = (int)j;
        if (cudaLaunchHostFunc(s, request_done, &sl.ctx[j]) != cudaSuccess) break;
        queued++;
    }
    cudaFreeAsync(d, s);
    return queued;
}

// One request of a slot's batch has its result in host memory.
void complete(mxfft_server_s* S, int i, int j, double t) {
    Slot& sl = S->slots[i];
    const SReq& q = sl.reqs[j];
    int first = 0;
    for (int r = 0; r < j; r++) first += sl.reqs[r].r.slices;
    int fl = 0;
    for (int k = 0; k < q.r.slices; k++)
        if (sl.status == MXFFT_OK && sl.h_flags && sl.h_flags[first + k]) fl = 1;
    S->done.push_back(mxfft_completion{q.r.tag, sl.status, fl, q.t_submit, q.t_admit, t});
    S->completed++;
    S->cv_done.notify_all();
    if (++sl.n_done == (int)sl.reqs.size()) {
        S->inflight -= sl.bytes;
        sl.bytes = 0;
        sl.reqs.clear();
        sl.n_done = 0;
        sl.busy = false;
    }
}

void worker_main(mxfft_server_s* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        for (const Finished& f : S->finished) complete(S, f.slot, f.req, f.t);
        S->finished.clear();
        bool busy = false;
        int free_slot = -1;
        for (size_t i = 0; i < S->slots.size(); i++) {
            busy = busy || S->slots[i].busy;
            if (!S->slots[i].busy && free_slot < 0) free_slot = (int)i;
        }
        if (S->stop && S->pending.empty() && !busy) break;
        if (free_slot >= 0 && !S->pending.empty()) {
            std::vector<SReq> batch;
            size_t bytes = 0;
            int slices = 0;
            const double ta = now_us();
            const size_t max_bytes = S->cfg.max_batch_bytes ? (size_t)S->cfg.max_batch_bytes : SIZE_MAX;
            while (!S->pending.empty()) {
                SReq q = S->pending.front();
                const size_t qb = q.bytes + q.rss_bytes;
                if (qb > S->budget) {
                    // can never be admitted
                    S->pending.pop_front();
                    S->done.push_back(mxfft_completion{q.r.tag, MXFFT_ERR_NOMEM, 0, q.t_submit, ta, ta});
                    S->completed++;
                    S->cv_done.notify_all();
                    continue;
                }
                if (S->inflight + bytes + qb > S->budget) break;
                if (!batch.empty() &&
                    (slices + q.r.slices > S->cfg.max_batch_slices || bytes + qb > max_bytes))
                    break;
                q.t_admit = ta;
                batch.push_back(q);
                bytes += qb;
                slices += q.r.slices;
                S->pending.pop_front();
            }
            if (!batch.empty()) {
                Slot& sl = S->slots[free_slot];
                sl.busy = true;
                sl.bytes = bytes;
                sl.n_done = 0;
                sl.reqs.swap(batch);
                S->inflight += bytes;
                S->peak = std::max(S->peak, S->inflight);
                S->batches++;
                lk.unlock();
                const int queued = launch_batch(S, free_slot);
                lk.lock();
                // requests without a callback complete here, with the slot's status
                Slot& sl2 = S->slots[free_slot];
                if (queued < (int)sl2.reqs.size() && sl2.status == MXFFT_OK) sl2.status = MXFFT_ERR_CUDA;
                for (int j = queued, n = (int)sl2.reqs.size(); j < n; j++)
                    S->finished.push_back(Finished{free_slot, j, now_us()});
                continue;
            }
        }
        S->cv.wait_for(lk, std::chrono::milliseconds(5));
    }
}

void destroy_slots(mxfft_server_s* S) {
    for (Slot& sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.eng) mxfft_engine_destroy(sl.eng);
        if (sl.h_flags) cudaFreeHost(sl.h_flags);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    S->slots.clear();
}

}  // namespace

extern "C" {

int mxfft_server_create(const mxfft_server_config* cfg, mxfft_server_t* out) {
    if (!out || !cfg) return MXFFT_ERR_INVALID;
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 64 || cfg->max_batch_slices < 1) return MXFFT_ERR_INVALID;
    mxfft_server_s* S = new (std::nothrow) mxfft_server_s;
    if (!S) return MXFFT_ERR_NOMEM;
    S->cfg = *cfg;
    int rc = cuda_status(cudaGetDevice(&S->device));
    if (rc == MXFFT_OK) {
        size_t fr = 0, tot = 0;
        rc = cuda_status(cudaMemGetInfo(&fr, &tot));
        S->budget = cfg->mem_budget ? (size_t)cfg->mem_budget : (size_t)(0.8 * (double)fr);
    }
    S->slots.resize(cfg->slots);
    for (int i = 0; i < cfg->slots && rc == MXFFT_OK; i++) {
        Slot& sl = S->slots[i];
        rc = cuda_status(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
        if (rc == MXFFT_OK) rc = mxfft_engine_create(cfg->tau, cfg->target, cfg->engine_flags, &sl.eng);
    }
    if (rc != MXFFT_OK) {
        destroy_slots(S);
        delete S;
        return rc;
    }
    try {
        S->worker = std::thread(worker_main, S);
    } catch (...) {
        destroy_slots(S);
        delete S;
        return MXFFT_ERR_NOMEM;
    }
    *out = S;
    return MXFFT_OK;
}

int mxfft_server_submit(mxfft_server_t S, const mxfft_request* r) {
    if (!S || !r) return MXFFT_ERR_INVALID;
    if (!pow2_in(r->n0, 2, 2048) || !pow2_in(r->n1, 2, 2048) || r->format < 0 || r->format > MXFFT_FP32_REF ||
        !pow2_in(r->k, 2, 128) || r->op < 0 || r->op > 3 || r->slices < 1 || !r->host_in ||
        r->reserved != 0 || (!r->host_out && !r->host_rss))
        return MXFFT_ERR_INVALID;
    if (r->host_rss && (r->coils < 1 || r->slices % r->coils)) return MXFFT_ERR_INVALID;
    if (r->op == MXFFT_OP_ROUNDTRIP_FUSED && r->format == MXFFT_FP16) return MXFFT_ERR_UNSUPPORTED;
    SReq q;
    q.r = *r;
    q.bytes = (size_t)r->slices * r->n0 * r->n1 * sizeof(float2);
    // (a multiple of 16 bytes: n0 n1 >= 4 points of 4 bytes)
    q.rss_bytes = r->host_rss ? (size_t)(r->slices / r->coils) * r->n0 * r->n1 * sizeof(float) : 0;
    q.t_submit = now_us();
    q.t_admit = 0.0;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return MXFFT_ERR_INVALID;
    S->pending.push_back(q);
    S->submitted++;
    S->cv.notify_all();
    return MXFFT_OK;
}

int mxfft_server_poll(mxfft_server_t S, mxfft_completion* out, int max, int* n_out) {
    if (!S || !n_out || max < 0 || (max > 0 && !out)) return MXFFT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    int n = 0;
    while (n < max && !S->done.empty()) {
        out[n++] = S->done.front();
        S->done.pop_front();
    }
    *n_out = n;
    return MXFFT_OK;
}

int mxfft_server_wait(mxfft_server_t S, double timeout_s) {
    if (!S || !(timeout_s >= 0.0)) return MXFFT_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                           std::chrono::duration<double>(timeout_s));
    const bool ok = S->cv_done.wait_until(lk, until, [S] { return S->completed == S->submitted; });
    return ok ? MXFFT_OK : MXFFT_ERR_TIMEOUT;
}

int mxfft_server_stats(mxfft_server_t S, uint64_t* batches, uint64_t* peak_bytes, uint64_t* budget) {
    if (!S) return MXFFT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (batches) *batches = S->batches;
    if (peak_bytes) *peak_bytes = S->peak;
    if (budget) *budget = S->budget;
    return MXFFT_OK;
}

int mxfft_server_destroy(mxfft_server_t S) {
    if (!S) return MXFFT_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    destroy_slots(S);
    delete S;
    return MXFFT_OK;
}

}  // extern "C"
