// Serving (include/emd.h, emd_server_*): a request loop over a resident database.
//
// Requests are single queries.  A worker thread admits them in arrival order onto slots --
// each slot a stream with pinned staging -- as long as a slot is free and the device
// workspace pool can hold the request, and runs on the slot the same kernel sequence as
// the batch entry points (Phase 1, table, forward pass, pruned reverse pass and top-K of
// Section 4/5; the unpruned path with a full top-K otherwise).  Requests that arrive while
// others are on the device are admitted as slots and workspace free up, so their kernels
// overlap on the GPU.  A request's arithmetic depends only on its own inputs: no sum or
// selection crosses requests, hence a result is the same alone and in any mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "emd_db.cuh"

using namespace emd;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int64_t kAlign = 256;

int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over the workspace pool: free blocks keyed by offset, coalesced on
// release.  Sizes are multiples of kAlign.
class PoolAllocator {
public:
    void reset(int64_t bytes)
    {
        free_.clear();
        if (bytes > 0) free_[0] = bytes;
        used_ = 0;
    }
    bool alloc(int64_t size, int64_t* off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < size) continue;
            *off = it->first;
            const int64_t rest = it->second - size;
            const int64_t next = it->first + size;
            free_.erase(it);
            if (rest > 0) free_[next] = rest;
            used_ += size;
            return true;
        }
        return false;
    }
    void release(int64_t off, int64_t size)
    {
        auto it = free_.emplace(off, size).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
        used_ -= size;
    }
    int64_t used() const { return used_; }

private:
    std::map<int64_t, int64_t> free_;
    int64_t used_ = 0;
};

// Device buffers of one request, carved from the pool.
struct ReqDev {
    int32_t* idx = nullptr;
    float* w = nullptr;
    Lane L;
    float* t_out = nullptr;
    int64_t* out_idx = nullptr;
    float* out_dist = nullptr;
    int* ok = nullptr;
};

// Lays out a request's buffers from `base` (nullptr: sizes only) and returns the bytes.
int64_t layout(const emd_db* db, int h, int tk, char* base, ReqDev* r)
{
    int64_t off = 0;
    auto take = [&](auto** p, int64_t bytes) {
        using T = std::remove_reference_t<decltype(**p)>;
        if (base) *p = reinterpret_cast<T*>(base + off);
        off += align_up(std::max<int64_t>(bytes, 1));
    };
    ReqDev tmp;
    ReqDev& d = r ? *r : tmp;
    const int ldd = (int)round_up(h, 32);
    const int qrows = (int)round_up(ldd, kDistBN);
    const int64_t npad = round_up(h, 128);
    take(&d.idx, (int64_t)h * 4);
    take(&d.w, (int64_t)h * 4);
    if (!db->cost_mode) {
        take(&d.L.Q, (int64_t)qrows * db->ldm * 4);
        take(&d.L.qnorm, (int64_t)qrows * 4);
        if (db->tc) {
            take(&d.L.q_hi, npad * db->kpad * 2);
            if (db->tcfmt == TC_SPLIT) take(&d.L.q_lo, npad * db->kpad * 2);
            take(&d.L.q_scale, npad * 4);
        }
    }
    take(&d.L.D, db->v_used * ldd * 4);
    take(&d.L.tab, db->v_used * tk * 8);
    take(&d.L.t_fwd, db->n * 4);
    take(&d.L.t_rev, db->n * 4);
    take(&d.t_out, db->n * 4);
    take(&d.L.sel_idx, kPruneMaxK * 8);
    take(&d.L.sel_val, kPruneMaxK * 4);
    take(&d.L.cand_idx, kPruneCap * 8);
    take(&d.L.cand_sym, 2 * kPruneCap * 4);
    take(&d.L.cand_count, 4);
    take(&d.L.scratch, kTopkScratchRow * 8);
    take(&d.out_idx, kMaxTopK * 8);
    take(&d.out_dist, kMaxTopK * 4);
    take(&d.ok, 4);
    return off;
}

enum ReqState { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct Request {
    uint64_t ticket = 0;
    int h = 0, meas = 0, k = 0, K = 0;
    bool pruned = false;
    std::vector<int32_t> idx;
    std::vector<float> w;
    Clock::time_point t_submit;
    int64_t ws_off = -1, ws_bytes = 0;
    int state = QUEUED;
    emd_status status = EMD_OK;
    std::string err;
    std::vector<int64_t> out_idx;
    std::vector<float> out_dist;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    char* pinned = nullptr;  // idx | w | out_idx | out_dist | ok
    int32_t* h_idx = nullptr;
    float* h_w = nullptr;
    int64_t* h_oidx = nullptr;
    float* h_odist = nullptr;
    int* h_ok = nullptr;
    Request* req = nullptr;
    ReqDev dev;
    bool fallback = false;  // the unpruned recomputation is in flight
};

double pct(std::vector<double> v, double p)
{
    if (v.empty()) return 0.0;
    const size_t i = std::min(v.size() - 1, (size_t)floor(p * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + (long)i, v.end());
    return v[i];
}

}  // namespace

struct emd_server {
    emd_db* db = nullptr;
    emd_server_options opt{};
    char* pool = nullptr;
    int64_t pool_bytes = 0;
    PoolAllocator alloc;
    std::vector<Slot> slots;
    std::vector<int> free_slots;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    int running = 0;
    std::thread worker;

    // statistics since the last reset
    int64_t submitted = 0, completed = 0, rejected = 0, failed = 0, fallbacks = 0, max_running = 0,
            pool_used_max = 0;
    bool have_first = false;
    Clock::time_point t_first, t_last;
    std::vector<double> lat_us;
};

namespace {

void finish(emd_server* s, Slot& sl, emd_status st, const char* why)
{
    // caller holds s->mu
    Request* r = sl.req;
    r->status = st;
    if (st != EMD_OK) {
        r->err = why ? why : "";
        ++s->failed;
    } else {
        r->out_idx.assign(sl.h_oidx, sl.h_oidx + r->K);
        r->out_dist.assign(sl.h_odist, sl.h_odist + r->K);
        ++s->completed;
        const Clock::time_point now = Clock::now();
        s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
        s->t_last = now;
    }
    r->state = DONE;
    s->alloc.release(r->ws_off, r->ws_bytes);
    sl.req = nullptr;
    sl.fallback = false;
    --s->running;
    s->free_slots.push_back((int)(&sl - s->slots.data()));
    s->cv_done.notify_all();
}

// Issues a request's kernels on its slot (worker thread, s->mu not held).
emd_status launch(emd_server* s, Slot& sl)
{
    emd_db* db = s->db;
    Request* r = sl.req;
    layout(db, r->h, table_width(r->meas, r->k, r->h), s->pool + r->ws_off, &sl.dev);
    memcpy(sl.h_idx, r->idx.data(), (size_t)r->h * 4);
    memcpy(sl.h_w, r->w.data(), (size_t)r->h * 4);
    EMD_CUDA(cudaMemcpyAsync(sl.dev.idx, sl.h_idx, (size_t)r->h * 4, cudaMemcpyHostToDevice, sl.st), "query copy");
    EMD_CUDA(cudaMemcpyAsync(sl.dev.w, sl.h_w, (size_t)r->h * 4, cudaMemcpyHostToDevice, sl.st), "query copy");
    {
        std::lock_guard<std::mutex> lock(db->mu);
        emd_status st;
        if (r->pruned) {
            st = run_topk_pruned(db, sl.dev.L, sl.dev.idx, sl.dev.w, r->h, r->meas, r->k, r->K, sl.dev.ok,
                                 sl.dev.out_idx, sl.dev.out_dist, sl.st);
            if (st == EMD_OK) db->pruned_queries += 1;
        } else {
            st = run_query(db, sl.dev.L, sl.dev.idx, sl.dev.w, r->h, r->meas, r->k, EMD_DIR_MAX, sl.dev.t_out, sl.st);
            if (st == EMD_OK) {
                db->launches[5] += topk_launch_count(db->n);
                db->total_launches += topk_launch_count(db->n);
                EMD_CUDA(launch_topk(sl.dev.t_out, db->n, r->K, sl.dev.L.scratch, sl.dev.out_idx, sl.dev.out_dist,
                                     sl.st), "top-K");
            }
        }
        if (st != EMD_OK) return st;
    }
    EMD_CUDA(cudaMemcpyAsync(sl.h_oidx, sl.dev.out_idx, (size_t)r->K * 8, cudaMemcpyDeviceToHost, sl.st), "result copy");
    EMD_CUDA(cudaMemcpyAsync(sl.h_odist, sl.dev.out_dist, (size_t)r->K * 4, cudaMemcpyDeviceToHost, sl.st), "result copy");
    if (r->pruned)
        EMD_CUDA(cudaMemcpyAsync(sl.h_ok, sl.dev.ok, 4, cudaMemcpyDeviceToHost, sl.st), "flag copy");
    EMD_CUDA(cudaEventRecord(sl.ev, sl.st), "event");
    return EMD_OK;
}

// The unpruned recomputation of a request whose pruning certificate failed.
emd_status launch_fallback(emd_server* s, Slot& sl)
{
    emd_db* db = s->db;
    Request* r = sl.req;
    {
        std::lock_guard<std::mutex> lock(db->mu);
        emd_status st = run_query(db, sl.dev.L, sl.dev.idx, sl.dev.w, r->h, r->meas, r->k, EMD_DIR_MAX,
                                  sl.dev.t_out, sl.st);
        if (st != EMD_OK) return st;
        db->prune_fallbacks += 1;
        db->launches[5] += topk_launch_count(db->n);
        db->total_launches += topk_launch_count(db->n);
        EMD_CUDA(launch_topk(sl.dev.t_out, db->n, r->K, sl.dev.L.scratch, sl.dev.out_idx, sl.dev.out_dist, sl.st),
                 "top-K");
    }
    EMD_CUDA(cudaMemcpyAsync(sl.h_oidx, sl.dev.out_idx, (size_t)r->K * 8, cudaMemcpyDeviceToHost, sl.st), "result copy");
    EMD_CUDA(cudaMemcpyAsync(sl.h_odist, sl.dev.out_dist, (size_t)r->K * 4, cudaMemcpyDeviceToHost, sl.st), "result copy");
    EMD_CUDA(cudaEventRecord(sl.ev, sl.st), "event");
    return EMD_OK;
}

void worker_main(emd_server* s)
{
    cudaSetDevice(s->db->dev);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // admit the head of the queue while a slot and workspace are free
        while (!s->queue.empty() && !s->free_slots.empty()) {
            Request* r = s->queue.front();
            int64_t off = 0;
            if (!s->alloc.alloc(r->ws_bytes, &off)) break;
            s->queue.pop_front();
            r->ws_off = off;
            r->state = RUNNING;
            const int si = s->free_slots.back();
            s->free_slots.pop_back();
            Slot& sl = s->slots[si];
            sl.req = r;
            sl.fallback = false;
            ++s->running;
            s->max_running = std::max<int64_t>(s->max_running, s->running);
            s->pool_used_max = std::max(s->pool_used_max, s->alloc.used());
            lk.unlock();
            emd_status st = launch(s, sl);
            std::string why = st != EMD_OK ? emd_last_error() : "";
            lk.lock();
            if (st != EMD_OK) {
                cudaStreamSynchronize(sl.st);  // nothing of the request may still use its workspace
                finish(s, sl, st, why.c_str());
            }
        }
        if (s->running == 0) {
            if (s->stop && s->queue.empty()) break;
            s->cv_work.wait(lk, [s] { return s->stop || !s->queue.empty(); });
            continue;
        }
        // completions
        bool progressed = false;
        for (Slot& sl : s->slots) {
            if (!sl.req) continue;
            const cudaError_t e = cudaEventQuery(sl.ev);
            if (e == cudaErrorNotReady) continue;
            progressed = true;
            if (e != cudaSuccess) {
                finish(s, sl, EMD_ERR_CUDA, cudaGetErrorString(e));
                continue;
            }
            if (sl.req->pruned && !sl.fallback && !*sl.h_ok) {
                sl.fallback = true;
                ++s->fallbacks;
                lk.unlock();
                emd_status st = launch_fallback(s, sl);
                std::string why = st != EMD_OK ? emd_last_error() : "";
                lk.lock();
                if (st != EMD_OK) {
                    cudaStreamSynchronize(sl.st);
                    finish(s, sl, st, why.c_str());
                }
                continue;
            }
            finish(s, sl, EMD_OK, nullptr);
        }
        if (!progressed) {
            // requests in flight: poll again soon, admitting new arrivals in between
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        }
    }
}

emd_status check_bins(const emd_db* db, const int32_t* idx, const float* w, int h)
{
    std::vector<int32_t> ids(idx, idx + h);
    double sum = 0.0;
    for (int i = 0; i < h; ++i) {
        if (ids[i] < 0 || ids[i] >= db->v) return fail(EMD_ERR_INVALID_ARG, "id %d out of range", ids[i]);
        if (!(w[i] >= 0.f) || !isfinite(w[i])) return fail(EMD_ERR_INVALID_ARG, "weight %g invalid", (double)w[i]);
        sum += w[i];
    }
    if (fabs(sum - 1.0) > 1e-5) return fail(EMD_ERR_INVALID_ARG, "weights sum to %.9g, not 1", sum);
    std::sort(ids.begin(), ids.end());
    for (int i = 1; i < h; ++i)
        if (ids[i] == ids[i - 1]) return fail(EMD_ERR_INVALID_ARG, "id %d repeated", ids[i]);
    return EMD_OK;
}

void destroy_resources(emd_server* s)
{
    for (Slot& sl : s->slots) {
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    if (s->pool) cudaFree(s->pool);
}

}  // namespace

extern "C" {

void emd_server_options_default(emd_server_options* opt)
{
    if (!opt) return;
    opt->max_inflight = 8;
    opt->queue_capacity = 4096;
    opt->workspace_bytes = 0;
    opt->max_query_h = 0;
}

emd_status emd_server_create(emd_db* db, const emd_server_options* opt_in, emd_server** out)
{
    clear_error();
    if (!db || !out) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    emd_server_options opt;
    emd_server_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.max_inflight < 1 || opt.max_inflight > 64) return fail(EMD_ERR_INVALID_ARG, "max_inflight must be 1..64");
    if (opt.queue_capacity < 1) return fail(EMD_ERR_INVALID_ARG, "queue_capacity must be >= 1");
    if (opt.workspace_bytes < 0) return fail(EMD_ERR_INVALID_ARG, "workspace_bytes < 0");
    if (opt.max_query_h == 0) opt.max_query_h = db->opt.max_query_h;
    if (opt.max_query_h < 1 || opt.max_query_h > db->opt.max_query_h)
        return fail(EMD_ERR_INVALID_ARG, "max_query_h must be 1..%d (the database's limit)", db->opt.max_query_h);
    EMD_CUDA(cudaSetDevice(db->dev), "cudaSetDevice");
    auto s = std::make_unique<emd_server>();
    s->db = db;
    s->opt = opt;
    const int tk_max = std::min(db->opt.max_table_k, opt.max_query_h);
    const int64_t per_req = layout(db, opt.max_query_h, tk_max, nullptr, nullptr);
    int64_t bytes = opt.workspace_bytes;
    if (bytes == 0) {
        size_t fr = 0, tot = 0;
        EMD_CUDA(cudaMemGetInfo(&fr, &tot), "memory info");
        bytes = std::min<int64_t>(per_req * opt.max_inflight, (int64_t)(fr / 2));
    }
    bytes = bytes / kAlign * kAlign;
    if (bytes < kAlign) return fail(EMD_ERR_INVALID_ARG, "workspace pool too small");
    cudaError_t e = cudaMalloc(&s->pool, (size_t)bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EMD_ERR_OUT_OF_MEMORY, "workspace pool of %lld bytes: %s", (long long)bytes, cudaGetErrorString(e));
    }
    s->pool_bytes = bytes;
    s->alloc.reset(bytes);
    s->slots.resize((size_t)opt.max_inflight);
    const size_t hbytes = align_up((int64_t)opt.max_query_h * 4) * 2 + kMaxTopK * 8 + kMaxTopK * 4 + 64;
    for (size_t i = 0; i < s->slots.size(); ++i) {
        Slot& sl = s->slots[i];
        e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.pinned, hbytes, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();
            destroy_resources(s.get());
            return fail(e == cudaErrorMemoryAllocation ? EMD_ERR_OUT_OF_MEMORY : EMD_ERR_CUDA, "server slot: %s",
                        cudaGetErrorString(e));
        }
        const int64_t hb = align_up((int64_t)opt.max_query_h * 4);
        sl.h_idx = reinterpret_cast<int32_t*>(sl.pinned);
        sl.h_w = reinterpret_cast<float*>(sl.pinned + hb);
        sl.h_oidx = reinterpret_cast<int64_t*>(sl.pinned + 2 * hb);
        sl.h_odist = reinterpret_cast<float*>(sl.pinned + 2 * hb + kMaxTopK * 8);
        sl.h_ok = reinterpret_cast<int*>(sl.pinned + 2 * hb + kMaxTopK * 12);
        s->free_slots.push_back((int)(s->slots.size() - 1 - i));
    }
    db->servers.fetch_add(1);
    emd_server* raw = s.release();
    raw->worker = std::thread(worker_main, raw);
    *out = raw;
    return EMD_OK;
}

emd_status emd_server_submit(emd_server* s, const int32_t* idx, const float* w, int32_t h_q, emd_measure meas,
                             int32_t k, int32_t K, uint64_t* ticket)
{
    clear_error();
    if (!s || !idx || !w || !ticket) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    const emd_db* db = s->db;
    if (meas < EMD_RWMD || meas > EMD_ICT) return fail(EMD_ERR_INVALID_ARG, "unknown measure %d", meas);
    if (meas == EMD_ACT && k < 1) return fail(EMD_ERR_INVALID_ARG, "k must be >= 1 (got %d)", k);
    if (h_q < 1 || h_q > s->opt.max_query_h)
        return fail(EMD_ERR_INVALID_ARG, "h_q must be 1..%d", s->opt.max_query_h);
    if (K < 1 || K > kMaxTopK || K > db->n) return fail(EMD_ERR_INVALID_ARG, "K must be in 1..min(n_docs, %d)", kMaxTopK);
    const int tk = table_width(meas, k, h_q);
    if (tk > db->opt.max_table_k)
        return fail(EMD_ERR_UNSUPPORTED, "forward table width %d exceeds max_table_k %d", tk, db->opt.max_table_k);
    if (db->approx && rerank_width(db, tk, h_q) > kRerankMax)
        return fail(EMD_ERR_UNSUPPORTED, "re-rank width %d exceeds %d", rerank_width(db, tk, h_q), kRerankMax);
    emd_status st = check_bins(db, idx, w, h_q);
    if (st != EMD_OK) return st;
    auto r = std::make_unique<Request>();
    r->h = h_q;
    r->meas = meas;
    r->k = k;
    r->K = K;
    r->pruned = prunable(db, meas, k, EMD_DIR_MAX, K);
    r->idx.assign(idx, idx + h_q);
    r->w.assign(w, w + h_q);
    r->ws_bytes = layout(db, h_q, tk, nullptr, nullptr);
    if (r->ws_bytes > s->pool_bytes)
        return fail(EMD_ERR_INVALID_ARG, "request needs %lld bytes of workspace, the pool has %lld",
                    (long long)r->ws_bytes, (long long)s->pool_bytes);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return fail(EMD_ERR_SHUTDOWN, "server is shutting down");
        if ((int64_t)s->queue.size() >= s->opt.queue_capacity) {
            ++s->rejected;
            return fail(EMD_ERR_BUSY, "submit queue full (%d requests)", s->opt.queue_capacity);
        }
        r->ticket = s->next_ticket++;
        r->t_submit = Clock::now();
        if (!s->have_first) {
            s->have_first = true;
            s->t_first = r->t_submit;
        }
        ++s->submitted;
        *ticket = r->ticket;
        s->queue.push_back(r.get());
        s->reqs.emplace(r->ticket, std::move(r));
    }
    s->cv_work.notify_one();
    return EMD_OK;
}

emd_status emd_server_poll(emd_server* s, uint64_t ticket, int32_t timeout_ms, int64_t* out_idx, float* out_dist)
{
    clear_error();
    if (!s || !out_idx || !out_dist) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(EMD_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Request* r = it->second.get();
    auto ready = [r] { return r->state == DONE; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, ready);
    else if (timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    if (!ready()) return fail(EMD_ERR_TIMEOUT, "request %llu not finished", (unsigned long long)ticket);
    const emd_status st = r->status;
    std::string why = r->err;
    if (st == EMD_OK) {
        std::copy(r->out_idx.begin(), r->out_idx.end(), out_idx);
        std::copy(r->out_dist.begin(), r->out_dist.end(), out_dist);
    }
    s->reqs.erase(it);
    if (st != EMD_OK) return fail(st, "request failed: %s", why.c_str());
    return EMD_OK;
}

emd_status emd_server_stats_get(emd_server* s, emd_server_stats* out)
{
    clear_error();
    if (!s || !out) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        out->submitted = s->submitted;
        out->completed = s->completed;
        out->rejected_busy = s->rejected;
        out->failed = s->failed;
        out->prune_fallbacks = s->fallbacks;
        out->queued = (int64_t)s->queue.size();
        out->in_flight = s->running;
        out->max_in_flight = s->max_running;
        out->pool_bytes = s->pool_bytes;
        out->pool_used_max = s->pool_used_max;
        const double span = s->have_first && s->completed
                                ? std::chrono::duration<double>(s->t_last - s->t_first).count()
                                : 0.0;
        out->qps = span > 0 ? (double)s->completed / span : 0.0;
        lat = s->lat_us;
    }
    out->latency_p50_us = pct(lat, 0.50);
    out->latency_p99_us = pct(lat, 0.99);
    double sum = 0.0, mx = 0.0;
    for (double x : lat) { sum += x; mx = std::max(mx, x); }
    out->latency_mean_us = lat.empty() ? 0.0 : sum / (double)lat.size();
    out->latency_max_us = mx;
    return EMD_OK;
}

emd_status emd_server_stats_reset(emd_server* s)
{
    clear_error();
    if (!s) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    s->submitted = s->completed = s->rejected = s->failed = s->fallbacks = 0;
    s->max_running = s->running;
    s->pool_used_max = s->alloc.used();
    s->have_first = false;
    s->lat_us.clear();
    return EMD_OK;
}

emd_status emd_server_destroy(emd_server* s)
{
    clear_error();
    if (!s) return EMD_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->db->dev);
    for (Slot& sl : s->slots)
        if (sl.st) cudaStreamSynchronize(sl.st);
    destroy_resources(s);
    s->db->servers.fetch_sub(1);
    delete s;
    return EMD_OK;
}

}  // extern "C"
