// Serving (include/emd.h, emd_server_*): a request loop over a resident database.
//
// Requests are single queries.  A worker thread forms batches from the head of the queue
// and runs each on one of two executors -- a batch workspace of its own, pinned staging
// and a stream -- with the same batched kernel sequence as the host entry points (Phase 1,
// table, forward pass, pruned reverse pass and top-K of Sections 5-6, replayed from a
// captured graph).  While one batch is on the GPU the next one collects the requests that
// arrived meanwhile (continuous batching), admitted in arrival order as long as the
// executor's workspace -- its distance-matrix columns, i.e. device memory -- can hold them.
// The batched kernels compute every query exactly as the per-query ones do (no sum or
// selection crosses queries), so a result is the same alone and in any mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
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

constexpr int kExecs = 2;

enum ReqState { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct Request {
    uint64_t ticket = 0;
    int h = 0, meas = 0, k = 0, K = 0;
    bool pruned = false;
    std::vector<int32_t> idx;
    std::vector<float> w;
    Clock::time_point t_submit;
    int state = QUEUED;
    emd_status status = EMD_OK;
    std::string err;
    std::vector<int64_t> out_idx;
    std::vector<float> out_dist;
};

// One batch executor.
struct Exec {
    BatchWS ws;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    char* pinned = nullptr;  // rp | idx | w | out_idx | out_dist | ok
    int64_t* h_rp = nullptr;
    int32_t* h_idx = nullptr;
    float* h_w = nullptr;
    int64_t* h_oidx = nullptr;
    float* h_odist = nullptr;
    int* h_ok = nullptr;
    int* h_over = nullptr;          // ICT table overflow flags
    int32_t* d_idx = nullptr;
    float* d_w = nullptr;
    int64_t* d_oidx = nullptr;
    float* d_odist = nullptr;
    std::vector<Request*> batch;
    int meas = 0, k = 0, K = 0;
    bool pruned = false;
    int64_t cols = 0;
    bool busy = false;
};

double pct(std::vector<double> v, double p)
{
    if (v.empty()) return 0.0;
    const size_t i = std::min(v.size() - 1, (size_t)floor(p * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + (long)i, v.end());
    return v[i];
}

int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct emd_server {
    emd_db* db = nullptr;
    emd_server_options opt{};
    Exec ex[kExecs];
    Lane fb;                        // per-query workspace for uncertified pruned requests
    float* fb_out = nullptr;        // its n symmetric distances
    std::vector<void*> allocs;      // device memory of the executors and the fallback lane
    int64_t bytes = 0, pool_bytes = 0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    int in_flight = 0;
    std::thread worker;

    // statistics since the last reset
    int64_t submitted = 0, completed = 0, rejected = 0, failed = 0, fallbacks = 0, max_running = 0,
            pool_used_max = 0;
    bool have_first = false;
    Clock::time_point t_first, t_last;
    std::vector<double> lat_us;
};

namespace {

template <typename T>
emd_status sdal(emd_server* s, T** p, int64_t count)
{
    const size_t nb = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, nb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EMD_ERR_OUT_OF_MEMORY, "server: cudaMalloc of %zu bytes failed", nb);
    }
    s->allocs.push_back(q);
    s->bytes += (int64_t)nb;
    *p = static_cast<T*>(q);
    return EMD_OK;
}

void destroy_resources(emd_server* s)
{
    for (Exec& e : s->ex) {
        free_batch_ws(e.ws);
        if (e.done) cudaEventDestroy(e.done);
        if (e.st) cudaStreamDestroy(e.st);
        if (e.pinned) cudaFreeHost(e.pinned);
    }
    for (void* p : s->allocs) cudaFree(p);
    s->allocs.clear();
}

// Marks every request of the executor's batch finished (caller holds s->mu).
void finish_batch(emd_server* s, Exec& e, emd_status st, const char* why)
{
    const Clock::time_point now = Clock::now();
    for (size_t i = 0; i < e.batch.size(); ++i) {
        Request* r = e.batch[i];
        r->status = st;
        if (st != EMD_OK) {
            r->err = why ? why : "";
            ++s->failed;
        } else {
            r->out_idx.assign(e.h_oidx + i * r->K, e.h_oidx + (i + 1) * r->K);
            r->out_dist.assign(e.h_odist + i * r->K, e.h_odist + (i + 1) * r->K);
            ++s->completed;
            s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
            s->t_last = now;
        }
        r->state = DONE;
    }
    s->in_flight -= (int)e.batch.size();
    e.batch.clear();
    e.busy = false;
    s->cv_done.notify_all();
}

// Stages the batch's bins and issues its kernels and result copies (worker thread, s->mu
// not held).
// ICT batches whose tables can overflow (FP32 distances) report per-request flags.
bool ict_batch(const emd_db* db, const Exec& e) { return e.meas == M_ICT && !db->approx; }

emd_status launch_batch(emd_server* s, Exec& e)
{
    emd_db* db = s->db;
    const int nb = (int)e.batch.size();
    int64_t bins = 0;
    e.h_rp[0] = 0;
    for (int i = 0; i < nb; ++i) {
        const Request* r = e.batch[(size_t)i];
        memcpy(e.h_idx + bins, r->idx.data(), (size_t)r->h * 4);
        memcpy(e.h_w + bins, r->w.data(), (size_t)r->h * 4);
        bins += r->h;
        e.h_rp[i + 1] = bins;
    }
    EMD_CUDA(cudaMemcpyAsync(e.d_idx, e.h_idx, (size_t)bins * 4, cudaMemcpyHostToDevice, e.st), "query copy");
    EMD_CUDA(cudaMemcpyAsync(e.d_w, e.h_w, (size_t)bins * 4, cudaMemcpyHostToDevice, e.st), "query copy");
    {
        std::lock_guard<std::mutex> lock(db->mu);
        emd_status st = run_subbatch(db, e.ws, e.h_rp, e.d_idx, e.d_w, 0, 0, nb, e.meas, e.k, EMD_DIR_MAX, e.K,
                                     e.pruned, nullptr, e.d_oidx, e.d_odist, e.st);
        if (st != EMD_OK) return st;
        if (e.pruned) db->pruned_queries += nb;
    }
    EMD_CUDA(cudaMemcpyAsync(e.h_oidx, e.d_oidx, (size_t)nb * e.K * 8, cudaMemcpyDeviceToHost, e.st), "result copy");
    EMD_CUDA(cudaMemcpyAsync(e.h_odist, e.d_odist, (size_t)nb * e.K * 4, cudaMemcpyDeviceToHost, e.st),
             "result copy");
    if (e.pruned)
        EMD_CUDA(cudaMemcpyAsync(e.h_ok, e.ws.cand_ok, (size_t)nb * 4, cudaMemcpyDeviceToHost, e.st), "flag copy");
    if (ict_batch(db, e))
        EMD_CUDA(cudaMemcpyAsync(e.h_over, e.ws.ict_over, (size_t)nb * 4, cudaMemcpyDeviceToHost, e.st), "flag copy");
    EMD_CUDA(cudaEventRecord(e.done, e.st), "event");
    return EMD_OK;
}

// Recomputes over all documents, in place in the pinned results, the batch's uncertified
// pruned requests and its ICT requests whose table overflowed (both rare; ICT with tables of
// full width); *count receives how many.
emd_status run_fallbacks(emd_server* s, Exec& e, int* count)
{
    emd_db* db = s->db;
    *count = 0;
    const bool ict = ict_batch(db, e);
    if (!e.pruned && !ict) return EMD_OK;
    for (size_t i = 0; i < e.batch.size(); ++i) {
        const bool over = ict && e.h_over[i];
        const Request* r = e.batch[i];
        if (!over && e.pruned && e.h_ok[i] == 2) {  // the fused candidate block overflowed
            {
                std::lock_guard<std::mutex> lock(db->mu);
                ++db->fused_retries;
                emd_status st = retry_materialized(db, e.ws, e.h_rp, e.d_idx, e.d_w, 0, (int64_t)i, r->meas, r->k,
                                                   r->K, e.d_oidx, e.d_odist, e.st, &e.h_ok[i]);
                if (st != EMD_OK) return st;
            }
            if (e.h_ok[i] == 1) {
                EMD_CUDA(cudaMemcpyAsync(e.h_oidx + i * r->K, e.d_oidx + i * r->K, (size_t)r->K * 8,
                                         cudaMemcpyDeviceToHost, e.st),
                         "result copy");
                EMD_CUDA(cudaMemcpyAsync(e.h_odist + i * r->K, e.d_odist + i * r->K, (size_t)r->K * 4,
                                         cudaMemcpyDeviceToHost, e.st),
                         "result copy");
                EMD_CUDA(cudaStreamSynchronize(e.st), "synchronize");
                continue;
            }
        }
        if (!over && (!e.pruned || e.h_ok[i] == 1)) continue;
        const int64_t off = e.h_rp[i];
        {
            std::lock_guard<std::mutex> lock(db->mu);
            emd_status st = run_query(db, s->fb, e.d_idx + off, e.d_w + off, r->h, r->meas, r->k, EMD_DIR_MAX,
                                      s->fb_out, nullptr, e.st);
            if (st != EMD_OK) return st;
            EMD_CUDA(launch_topk(s->fb_out, db->n, r->K, s->fb.scratch, e.d_oidx + i * r->K, e.d_odist + i * r->K,
                                 e.st),
                     "top-K");
            if (over) db->ict_wide += 1; else db->prune_fallbacks += 1;
        }
        EMD_CUDA(cudaMemcpyAsync(e.h_oidx + i * r->K, e.d_oidx + i * r->K, (size_t)r->K * 8, cudaMemcpyDeviceToHost,
                                 e.st),
                 "result copy");
        EMD_CUDA(cudaMemcpyAsync(e.h_odist + i * r->K, e.d_odist + i * r->K, (size_t)r->K * 4,
                                 cudaMemcpyDeviceToHost, e.st),
                 "result copy");
        EMD_CUDA(cudaStreamSynchronize(e.st), "synchronize");
        ++*count;
    }
    return EMD_OK;
}

// Takes the batch for executor e from the head of the queue: requests with the head's
// (measure, k, K), in arrival order, while the executor's workspace and the in-flight limit
// allow (caller holds s->mu).
void form_batch(emd_server* s, Exec& e)
{
    const Request* head = s->queue.front();
    e.meas = head->meas;
    e.k = head->k;
    e.K = head->K;
    e.pruned = head->pruned;
    std::vector<int64_t> rp(1, 0);
    while (!s->queue.empty() && (int)e.batch.size() < e.ws.max_batch && s->in_flight < s->opt.max_inflight) {
        Request* r = s->queue.front();
        if (r->meas != e.meas || r->k != e.k || r->K != e.K) break;
        rp.push_back(rp.back() + r->h);
        if (!batch_fits(s->db, e.ws, rp.data(), 0, (int64_t)rp.size() - 1, e.meas, e.k, EMD_DIR_MAX)) break;
        s->queue.pop_front();
        r->state = RUNNING;
        e.batch.push_back(r);
        ++s->in_flight;
    }
    e.cols = 0;
    for (const Request* r : e.batch) e.cols += round_up(r->h, 32);
    e.busy = true;
    s->max_running = std::max<int64_t>(s->max_running, s->in_flight);
    s->pool_used_max = std::max<int64_t>(s->pool_used_max, e.cols * 4 * s->db->v_used);
}

void worker_main(emd_server* s)
{
    cudaSetDevice(s->db->dev);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // launch batches on free executors
        for (Exec& e : s->ex) {
            if (e.busy || s->queue.empty() || s->in_flight >= s->opt.max_inflight) continue;
            form_batch(s, e);
            lk.unlock();
            const emd_status st = launch_batch(s, e);
            const std::string why = st != EMD_OK ? emd_last_error() : "";
            lk.lock();
            if (st != EMD_OK) {
                cudaStreamSynchronize(e.st);
                finish_batch(s, e, st, why.c_str());
            }
        }
        bool busy = false;
        for (Exec& e : s->ex) busy |= e.busy;
        if (!busy) {
            if (s->stop && s->queue.empty()) break;
            s->cv_work.wait(lk, [s] { return s->stop || !s->queue.empty(); });
            continue;
        }
        // completions
        bool progressed = false;
        for (Exec& e : s->ex) {
            if (!e.busy) continue;
            const cudaError_t q = cudaEventQuery(e.done);
            if (q == cudaErrorNotReady) continue;
            progressed = true;
            if (q != cudaSuccess) {
                finish_batch(s, e, EMD_ERR_CUDA, cudaGetErrorString(q));
                continue;
            }
            lk.unlock();
            int nfb = 0;
            const emd_status st = run_fallbacks(s, e, &nfb);
            const std::string why = st != EMD_OK ? emd_last_error() : "";
            lk.lock();
            s->fallbacks += nfb;
            finish_batch(s, e, st, why.c_str());
        }
        if (!progressed) {
            // batches in flight: poll again soon, admitting new arrivals in between
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

// Per-query workspace of the fallback lane (sizes as the handle's own lanes).
emd_status alloc_lane(emd_server* s, Lane& L)
{
    emd_db* db = s->db;
    const int64_t npad = round_up(s->opt.max_query_h, 128);
    const int64_t ldd = round_up(s->opt.max_query_h, 32);
    const int64_t qrows = round_up(ldd, kDistBN);
    emd_status st;
#define TRYL(x)                               \
    do {                                      \
        if ((st = (x)) != EMD_OK) return st;  \
    } while (0)
    if (!db->cost_mode) {
        TRYL(sdal(s, &L.Q, qrows * db->ldm));
        TRYL(sdal(s, &L.qnorm, qrows));
        if (db->tc) {
            TRYL(sdal(s, &L.q_hi, npad * db->kpad));
            if (db->tcfmt == TC_SPLIT) TRYL(sdal(s, &L.q_lo, npad * db->kpad));
            TRYL(sdal(s, &L.q_scale, npad));
        }
    }
    TRYL(sdal(s, &L.D, db->v_used * ldd));
    TRYL(sdal(s, &L.tab, db->v_used * db->opt.max_table_k));
    TRYL(sdal(s, &L.t_fwd, db->n));
    TRYL(sdal(s, &L.t_rev, db->n));
    TRYL(sdal(s, &L.sel_idx, kPruneMaxK));
    TRYL(sdal(s, &L.sel_val, kPruneMaxK));
    TRYL(sdal(s, &L.cand_idx, kPruneCap));
    TRYL(sdal(s, &L.cand_sym, 2 * kPruneCap));
    TRYL(sdal(s, &L.cand_count, 1));
    TRYL(sdal(s, &L.scratch, kTopkScratchRow));
#undef TRYL
    return EMD_OK;
}

}  // namespace

extern "C" {

void emd_server_options_default(emd_server_options* opt)
{
    if (!opt) return;
    opt->max_inflight = 128;
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
    if (opt.max_inflight < 1) return fail(EMD_ERR_INVALID_ARG, "max_inflight must be >= 1");
    if (opt.queue_capacity < 1) return fail(EMD_ERR_INVALID_ARG, "queue_capacity must be >= 1");
    if (opt.workspace_bytes < 0) return fail(EMD_ERR_INVALID_ARG, "workspace_bytes < 0");
    if (opt.max_query_h == 0) opt.max_query_h = db->opt.max_query_h;
    if (opt.max_query_h < 1 || opt.max_query_h > db->opt.max_query_h)
        return fail(EMD_ERR_INVALID_ARG, "max_query_h must be 1..%d (the database's limit)", db->opt.max_query_h);
    // distance-matrix columns per executor: the pool split in two, at least one request
    const int64_t col_bytes = 4 * db->v_used;
    const int64_t min_cols = round_up(opt.max_query_h, 32);
    const int64_t cols = opt.workspace_bytes > 0 ? (opt.workspace_bytes / kExecs) / col_bytes / 32 * 32
                                                 : std::max<int64_t>(db->opt.batch_columns, min_cols);
    if (cols < min_cols)
        return fail(EMD_ERR_INVALID_ARG, "workspace_bytes too small: %lld bytes hold less than one request of %d bins",
                    (long long)opt.workspace_bytes, opt.max_query_h);
    EMD_CUDA(cudaSetDevice(db->dev), "cudaSetDevice");
    auto s = std::make_unique<emd_server>();
    s->db = db;
    s->opt = opt;
    const int mb = std::min(db->opt.max_batch, opt.max_inflight);
    emd_status st = EMD_OK;
    for (Exec& e : s->ex) {
        int64_t wsb = 0;
        st = alloc_batch_ws(db, e.ws, mb, cols, s->allocs, &wsb);
        s->bytes += wsb;
        s->pool_bytes += e.ws.b_cols * col_bytes;
        if (st == EMD_OK) st = sdal(s.get(), &e.d_idx, e.ws.b_cols);
        if (st == EMD_OK) st = sdal(s.get(), &e.d_w, e.ws.b_cols);
        if (st == EMD_OK) st = sdal(s.get(), &e.d_oidx, (int64_t)mb * kMaxTopK);
        if (st == EMD_OK) st = sdal(s.get(), &e.d_odist, (int64_t)mb * kMaxTopK);
        cudaError_t ce = cudaSuccess;
        const int64_t hb = align256(8 * ((int64_t)mb + 1)) + 2 * align256(4 * e.ws.b_cols) +
                           align256(8 * (int64_t)mb * kMaxTopK) + align256(4 * (int64_t)mb * kMaxTopK) +
                           2 * align256(4 * (int64_t)mb);
        if (st == EMD_OK) ce = cudaStreamCreateWithFlags(&e.st, cudaStreamNonBlocking);
        if (st == EMD_OK && ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming);
        if (st == EMD_OK && ce == cudaSuccess) ce = cudaHostAlloc((void**)&e.pinned, (size_t)hb, cudaHostAllocDefault);
        if (st == EMD_OK && ce != cudaSuccess) {
            cudaGetLastError();
            st = fail(EMD_ERR_OUT_OF_MEMORY, "server executor: %s", cudaGetErrorString(ce));
        }
        if (st != EMD_OK) {
            destroy_resources(s.get());
            return st;
        }
        char* p = e.pinned;
        e.h_rp = reinterpret_cast<int64_t*>(p);
        p += align256(8 * ((int64_t)mb + 1));
        e.h_idx = reinterpret_cast<int32_t*>(p);
        p += align256(4 * e.ws.b_cols);
        e.h_w = reinterpret_cast<float*>(p);
        p += align256(4 * e.ws.b_cols);
        e.h_oidx = reinterpret_cast<int64_t*>(p);
        p += align256(8 * (int64_t)mb * kMaxTopK);
        e.h_odist = reinterpret_cast<float*>(p);
        p += align256(4 * (int64_t)mb * kMaxTopK);
        e.h_ok = reinterpret_cast<int*>(p);
        p += align256(4 * (int64_t)mb);
        e.h_over = reinterpret_cast<int*>(p);
    }
    if ((st = alloc_lane(s.get(), s->fb)) != EMD_OK || (st = sdal(s.get(), &s->fb_out, db->n)) != EMD_OK) {
        destroy_resources(s.get());
        return st;
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
    const int tk = table_width(db, meas, k, h_q);
    if (tk > db->opt.max_table_k)
        return fail(EMD_ERR_UNSUPPORTED, "forward table width %d exceeds max_table_k %d", tk, db->opt.max_table_k);
    if (db->approx && rerank_width(db, tk, h_q) > kRerankMax)
        return fail(EMD_ERR_UNSUPPORTED, "re-rank width %d exceeds %d", rerank_width(db, tk, h_q), kRerankMax);
    const int64_t one[2] = {0, h_q};
    if (!batch_fits(db, s->ex[0].ws, one, 0, 1, meas, k, EMD_DIR_MAX))
        return fail(EMD_ERR_INVALID_ARG, "the request does not fit an executor's workspace");
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
        out->in_flight = s->in_flight;
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
    s->max_running = s->in_flight;
    s->pool_used_max = 0;
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
    for (Exec& e : s->ex)
        if (e.st) cudaStreamSynchronize(e.st);
    destroy_resources(s);
    s->db->servers.fetch_sub(1);
    delete s;
    return EMD_OK;
}

}  // extern "C"
