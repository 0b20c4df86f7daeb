/*
 * orbg_serve.cpp -- continuous-batching decode server over a code set.
 *
 * Requests (a code index and B blocks of LLRs) arrive at any time through
 * orbg_server_submit.  A dispatcher thread owns the device side:
 *   - admission: pending requests are packed, first come first served, into
 *     the next batch while the batch's footprint (LLRs, outputs, per-block
 *     layout arrays and the batched kernels' scratch) still fits the free
 *     part of a device pool of mem_budget bytes and of a pinned host pool of
 *     the same size; a request waits on the host until it fits;
 *   - each batch is one mixed-code orbg batched decode (the same kernels as
 *     orbg_decode_batched) on one of several streams: H2D copy of the
 *     batch's inputs, the two kernels, D2H copy of its outputs, an event;
 *     batches on different streams overlap on the GPU, and requests that
 *     arrive while batches run go into the next batch as soon as a stream
 *     and pool space are free;
 *   - completion is seen by polling the batches' events; the results of
 *     each request are copied out of the pinned pool and the batch's pool
 *     space is returned.
 * The code tables stay resident on the device for the server's life.
 * Nothing here waits on the GPU except cudaEventQuery polls and the final
 * drain in orbg_server_destroy.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/orbg.h"
#include "orbg_internal.h"
#include "orbg_regions.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Request {
    uint64_t id;
    int code;
    int64_t B;
    int n;
    std::vector<float> llr;
    std::vector<uint8_t> cw;
    std::vector<uint32_t> q;
    std::vector<uint8_t> ab;
    double t_submit = 0, t_done = 0;
    bool cancelled = false; /* in a batch when cancelled: dropped when it retires */
};

/* Byte layout of one batch; identical in the device and the pinned pool. */
struct Layout {
    size_t llr, code_id, llr_off, cw_off, in_end;
    size_t cw, q, ab, out_end;
    size_t scratch, total;
    static Layout make(int64_t B, size_t n_llr)
    {
        Layout L;
        size_t o = 0;
        L.llr = o;
        o = align_up(o + n_llr * sizeof(float), 256);
        L.code_id = o;
        o = align_up(o + (size_t)B * sizeof(int32_t), 256);
        L.llr_off = o;
        o = align_up(o + (size_t)B * sizeof(int64_t), 256);
        L.cw_off = o;
        o = align_up(o + (size_t)B * sizeof(int64_t), 256);
        L.in_end = o;
        L.cw = o;
        o = align_up(o + n_llr, 256);
        L.q = o;
        o = align_up(o + (size_t)B * sizeof(uint32_t), 256);
        L.ab = o;
        o = align_up(o + (size_t)B, 256);
        L.out_end = o;
        L.scratch = o;
        o = align_up(o + orbg_batched_scratch_bytes(B, ORBG_MAX_CODES), 256);
        L.total = o;
        return L;
    }
};

struct Batch {
    std::vector<Request *> reqs;
    int64_t B = 0;
    size_t n_llr = 0;
    Layout L;
    size_t dev_off = 0, pin_off = 0;
    int stream = 0;
    cudaEvent_t done = nullptr;
};

}  // namespace

struct orbg_server {
    const orbg_codeset *set = nullptr;
    OrbgSetView view;
    std::vector<int> n_of;
    uint32_t cap = 0;
    int device = 0;
    size_t budget = 0;
    int64_t max_batch_blocks = 0;
    unsigned char *d_pool = nullptr;
    unsigned char *h_pool = nullptr;
    orbg_host::Regions *dreg = nullptr, *hreg = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<char> stream_busy;
    std::deque<Request *> pending;
    std::deque<Batch> inflight;
    std::unordered_map<uint64_t, Request *> done;
    std::deque<uint64_t> done_order;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread th;
    bool stop = false;
    int error = 0;
    orbg_server_stats stats;
};

namespace {

size_t request_footprint(int64_t B, int n)
{
    return Layout::make(B, (size_t)B * (size_t)n).total;
}

/* Copies finished batches' results out; caller holds the lock. */
void retire(orbg_server *s)
{
    for (auto it = s->inflight.begin(); it != s->inflight.end();) {
        cudaError_t e = cudaEventQuery(it->done);
        if (e == cudaErrorNotReady) {
            ++it;
            continue;
        }
        if (e != cudaSuccess && !s->error)
            s->error = orbg_note_cuda_error((int)e);
        const unsigned char *h = s->h_pool + it->pin_off;
        const uint8_t *cw = h + it->L.cw;
        const uint32_t *q = reinterpret_cast<const uint32_t *>(h + it->L.q);
        const uint8_t *ab = h + it->L.ab;
        int64_t b = 0;
        size_t off = 0;
        const double t = now_s();
        for (Request *r : it->reqs) {
            const size_t nb = (size_t)r->B * r->n;
            if (r->cancelled) {
                b += r->B;
                off += nb;
                delete r;
                continue;
            }
            r->cw.assign(cw + off, cw + off + nb);
            r->q.assign(q + b, q + b + r->B);
            r->ab.assign(ab + b, ab + b + r->B);
            r->llr.clear();
            r->llr.shrink_to_fit();
            r->t_done = t;
            s->done[r->id] = r;
            s->done_order.push_back(r->id);
            b += r->B;
            off += nb;
            s->stats.completed += 1;
        }
        s->stats.blocks_done += (uint64_t)it->B;
        s->dreg->release(it->dev_off, it->L.total);
        s->hreg->release(it->pin_off, it->L.total);
        s->stream_busy[it->stream] = 0;
        cudaEventDestroy(it->done);
        it = s->inflight.erase(it);
        s->cv_done.notify_all();
    }
}

/* Forms and launches one batch from the pending queue; false if nothing
 * could be admitted.  Caller holds the lock. */
bool dispatch_one(orbg_server *s)
{
    int stream = -1;
    for (size_t i = 0; i < s->streams.size(); i++)
        if (!s->stream_busy[i]) {
            stream = (int)i;
            break;
        }
    if (stream < 0 || s->pending.empty())
        return false;
    /* take requests in arrival order while the batch still fits */
    Batch bt;
    size_t take = 0;
    int64_t B = 0;
    size_t n_llr = 0;
    size_t best_dev = 0, best_pin = 0;
    Layout bestL;
    bool have = false;
    for (size_t i = 0; i < s->pending.size(); i++) {
        const Request *r = s->pending[i];
        const int64_t B2 = B + r->B;
        const size_t n2 = n_llr + (size_t)r->B * r->n;
        if (have && B2 > s->max_batch_blocks)
            break;
        Layout L = Layout::make(B2, n2);
        size_t doff, hoff;
        if (!s->dreg->alloc(L.total, &doff))
            break;
        if (!s->hreg->alloc(L.total, &hoff)) {
            s->dreg->release(doff, L.total);
            break;
        }
        if (have) {
            s->dreg->release(best_dev, bestL.total);
            s->hreg->release(best_pin, bestL.total);
        }
        best_dev = doff;
        best_pin = hoff;
        bestL = L;
        have = true;
        take = i + 1;
        B = B2;
        n_llr = n2;
    }
    if (!have)
        return false;
    bt.L = bestL;
    bt.dev_off = best_dev;
    bt.pin_off = best_pin;
    bt.B = B;
    bt.n_llr = n_llr;
    bt.stream = stream;
    bt.reqs.assign(s->pending.begin(), s->pending.begin() + (long)take);
    s->pending.erase(s->pending.begin(), s->pending.begin() + (long)take);

    /* stage inputs in the pinned pool */
    unsigned char *h = s->h_pool + bt.pin_off;
    float *llr = reinterpret_cast<float *>(h + bt.L.llr);
    int32_t *cid = reinterpret_cast<int32_t *>(h + bt.L.code_id);
    int64_t *lo = reinterpret_cast<int64_t *>(h + bt.L.llr_off);
    int64_t *co = reinterpret_cast<int64_t *>(h + bt.L.cw_off);
    int64_t b = 0;
    size_t off = 0;
    for (Request *r : bt.reqs) {
        std::memcpy(llr + off, r->llr.data(), sizeof(float) * (size_t)r->B * r->n);
        for (int64_t i = 0; i < r->B; i++) {
            cid[b + i] = r->code;
            lo[b + i] = (int64_t)(off + (size_t)i * r->n);
            co[b + i] = (int64_t)(off + (size_t)i * r->n);
        }
        b += r->B;
        off += (size_t)r->B * r->n;
    }
    OrbgRange range("orbg_server batch");
    unsigned char *d = s->d_pool + bt.dev_off;
    cudaStream_t st = s->streams[stream];
    cudaError_t e = cudaMemcpyAsync(d, h, bt.L.in_end, cudaMemcpyHostToDevice, st);
    const uint32_t budget = s->view.tuning.warp_budget < s->cap ? s->view.tuning.warp_budget
                                                                : s->cap;
    int le = 0;
    if (e == cudaSuccess) {
        OrbgBatchedArgs a{};
        a.d_codes = s->view.d_codes;
        a.code0 = nullptr; /* requests mix codes: per-block code ids */
        a.ncodes = s->view.ncodes;
        a.n_max = s->view.n_max;
        a.var = s->view.var;
        a.has_stride = s->view.has_stride;
        a.w32_max = s->view.w32_max;
        a.code_id = reinterpret_cast<const int32_t *>(d + bt.L.code_id);
        a.llr_off = reinterpret_cast<const int64_t *>(d + bt.L.llr_off);
        a.llr = reinterpret_cast<const float *>(d + bt.L.llr);
        a.B = bt.B;
        a.cap = s->cap;
        a.budget = budget;
        a.cw = d + bt.L.cw;
        a.cw_off = reinterpret_cast<const int64_t *>(d + bt.L.cw_off);
        a.q = reinterpret_cast<uint32_t *>(d + bt.L.q);
        a.ab = d + bt.L.ab;
        a.scratch = reinterpret_cast<unsigned long long *>(d + bt.L.scratch);
        a.warps_per_cta = s->view.tuning.warps_per_cta;
        a.ctas_per_sm = s->view.tuning.ctas_per_sm;
        a.grab = s->view.tuning.blocks_per_grab;
        a.heavy_warps = s->view.tuning.heavy_warps;
        a.ntrip_max = s->view.ntrip_max;
        a.x3w_max = s->view.x3w_max;
        a.stream = st;
        le = orbg_launch_batched(a);
    }
    if (e == cudaSuccess && le != 0)
        e = (cudaError_t)le;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h + bt.L.cw, d + bt.L.cw, bt.L.out_end - bt.L.cw,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&bt.done, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventRecord(bt.done, st);
    if (e != cudaSuccess) {
        if (!s->error)
            s->error = orbg_note_cuda_error((int)e);
        /* give the requests back as failed: abandoned flag 2, no queries */
        for (Request *r : bt.reqs) {
            r->cw.assign((size_t)r->B * r->n, 0);
            r->q.assign((size_t)r->B, 0);
            r->ab.assign((size_t)r->B, 2);
            r->t_done = now_s();
            s->done[r->id] = r;
            s->done_order.push_back(r->id);
        }
        if (bt.done)
            cudaEventDestroy(bt.done);
        s->dreg->release(bt.dev_off, bt.L.total);
        s->hreg->release(bt.pin_off, bt.L.total);
        s->cv_done.notify_all();
        return false;
    }
    s->stream_busy[stream] = 1;
    s->stats.batches += 1;
    s->stats.max_batch_blocks = std::max<uint64_t>(s->stats.max_batch_blocks, (uint64_t)bt.B);
    s->inflight.push_back(std::move(bt));
    s->stats.max_inflight_batches =
        std::max<uint64_t>(s->stats.max_inflight_batches, (uint64_t)s->inflight.size());
    return true;
}

void dispatcher(orbg_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        retire(s);
        while (dispatch_one(s)) {
        }
        if (s->stop && s->pending.empty() && s->inflight.empty())
            break;
        /* short sleeps while batches run; longer when idle */
        s->cv_work.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 2000 : 20));
    }
}

}  // namespace

extern "C" {

int orbg_server_create(const orbg_codeset *set, size_t mem_budget_bytes, uint32_t query_cap,
                       int streams, int64_t max_batch_blocks, orbg_server **out)
{
    if (!out)
        return ORBG_EINVAL;
    *out = nullptr;
    OrbgSetView v;
    if (!set || orbg_codeset_view(set, &v) != 0 || query_cap < 1 || streams < 0 ||
        streams > 16 || max_batch_blocks < 0)
        return ORBG_EINVAL;
    if (query_cap > v.cap_min)
        return ORBG_ELIMIT;
    orbg_server *s = new (std::nothrow) orbg_server();
    if (!s)
        return ORBG_ENOMEM;
    s->set = set;
    s->view = v;
    s->cap = query_cap;
    s->budget = mem_budget_bytes ? mem_budget_bytes : ((size_t)1 << 30);
    s->max_batch_blocks = max_batch_blocks ? max_batch_blocks : (int64_t)1 << 20;
    std::memset(&s->stats, 0, sizeof(s->stats));
    orbg_codeset_lengths(set, &s->n_of);
    cudaError_t e = cudaGetDevice(&s->device);
    const int ns = streams ? streams : 4;
    if (e == cudaSuccess)
        e = cudaMalloc(&s->d_pool, s->budget);
    if (e == cudaSuccess)
        e = cudaHostAlloc(&s->h_pool, s->budget, cudaHostAllocDefault);
    for (int i = 0; i < ns && e == cudaSuccess; i++) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            s->streams.push_back(st);
    }
    if (e != cudaSuccess) {
        int rc = orbg_note_cuda_error((int)e);
        for (cudaStream_t st : s->streams)
            cudaStreamDestroy(st);
        if (s->d_pool) cudaFree(s->d_pool);
        if (s->h_pool) cudaFreeHost(s->h_pool);
        delete s;
        return rc;
    }
    s->stream_busy.assign(s->streams.size(), 0);
    s->dreg = new orbg_host::Regions(s->budget);
    s->hreg = new orbg_host::Regions(s->budget);
    s->th = std::thread(dispatcher, s);
    *out = s;
    return ORBG_OK;
}

int orbg_server_submit(orbg_server *s, uint64_t request_id, int code_index, const float *llr,
                       int64_t B)
{
    if (!s || !llr || B < 1)
        return ORBG_EINVAL;
    if (code_index < 0 || code_index >= (int)s->n_of.size())
        return ORBG_EINVAL;
    const int n = s->n_of[code_index];
    if (request_footprint(B, n) > s->budget || B > s->max_batch_blocks)
        return ORBG_ELIMIT; /* could never be admitted */
    Request *r = new (std::nothrow) Request();
    if (!r)
        return ORBG_ENOMEM;
    r->id = request_id;
    r->code = code_index;
    r->B = B;
    r->n = n;
    r->t_submit = now_s();
    try {
        r->llr.assign(llr, llr + (size_t)B * n);
    } catch (...) {
        delete r;
        return ORBG_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return ORBG_EINVAL;
        }
        if (s->done.count(request_id)) {
            delete r;
            return ORBG_EINVAL; /* id still holds unfetched results */
        }
        s->pending.push_back(r);
        s->stats.submitted += 1;
        s->stats.blocks_submitted += (uint64_t)B;
    }
    s->cv_work.notify_one();
    return ORBG_OK;
}

int orbg_server_poll(orbg_server *s, uint64_t *ids, int max_ids, int timeout_us)
{
    if (!s || (max_ids > 0 && !ids) || max_ids < 0)
        return ORBG_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done_order.empty() && timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                            [s] { return !s->done_order.empty(); });
    int k = 0;
    while (k < max_ids && !s->done_order.empty()) {
        ids[k++] = s->done_order.front();
        s->done_order.pop_front();
    }
    if (s->error)
        return s->error;
    return k;
}

int orbg_server_fetch(orbg_server *s, uint64_t request_id, uint8_t *codeword, uint32_t *queries,
                      uint8_t *abandoned, double *latency_s)
{
    if (!s)
        return ORBG_EINVAL;
    Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->done.find(request_id);
        if (it == s->done.end())
            return ORBG_EINVAL;
        r = it->second;
        s->done.erase(it);
    }
    if (codeword) std::memcpy(codeword, r->cw.data(), r->cw.size());
    if (queries) std::memcpy(queries, r->q.data(), r->q.size() * sizeof(uint32_t));
    if (abandoned) std::memcpy(abandoned, r->ab.data(), r->ab.size());
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    delete r;
    return ORBG_OK;
}

int orbg_server_cancel(orbg_server *s, uint64_t request_id)
{
    if (!s)
        return ORBG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
        if ((*it)->id == request_id) {
            delete *it;
            s->pending.erase(it);
            s->stats.cancelled += 1;
            return ORBG_OK;
        }
    }
    for (Batch &bt : s->inflight) {
        for (Request *r : bt.reqs) {
            if (r->id == request_id && !r->cancelled) {
                r->cancelled = true;
                s->stats.cancelled += 1;
                return ORBG_OK;
            }
        }
    }
    auto d = s->done.find(request_id);
    if (d != s->done.end()) {
        delete d->second;
        s->done.erase(d);
        auto o = std::find(s->done_order.begin(), s->done_order.end(), request_id);
        if (o != s->done_order.end())
            s->done_order.erase(o);
        s->stats.cancelled += 1;
        return ORBG_OK;
    }
    return ORBG_EINVAL;
}

int orbg_server_stats_get(orbg_server *s, orbg_server_stats *out)
{
    if (!s || !out)
        return ORBG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->pending = (uint64_t)s->pending.size();
    out->inflight_batches = (uint64_t)s->inflight.size();
    return ORBG_OK;
}

int orbg_server_destroy(orbg_server *s)
{
    if (!s)
        return ORBG_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable())
        s->th.join();
    for (auto &kv : s->done)
        delete kv.second;
    for (Request *r : s->pending)
        delete r;
    for (cudaStream_t st : s->streams)
        cudaStreamDestroy(st);
    cudaFree(s->d_pool);
    cudaFreeHost(s->h_pool);
    delete s->dreg;
    delete s->hreg;
    int err = s->error;
    delete s;
    return err;
}

/*
 * Replays a request trace: a submitter thread submits request i at
 * arrival_s[i] seconds after the call starts; this thread polls and fetches
 * results into the caller's arrays.  Request i has code code[i], B[i]
 * blocks whose LLRs start at element llr_off[i] of llr_all; its outputs go
 * to the same element offset of cw_all, and to q_all / ab_all at block
 * offset blk_off[i].  latency_s[i] gets submit-to-completion time.
 */
int orbg_server_replay(orbg_server *s, int64_t nreq, const double *arrival_s, const int32_t *code,
                       const int64_t *B, const int64_t *llr_off, const int64_t *blk_off,
                       const float *llr_all, uint8_t *cw_all, uint32_t *q_all, uint8_t *ab_all,
                       double *latency_s, double *wall_s)
{
    if (!s || nreq < 0 || (nreq > 0 && (!arrival_s || !code || !B || !llr_off || !blk_off ||
                                        !llr_all || !cw_all || !q_all || !ab_all || !latency_s)))
        return ORBG_EINVAL;
    std::atomic<int> submit_rc(ORBG_OK);
    std::atomic<bool> abort_submit(false);
    const auto t0 = Clock::now();
    const uint64_t base = 0x5E41000000000000ull;
    std::thread sub([&] {
        for (int64_t i = 0; i < nreq && !abort_submit.load(); i++) {
            std::this_thread::sleep_until(
                t0 + std::chrono::duration_cast<Clock::duration>(
                         std::chrono::duration<double>(arrival_s[i])));
            int rc = orbg_server_submit(s, base + (uint64_t)i, code[i], llr_all + llr_off[i], B[i]);
            if (rc != ORBG_OK) {
                submit_rc = rc;
                return;
            }
        }
    });
    int64_t got = 0;
    int rc = ORBG_OK;
    std::vector<uint64_t> ids(1024);
    while (got < nreq) {
        int k = orbg_server_poll(s, ids.data(), (int)ids.size(), 1000);
        if (k < 0) {
            rc = k;
            break;
        }
        if (submit_rc.load() != ORBG_OK) {
            rc = submit_rc.load();
            break;
        }
        for (int j = 0; j < k; j++) {
            const int64_t i = (int64_t)(ids[j] - base);
            int frc = orbg_server_fetch(s, ids[j], cw_all + llr_off[i], q_all + blk_off[i],
                                        ab_all + blk_off[i], latency_s + i);
            if (frc != ORBG_OK)
                rc = frc;
            got++;
        }
    }
    abort_submit = true;
    sub.join();
    if (wall_s)
        *wall_s = std::chrono::duration<double>(Clock::now() - t0).count();
    if (rc == ORBG_OK && submit_rc.load() != ORBG_OK)
        rc = submit_rc.load();
    return rc;
}

}  // extern "C"
