// External queries against a resident index (the matching step of the horizontal
// algorithm, Alg. 6: query vectors matched against a local index) and a request loop that
// serves query batches with continuous batching.
//
// Request loop: submitted batches wait in arrival order. A batch is admitted when one of
// the server's slots is free and its estimated device footprint fits the memory budget
// that running batches leave (a batch that alone exceeds the budget is admitted when
// nothing else runs). Every slot is a host thread with its own CUDA stream, so batches
// admitted while others run overlap on the device; results are copied to pinned host
// memory before the request is marked done.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "index.cuh"

using namespace aps;

namespace {

aps_status query_on_stream(aps_index *ix, const int64_t *qptr, const int32_t *qidx, const float *qval, int32_t nq,
                           float t, uint32_t flags, cudaStream_t s, aps_pairs *out, aps_stats *stats) {
    if (!(ix->flags & APS_QUERYABLE)) {
        set_error("the index was not built with APS_QUERYABLE: its prefixes do not bound external queries");
        return APS_EINVAL;
    }
    if (ix->k != 1) {
        set_error("queries need a single-instance index");
        return APS_EINVAL;
    }
    if (!(t >= ix->t) || !(t <= 1.f)) {
        set_error("query threshold %g must be in [build threshold %g, 1]", (double)t, (double)ix->t);
        return APS_EINVAL;
    }
    if (nq < 0 || !qptr) {
        set_error("need nq >= 0 and qptr");
        return APS_EINVAL;
    }
    DBuf<int64_t> dp;
    DBuf<int32_t> di;
    DBuf<float> dv;
    const int64_t *p = qptr;
    const int32_t *ii = qidx;
    const float *vv = qval;
    if (!(flags & APS_DEVICE_PTRS)) {
        if (qptr[0] != 0) {
            set_error("query indptr[0] must be 0");
            return APS_EINVAL;
        }
        const int64_t nnz = qptr[nq];
        if (nnz < 0 || (nnz > 0 && (!qidx || !qval))) {
            set_error("bad query CSR");
            return APS_EINVAL;
        }
        APS_TRY(dp.alloc((size_t)nq + 1, s));
        APS_TRY(di.alloc((size_t)std::max<int64_t>(nnz, 1), s));
        APS_TRY(dv.alloc((size_t)std::max<int64_t>(nnz, 1), s));
        APS_CUDA(cudaMemcpyAsync(dp.p, qptr, sizeof(int64_t) * (nq + 1), cudaMemcpyHostToDevice, s));
        if (nnz) {
            APS_CUDA(cudaMemcpyAsync(di.p, qidx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
            APS_CUDA(cudaMemcpyAsync(dv.p, qval, sizeof(float) * nnz, cudaMemcpyHostToDevice, s));
        }
        p = dp.p;
        ii = di.p;
        vv = dv.p;
    }
    QueryArrays qa;
    APS_TRY(prepare_queries(ix, p, ii, vv, nq, t, flags, s, qa, (flags & APS_DEVICE_PTRS) ? -1 : qptr[nq]));
    aps_stats local{};
    APS_TRY(join_queries(ix, qa, t, flags, s, out, &local));
    if (stats) *stats = local;
    {
        std::lock_guard<std::mutex> lk(ix->stats_mu);
        ix->stats = local;  // the index reports the counters of its last join or query batch
    }
    if (flags & APS_HOST_OUTPUT) {
        aps_status st = pairs_to_host(out, s);
        if (st != APS_OK) {
            pairs_release(out);
            return st;
        }
    }
    return APS_OK;
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { QUEUED, RUNNING, DONE };

struct Request {
    uint64_t ticket = 0;
    std::vector<int64_t> qptr;
    std::vector<int32_t> qidx;
    std::vector<float> qval;
    int32_t nq = 0;
    float t = 0.f;
    size_t est = 0;
    ReqState state = QUEUED;
    bool canceled = false;
    aps_status status = APS_OK;
    std::string err;
    aps_pairs result{};
    double t_submit = 0, t_start = 0, t_done = 0;
};

}  // namespace

struct aps_server {
    aps_index *ix = nullptr;
    size_t budget = 0;
    int slots = 0;
    size_t fixed = 0;  // per-batch scratch independent of the batch size
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> reqs;
    size_t reserved = 0;
    int running = 0;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    // device time line: every batch's device work lies between two events on its slot's
    // stream, read against one reference event recorded when the server was created
    cudaEvent_t ref = nullptr;
    std::vector<cudaEvent_t> ev_begin, ev_end;       // per slot
    std::vector<std::pair<float, float>> intervals;  // per completed batch: [begin, end) ms
};

namespace {

// Device bytes a batch may hold while it runs: per-warp emit lists, per-(query, window)
// counts/offsets/segments, the staged and final pairs (64 per query assumed), query rows.
size_t estimate(const aps_server *sv, int32_t nq, int64_t nnz) {
    const InstDesc &I = sv->ix->inst_h[0];
    const size_t per_q = (size_t)std::max(I.nw, 1) * (4 + 8 + sizeof(Segment)) + 64 * (8 + 12) + 64;
    return sv->fixed + (size_t)nq * per_q + (size_t)nnz * 48;
}

void worker(aps_server *sv, int slot) {
    cudaSetDevice(sv->ix->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        Request *r = nullptr;
        while (!sv->stop) {
            if (!sv->queue.empty()) {
                Request *h = sv->queue.front();
                if (sv->running == 0 || sv->reserved + h->est <= sv->budget) {
                    r = h;
                    sv->queue.pop_front();
                    break;
                }
            }
            sv->cv_work.wait(lk);
        }
        if (!r) return;
        sv->reserved += r->est;
        sv->running++;
        r->state = RUNNING;
        r->t_start = now_s();
        lk.unlock();
        aps_pairs out{};
        cudaStream_t s = sv->streams[slot];
        const bool timed = cudaEventRecord(sv->ev_begin[slot], s) == cudaSuccess;
        aps_status st = query_on_stream(sv->ix, r->qptr.data(), r->qidx.data(), r->qval.data(), r->nq, r->t,
                                        APS_HOST_OUTPUT, s, &out, nullptr);
        std::string msg = st == APS_OK ? std::string() : std::string(aps_last_error());
        float b_ms = 0.f, e_ms = 0.f;
        const bool have_iv = timed && st == APS_OK && cudaEventRecord(sv->ev_end[slot], s) == cudaSuccess &&
                             cudaEventSynchronize(sv->ev_end[slot]) == cudaSuccess &&
                             cudaEventElapsedTime(&b_ms, sv->ref, sv->ev_begin[slot]) == cudaSuccess &&
                             cudaEventElapsedTime(&e_ms, sv->ref, sv->ev_end[slot]) == cudaSuccess;
        if (!have_iv) cudaGetLastError();
        lk.lock();
        if (have_iv) sv->intervals.emplace_back(b_ms, e_ms);
        r->status = st;
        r->err = msg;
        r->result = out;
        r->t_done = now_s();
        r->state = DONE;
        sv->reserved -= r->est;
        sv->running--;
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

aps_status aps_query(aps_index *index, const int64_t *qptr, const int32_t *qidx, const float *qval, int32_t nq,
                     float t, uint32_t flags, aps_pairs *out) {
    if (!index || !out) {
        set_error("index and out must not be NULL");
        return APS_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    return query_on_stream(index, qptr, qidx, qval, nq, t, flags, index->stream, out, nullptr);
}

aps_status aps_server_create(aps_index *index, size_t mem_budget, int32_t slots, aps_server **out) {
    if (!out || !index || slots < 1 || slots > 64) {
        set_error("need an index, 1 <= slots <= 64 and out");
        return APS_EINVAL;
    }
    *out = nullptr;
    if (!(index->flags & APS_QUERYABLE) || index->k != 1) {
        set_error("serving needs a single-instance index built with APS_QUERYABLE");
        return APS_EINVAL;
    }
    aps_server *sv = new aps_server();
    sv->ix = index;
    sv->budget = mem_budget;
    sv->slots = slots;
    sv->fixed = (size_t)num_sms() * (JOIN_THREADS / 32) * JOIN_ECAP * sizeof(int2) + (1u << 20);
    for (int i = 0; i < slots; i++) {
        cudaStream_t st;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t s2 : sv->streams) cudaStreamDestroy(s2);
            delete sv;
            return cuda_status(e, "cudaStreamCreateWithFlags", __FILE__, __LINE__);
        }
        sv->streams.push_back(st);
    }
    cudaError_t e = cudaEventCreate(&sv->ref);
    for (int i = 0; i < slots && e == cudaSuccess; i++) {
        cudaEvent_t a = nullptr, b = nullptr;
        e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        sv->ev_begin.push_back(a);
        sv->ev_end.push_back(b);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sv->ref, sv->streams[0]);
    if (e == cudaSuccess) e = cudaEventSynchronize(sv->ref);
    if (e != cudaSuccess) {
        for (cudaEvent_t x : sv->ev_begin) if (x) cudaEventDestroy(x);
        for (cudaEvent_t x : sv->ev_end) if (x) cudaEventDestroy(x);
        if (sv->ref) cudaEventDestroy(sv->ref);
        for (cudaStream_t s2 : sv->streams) cudaStreamDestroy(s2);
        delete sv;
        return cuda_status(e, "server events", __FILE__, __LINE__);
    }
    for (int i = 0; i < slots; i++) sv->workers.emplace_back(worker, sv, i);
    *out = sv;
    return APS_OK;
}

aps_status aps_server_timeline(aps_server *sv, aps_timeline *out) {
    if (!sv || !out) {
        set_error("server and out must not be NULL");
        return APS_EINVAL;
    }
    std::vector<std::pair<float, int>> ev;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (const auto &iv : sv->intervals) {
            ev.emplace_back(iv.first, +1);
            ev.emplace_back(iv.second, -1);
        }
        out->batches = (int64_t)sv->intervals.size();
    }
    // sweep the batches' [begin, end) intervals: time with >= 1 and >= 2 batches on the device
    std::sort(ev.begin(), ev.end(), [](const std::pair<float, int> &a, const std::pair<float, int> &b) {
        return a.first < b.first || (a.first == b.first && a.second < b.second);
    });
    double busy = 0, overlap = 0, span_lo = 0, span_hi = 0;
    int cur = 0, most = 0;
    for (size_t k = 0; k < ev.size(); k++) {
        if (k > 0) {
            const double dt = (double)ev[k].first - (double)ev[k - 1].first;
            if (cur >= 1) busy += dt;
            if (cur >= 2) overlap += dt;
        }
        cur += ev[k].second;
        most = std::max(most, cur);
    }
    if (!ev.empty()) {
        span_lo = ev.front().first;
        span_hi = ev.back().first;
    }
    out->busy_ms = busy;
    out->overlap_ms = overlap;
    out->span_ms = span_hi - span_lo;
    out->max_in_flight = most;
    out->_reserved = 0;
    return APS_OK;
}

aps_status aps_stream_submit(aps_server *sv, const aps_query_req *req, uint64_t *ticket) {
    if (!sv || !req || !ticket || req->nq < 0 || !req->qptr) {
        set_error("need a server, a request with nq >= 0 and qptr, and a ticket pointer");
        return APS_EINVAL;
    }
    const int64_t nnz = req->qptr[req->nq];
    if (req->qptr[0] != 0 || nnz < 0 || (nnz > 0 && (!req->qidx || !req->qval))) {
        set_error("bad query CSR");
        return APS_EINVAL;
    }
    if (!(req->t >= sv->ix->t) || !(req->t <= 1.f)) {
        set_error("query threshold %g must be in [build threshold %g, 1]", (double)req->t, (double)sv->ix->t);
        return APS_EINVAL;
    }
    Request *r = new Request();
    r->qptr.assign(req->qptr, req->qptr + req->nq + 1);
    r->qidx.assign(req->qidx, req->qidx + nnz);
    r->qval.assign(req->qval, req->qval + nnz);
    r->nq = req->nq;
    r->t = req->t;
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lk(sv->mu);
    r->est = estimate(sv, req->nq, nnz);
    r->ticket = sv->next_ticket++;
    sv->reqs[r->ticket] = r;
    sv->queue.push_back(r);
    *ticket = r->ticket;
    sv->cv_work.notify_one();
    return APS_OK;
}

aps_status aps_stream_poll(aps_server *sv, uint64_t ticket, int32_t timeout_us, aps_pairs *out) {
    if (!sv || !out) {
        set_error("server and out must not be NULL");
        return APS_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return APS_EINVAL;
    }
    Request *r = it->second;
    if (r->state != DONE && timeout_us > 0)
        sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->state == DONE; });
    if (r->state != DONE) {
        if (r->canceled && r->state == QUEUED) {
            sv->reqs.erase(it);
            delete r;
            set_error("request canceled");
            return APS_ECANCELED;
        }
        return APS_EAGAIN;
    }
    sv->reqs.erase(it);
    const aps_status st = r->canceled ? APS_ECANCELED : r->status;
    if (st == APS_OK) {
        *out = r->result;
    } else {
        pairs_release(&r->result);
        set_error("%s", r->canceled ? "request canceled" : r->err.c_str());
    }
    delete r;
    return st;
}

aps_status aps_stream_cancel(aps_server *sv, uint64_t ticket) {
    if (!sv) {
        set_error("server must not be NULL");
        return APS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return APS_EINVAL;
    }
    Request *r = it->second;
    r->canceled = true;
    if (r->state == QUEUED) {
        for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q)
            if (*q == r) {
                sv->queue.erase(q);
                break;
            }
    }
    return APS_OK;
}

void aps_server_free(aps_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &w : sv->workers) w.join();
    for (auto &kv : sv->reqs) {
        pairs_release(&kv.second->result);
        delete kv.second;
    }
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    for (cudaEvent_t x : sv->ev_begin) cudaEventDestroy(x);
    for (cudaEvent_t x : sv->ev_end) cudaEventDestroy(x);
    if (sv->ref) cudaEventDestroy(sv->ref);
    delete sv;
}

}  // extern "C"
