// server.cu -- continuous-batching request loop over adsx_search_batched.
//
// A worker thread owns up to `n_streams` batches in flight, one per CUDA
// stream.  Whenever a stream is free and requests are queued, it forms the
// next batch from the head of the queue: requests with the same (eps0,
// delta_d) as the head, as many as the free query slots, the device-memory
// budget and max_batch allow (admission by memory).  A batch is copied to
// the device through its stream's pinned buffers, searched with
// adsx_search_batched (per-request K and nprobe), and copied back; its event
// marks completion.  Batches on different streams overlap on the device, so
// requests that arrive while others run are admitted as slots and memory
// free up -- no request waits for an unrelated batch to drain.
//
// Requests whose own cost exceeds the whole budget are failed with
// ADSX_ENOMEM at submission.  Waits on the host are bounded by the caller's
// timeout.  Nothing here blocks the device.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "adsx_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { QUEUED = 0, RUNNING = 1, DONE = 2, FAILED = 3, CANCELLED = 4 };

struct Req {
    int64_t ticket;
    std::vector<float> q;
    int32_t K, nprobe;
    float eps0;
    int32_t delta_d;
    int64_t cost;
    int state = QUEUED;
    int rc = ADSX_OK;
    std::vector<int64_t> ids;
    std::vector<float> dists;
    int64_t dims = 0;
    Clock::time_point t_submit, t_done;
};

struct Slot {                       // one stream and its staging buffers
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<int64_t> tickets;
    int64_t cost = 0;
    int rc = ADSX_OK;
    // pinned host and device staging, sized for max_batch queries
    float *h_q = nullptr, *d_q = nullptr;
    int32_t *h_kp = nullptr, *d_kp = nullptr;   // K then nprobe
    int64_t *h_ids = nullptr, *d_ids = nullptr, *h_dims = nullptr, *d_dims = nullptr;
    float *h_d2 = nullptr, *d_d2 = nullptr;
};

struct Server {
    const adsx_index *index = nullptr;
    const adsx::Index *ix = nullptr;
    int32_t max_slots = 0, max_batch = 0, max_K = 0, max_nprobe = 0;
    int64_t budget = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Req> reqs;
    int64_t next_ticket = 1;
    int32_t slots_used = 0;
    int64_t mem_used = 0;
    bool stop = false;
    std::thread worker;
    std::vector<double> lat_ms;        // completed requests' latencies
    Clock::time_point t_first, t_last;
    int64_t completed = 0, batches = 0, max_inflight_batches = 0, max_slots_used = 0;
};

// Device bytes one request needs inside adsx_search_batched: its rotated
// query and that query's TF32 halves, a row of centroid distances and of
// their tile summary, its probe list, plan entries, the partial lists of
// its splits and its outputs.  (The TF32 halves of a batch's queries are
// padded to a multiple of 128 rows; that padding, at most 127 * 8 * Dp
// bytes per batch, is not charged.)
int64_t request_cost(const adsx::Index *ix, int32_t K, int32_t max_nprobe, int32_t max_K)
{
    const int64_t tiles = (ix->nlist + adsx::SUMMARY_TILE - 1) / adsx::SUMMARY_TILE;
    return 12LL * ix->Dp + 4LL * ix->nlist + 16LL * tiles + 4LL * max_nprobe +
           8LL * adsx::BATCH_MAX_SPLITS + 8LL * adsx::BATCH_MAX_SPLITS * max_K + 12LL * K + 64;
}

void free_slot(Slot &s)
{
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaFreeHost(s.h_q);
    cudaFreeHost(s.h_kp);
    cudaFreeHost(s.h_ids);
    cudaFreeHost(s.h_d2);
    cudaFreeHost(s.h_dims);
    cudaFree(s.d_q);
    cudaFree(s.d_kp);
    cudaFree(s.d_ids);
    cudaFree(s.d_d2);
    cudaFree(s.d_dims);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot();
}

// Completes finished batches (called with the lock held).
void reap(Server &sv)
{
    for (Slot &s : sv.slots) {
        if (!s.busy) continue;
        cudaError_t e = cudaEventQuery(s.done);
        if (e == cudaErrorNotReady) continue;
        const auto now = Clock::now();
        int64_t off = 0;
        for (size_t i = 0; i < s.tickets.size(); ++i) {
            auto it = sv.reqs.find(s.tickets[i]);
            if (it == sv.reqs.end()) continue;
            Req &r = it->second;
            if (e != cudaSuccess || s.rc != ADSX_OK) {
                r.state = FAILED;
                r.rc = s.rc != ADSX_OK ? s.rc : ADSX_ECUDA;
            } else {
                r.ids.assign(s.h_ids + off, s.h_ids + off + r.K);
                r.dists.assign(s.h_d2 + off, s.h_d2 + off + r.K);
                r.dims = s.h_dims[i];
                r.state = DONE;
            }
            off += r.K;
            r.t_done = now;
            sv.lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
            sv.completed += 1;
            sv.t_last = now;
        }
        if (e != cudaSuccess) cudaGetLastError();
        sv.slots_used -= (int32_t)s.tickets.size();
        sv.mem_used -= s.cost;
        s.tickets.clear();
        s.cost = 0;
        s.busy = false;
        s.rc = ADSX_OK;
        sv.cv_done.notify_all();
    }
}

// Forms and launches one batch on a free stream (lock held); false if none.
bool admit(Server &sv)
{
    Slot *slot = nullptr;
    for (Slot &s : sv.slots)
        if (!s.busy) {
            slot = &s;
            break;
        }
    if (!slot) return false;
    while (!sv.queue.empty()) {
        auto f = sv.reqs.find(sv.queue.front());
        if (f != sv.reqs.end() && f->second.state == QUEUED) break;
        sv.queue.pop_front();
    }
    if (sv.queue.empty()) return false;
    const Req &head = sv.reqs[sv.queue.front()];
    std::vector<int64_t> take;
    int64_t cost = 0;
    for (auto it = sv.queue.begin(); it != sv.queue.end() && (int32_t)take.size() < sv.max_batch;) {
        auto rit = sv.reqs.find(*it);
        if (rit == sv.reqs.end() || rit->second.state != QUEUED) {
            it = sv.queue.erase(it);
            continue;
        }
        const Req &r = rit->second;
        if (r.eps0 != head.eps0 && !(isinf(r.eps0) && isinf(head.eps0))) { ++it; continue; }
        if (r.delta_d != head.delta_d) { ++it; continue; }
        if (sv.slots_used + (int32_t)take.size() + 1 > sv.max_slots) break;
        if (sv.mem_used + cost + r.cost > sv.budget) break;
        cost += r.cost;
        take.push_back(*it);
        it = sv.queue.erase(it);
    }
    if (take.empty()) return false;
    sv.max_slots_used = std::max<int64_t>(sv.max_slots_used, sv.slots_used + (int64_t)take.size());
    const int D = sv.ix->D;
    const int64_t n = (int64_t)take.size();
    int64_t total = 0;
    for (size_t i = 0; i < take.size(); ++i) {
        Req &r = sv.reqs[take[i]];
        memcpy(slot->h_q + i * D, r.q.data(), sizeof(float) * D);
        slot->h_kp[i] = r.K;
        slot->h_kp[n + i] = r.nprobe;
        r.state = RUNNING;
        total += r.K;
    }
    cudaStream_t st = slot->stream;
    int rc = ADSX_OK;
    cudaError_t e = cudaMemcpyAsync(slot->d_q, slot->h_q, sizeof(float) * n * D, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(slot->d_kp, slot->h_kp, sizeof(int32_t) * 2 * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = ADSX_ECUDA;
    if (rc == ADSX_OK)
        rc = adsx_search_batched(sv.index, slot->d_q, n, slot->d_kp, slot->d_kp + n, sv.max_K,
                                 sv.max_nprobe, head.eps0, head.delta_d, nullptr, total, slot->d_ids,
                                 slot->d_d2, slot->d_dims, st);
    if (rc == ADSX_OK) {
        e = cudaMemcpyAsync(slot->h_ids, slot->d_ids, sizeof(int64_t) * total, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(slot->h_d2, slot->d_d2, sizeof(float) * total, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(slot->h_dims, slot->d_dims, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = ADSX_ECUDA;
    }
    cudaEventRecord(slot->done, st);
    slot->busy = true;
    slot->rc = rc;
    slot->tickets = take;
    slot->cost = cost;
    sv.slots_used += (int32_t)n;
    sv.mem_used += cost;
    sv.batches += 1;
    int64_t inflight = 0;
    for (const Slot &s : sv.slots) inflight += s.busy;
    sv.max_inflight_batches = std::max(sv.max_inflight_batches, inflight);
    return true;
}

void worker_loop(Server *sv)
{
    cudaSetDevice(sv->ix->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        reap(*sv);
        bool launched = false;
        while (admit(*sv)) launched = true;
        bool busy = false;
        for (const Slot &s : sv->slots) busy |= s.busy;
        if (!launched) {
            // poll in-flight batches often; sleep longer when idle
            sv->cv_work.wait_for(lk, busy ? std::chrono::microseconds(20)
                                          : std::chrono::milliseconds(2));
        }
    }
    lk.unlock();
    for (Slot &s : sv->slots)
        if (s.stream) cudaStreamSynchronize(s.stream);
    lk.lock();
    reap(*sv);
}

int sfail(int code, const std::string &m)
{
    adsx::set_last_error(m);
    return code;
}

}  // namespace

extern "C" {

int adsx_server_create(const adsx_index *index, int32_t max_slots, int32_t max_batch,
                       int32_t n_streams, int64_t mem_budget_bytes, int32_t max_K,
                       int32_t max_nprobe, adsx_server **out)
{
    if (!out) return sfail(ADSX_EINVAL, "out is NULL");
    *out = nullptr;
    const adsx::Index *ix = reinterpret_cast<const adsx::Index *>(index);
    if (!ix) return sfail(ADSX_EINVAL, "index is NULL");
    if (max_slots < 1 || max_batch < 1 || n_streams < 1 || n_streams > 16 || mem_budget_bytes <= 0)
        return sfail(ADSX_EINVAL, "bad server limits");
    if (max_K < 1 || max_K > ADSX_MAX_K || max_nprobe < 1 || max_nprobe > ix->nlist ||
        max_nprobe > ADSX_MAX_NPROBE)
        return sfail(ADSX_EINVAL, "max_K / max_nprobe out of range");
    cudaError_t e = cudaSetDevice(ix->device);
    if (e != cudaSuccess) return sfail(ADSX_ECUDA, cudaGetErrorString(e));
    Server *sv = new Server();
    sv->index = index;
    sv->ix = ix;
    sv->max_slots = max_slots;
    sv->max_batch = std::min(max_batch, max_slots);
    sv->budget = mem_budget_bytes;
    sv->max_K = max_K;
    sv->max_nprobe = max_nprobe;
    sv->slots.resize(n_streams);
    const int64_t B = sv->max_batch, D = ix->D;
    for (Slot &s : sv->slots) {
        bool ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMallocHost(&s.h_q, sizeof(float) * B * D) == cudaSuccess &&
                  cudaMallocHost(&s.h_kp, sizeof(int32_t) * 2 * B) == cudaSuccess &&
                  cudaMallocHost(&s.h_ids, sizeof(int64_t) * B * max_K) == cudaSuccess &&
                  cudaMallocHost(&s.h_d2, sizeof(float) * B * max_K) == cudaSuccess &&
                  cudaMallocHost(&s.h_dims, sizeof(int64_t) * B) == cudaSuccess &&
                  cudaMalloc(&s.d_q, sizeof(float) * B * D) == cudaSuccess &&
                  cudaMalloc(&s.d_kp, sizeof(int32_t) * 2 * B) == cudaSuccess &&
                  cudaMalloc(&s.d_ids, sizeof(int64_t) * B * max_K) == cudaSuccess &&
                  cudaMalloc(&s.d_d2, sizeof(float) * B * max_K) == cudaSuccess &&
                  cudaMalloc(&s.d_dims, sizeof(int64_t) * B) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            for (Slot &t : sv->slots) free_slot(t);
            delete sv;
            return sfail(ADSX_ENOMEM, "server staging allocation failed");
        }
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = reinterpret_cast<adsx_server *>(sv);
    return ADSX_OK;
}

int adsx_server_submit(adsx_server *server, const float *q, int32_t K, int32_t nprobe,
                       float eps0, int32_t delta_d, int64_t *ticket)
{
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv || !q || !ticket) return sfail(ADSX_EINVAL, "bad submit arguments");
    if (K < 1 || K > sv->max_K || nprobe < 1 || nprobe > sv->max_nprobe)
        return sfail(ADSX_EINVAL, "K / nprobe outside the server's limits");
    if (!(eps0 >= 0.f)) return sfail(ADSX_EINVAL, "eps0 must be >= 0");
    if (delta_d != 0 && (delta_d < 16 || delta_d % 16)) return sfail(ADSX_EINVAL, "bad delta_d");
    Req r;
    r.q.assign(q, q + sv->ix->D);
    r.K = K;
    r.nprobe = nprobe;
    r.eps0 = eps0;
    r.delta_d = delta_d;
    r.cost = request_cost(sv->ix, K, sv->max_nprobe, sv->max_K);
    if (r.cost > sv->budget)
        return sfail(ADSX_ENOMEM, "request needs " + std::to_string(r.cost) +
                                      " device bytes, above the whole budget");
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r.ticket = sv->next_ticket++;
        *ticket = r.ticket;
        if (sv->completed == 0 && sv->reqs.empty()) sv->t_first = r.t_submit;
        sv->queue.push_back(r.ticket);
        sv->reqs.emplace(r.ticket, std::move(r));
    }
    sv->cv_work.notify_one();
    return ADSX_OK;
}

int adsx_server_submit_many(adsx_server *server, const float *Q, int64_t n, const int32_t *K,
                            const int32_t *nprobe, float eps0, int32_t delta_d, int64_t *tickets)
{
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv || (n > 0 && (!Q || !K || !nprobe || !tickets)) || n < 0)
        return sfail(ADSX_EINVAL, "bad submit arguments");
    if (!(eps0 >= 0.f)) return sfail(ADSX_EINVAL, "eps0 must be >= 0");
    if (delta_d != 0 && (delta_d < 16 || delta_d % 16)) return sfail(ADSX_EINVAL, "bad delta_d");
    const int D = sv->ix->D;
    std::vector<Req> rs((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        if (K[i] < 1 || K[i] > sv->max_K || nprobe[i] < 1 || nprobe[i] > sv->max_nprobe)
            return sfail(ADSX_EINVAL, "K / nprobe outside the server's limits");
        Req &r = rs[(size_t)i];
        r.q.assign(Q + i * D, Q + (i + 1) * D);
        r.K = K[i];
        r.nprobe = nprobe[i];
        r.eps0 = eps0;
        r.delta_d = delta_d;
        r.cost = request_cost(sv->ix, K[i], sv->max_nprobe, sv->max_K);
        if (r.cost > sv->budget) return sfail(ADSX_ENOMEM, "a request exceeds the whole budget");
    }
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->completed == 0 && sv->reqs.empty()) sv->t_first = now;
        for (int64_t i = 0; i < n; ++i) {
            Req &r = rs[(size_t)i];
            r.t_submit = now;
            r.ticket = sv->next_ticket++;
            tickets[i] = r.ticket;
            sv->queue.push_back(r.ticket);
            sv->reqs.emplace(r.ticket, std::move(r));
        }
    }
    sv->cv_work.notify_one();
    return ADSX_OK;
}

int adsx_server_wait(adsx_server *server, int64_t ticket, int32_t timeout_ms, int64_t *ids,
                     float *dists, int64_t *dims_read)
{
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv) return sfail(ADSX_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return sfail(ADSX_EINVAL, "unknown ticket");
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (it->second.state == QUEUED || it->second.state == RUNNING) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            it = sv->reqs.find(ticket);
            if (it->second.state == QUEUED || it->second.state == RUNNING)
                return sfail(ADSX_ETIMEOUT, "request not finished within the timeout");
        }
        it = sv->reqs.find(ticket);
    }
    Req &r = it->second;
    int rc = r.rc;
    if (r.state == DONE) {
        if (ids) memcpy(ids, r.ids.data(), sizeof(int64_t) * r.K);
        if (dists) memcpy(dists, r.dists.data(), sizeof(float) * r.K);
        if (dims_read) *dims_read = r.dims;
    } else if (r.state == CANCELLED) {
        rc = sfail(ADSX_EINVAL, "request was cancelled");
    } else {
        rc = sfail(rc ? rc : ADSX_ECUDA, "request failed");
    }
    sv->reqs.erase(it);
    return rc;
}

int adsx_server_cancel(adsx_server *server, int64_t ticket)
{
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv) return sfail(ADSX_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return sfail(ADSX_EINVAL, "unknown ticket");
    if (it->second.state != QUEUED) return sfail(ADSX_EINVAL, "request already running or done");
    it->second.state = CANCELLED;
    sv->cv_done.notify_all();
    return ADSX_OK;
}

int adsx_server_stats(adsx_server *server, double *p50_ms, double *p99_ms, double *qps,
                      int64_t *completed, int64_t *batches, int64_t *max_inflight_batches,
                      int64_t *max_inflight_queries)
{
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv) return sfail(ADSX_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::vector<double> l = sv->lat_ms;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
        if (l.empty()) return 0.0;
        size_t i = (size_t)std::min<double>(l.size() - 1, floor(p * (l.size() - 1) + 0.5));
        return l[i];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (qps) {
        double span = std::chrono::duration<double>(sv->t_last - sv->t_first).count();
        *qps = span > 0 ? sv->completed / span : 0.0;
    }
    if (completed) *completed = sv->completed;
    if (batches) *batches = sv->batches;
    if (max_inflight_batches) *max_inflight_batches = sv->max_inflight_batches;
    if (max_inflight_queries) *max_inflight_queries = sv->max_slots_used;
    return ADSX_OK;
}

int adsx_server_reset_stats(adsx_server *server)
{
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv) return sfail(ADSX_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->lat_ms.clear();
    sv->completed = 0;
    sv->batches = 0;
    sv->max_inflight_batches = 0;
    sv->max_slots_used = 0;
    sv->t_first = Clock::now();
    sv->t_last = sv->t_first;
    return ADSX_OK;
}

int adsx_server_destroy(adsx_server *server)
{
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv) return ADSX_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot &s : sv->slots) free_slot(s);
    delete sv;
    return ADSX_OK;
}

}  // extern "C"
