// server.cu -- a served request loop over the batched-region kernel.
//
// Requests (regions whose arrays are already resident on the device) arrive
// at any time.  A scheduler thread admits them in arrival order while the
// bytes in flight stay within the budget, packs the admitted ones into a
// batch whenever a stream slot is free, launches the batch (one persistent
// launch for the whole batch), copies the batch's variables back to pinned
// host memory and records an event.  Completed batches are noticed by polling
// their events; each request's result (with its submit / launch / done times
// on the steady clock) is then handed to accr_poll.  Batches on different
// slots overlap on the device, and requests that arrive while batches run
// form the next batch: continuous batching, not a queue in front of one
// launch at a time.
//
// The paper has no serving layer; this is the runtime around the device path
// of a region (IPMACC Stage 3.7: kernel setup, argument arrangement and
// invocation, here amortised over many regions per launch).
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "fold.cuh"

namespace accr {

static int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Req {
    uint64_t ticket;
    accr_region region;  // its clauses' init pointers point at nothing the caller owns (see init)
    uint64_t init[ACCR_MAX_CLAUSES];  // each clause's prior value, copied at submit
    uint32_t has_init;                // bit c: clause c had a prior value
    int64_t bytes;
    int64_t submit_ns;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Req> reqs;
    uint64_t *host_res = nullptr;  // pinned, max_batch * ACCR_MAX_CLAUSES; the kernel writes it
    int64_t launch_ns = 0;
    int64_t bytes = 0;
    int status = ACCR_OK;
};

// Validates a region as accr_reduce would (its clause outputs are the
// server's, so a stand-in non-null address is used for the check).
static int check_region(const accr_region &g) {
    if (g.flags & ~ACCR_COMPENSATED) return set_error(ACCR_EINVAL, "accr_submit: bad region flags");
    accr_clause cl[ACCR_MAX_CLAUSES];
    const int nc = g.nclauses;
    if (nc < 1 || nc > ACCR_MAX_CLAUSES) return set_error(ACCR_EINVAL, "accr_submit: nclauses = %d", nc);
    static char stand_in[8];
    for (int c = 0; c < nc; ++c) {
        cl[c] = g.clauses[c];
        cl[c].out = stand_in;
    }
    ClauseDev dev[ACCR_MAX_CLAUSES];
    int rc = lower_clauses(g.in_type, cl, nc, g.flags, dev);
    if (rc != ACCR_OK) return rc;
    if (g.n < 0) return set_error(ACCR_EINVAL, "accr_submit: n < 0");
    if (g.n > 0 && !g.in) return set_error(ACCR_EINVAL, "accr_submit: in is NULL");
    if (((uintptr_t)g.in % (uintptr_t)type_bytes(g.in_type)) != 0)
        return set_error(ACCR_EINVAL, "accr_submit: in is not aligned to its element size");
    return ACCR_OK;
}

}  // namespace accr

using namespace accr;

struct accr_server {
    int device = 0;
    uint64_t budget = 0;
    int max_batch = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> pending;
    std::unordered_map<uint64_t, accr_result> done;
    uint64_t next_ticket = 1;
    uint64_t inflight = 0;
    std::vector<Slot> slots;
    std::thread sched;
    bool stop = false;

    void run();
    void complete(Slot &s, int64_t t);
    int launch(Slot &s, std::unique_lock<std::mutex> &lk);
};

void accr_server::complete(Slot &s, int64_t t) {
    for (size_t i = 0; i < s.reqs.size(); ++i) {
        const Req &q = s.reqs[i];
        accr_result r;
        memset(&r, 0, sizeof r);
        r.status = s.status;
        r.nclauses = q.region.nclauses;
        for (int c = 0; c < q.region.nclauses; ++c) {
            uint64_t v = s.host_res[i * ACCR_MAX_CLAUSES + c];
            if (type_bytes(q.region.clauses[c].acc_type) == 4) v &= 0xffffffffull;
            r.value[c] = v;
        }
        r.submit_ns = q.submit_ns;
        r.launch_ns = s.launch_ns;
        r.done_ns = t;
        done[q.ticket] = r;
    }
    inflight -= (uint64_t)s.bytes;
    s.reqs.clear();
    s.busy = false;
}

// Forms a batch from the head of the queue (admission by budget, FIFO) and
// launches it on slot s.  Called with the lock held; drops it while launching.
// Returns 0 if nothing was admitted, 1 if a batch is in flight, 2 if the
// batch failed to launch (its requests are already completed with the error).
int accr_server::launch(Slot &s, std::unique_lock<std::mutex> &lk) {
    std::vector<Req> take;
    int64_t bytes = 0;
    while (!pending.empty() && (int)take.size() < max_batch) {
        const Req &q = pending.front();
        if (inflight + (uint64_t)bytes + (uint64_t)q.bytes > budget) break;
        bytes += q.bytes;
        take.push_back(q);
        pending.pop_front();
    }
    if (take.empty()) return 0;
    inflight += (uint64_t)bytes;
    log_msg(2, "server: batch of %zu regions, %lld bytes, %llu bytes in flight, %zu waiting", take.size(),
            (long long)bytes, (unsigned long long)inflight, pending.size());
    s.busy = true;
    s.bytes = bytes;
    s.reqs = std::move(take);
    lk.unlock();
    std::vector<accr_region> regs(s.reqs.size());
    for (size_t i = 0; i < s.reqs.size(); ++i) {
        regs[i] = s.reqs[i].region;
        // the kernel stores each variable straight into the pinned result slots
        // (no device-to-host copy in the batch's critical path); prior values
        // come from the request's own copy
        for (int c = 0; c < regs[i].nclauses; ++c) {
            regs[i].clauses[c].out = &s.host_res[i * ACCR_MAX_CLAUSES + c];
            regs[i].clauses[c].init = (s.reqs[i].has_init >> c & 1) ? (const void *)&s.reqs[i].init[c] : nullptr;
        }
    }
    s.launch_ns = now_ns();
    int rc = batch_launch_regions(regs.data(), (int64_t)regs.size(), (accr_stream_t)s.stream, ACCR_SERVED_TILE_BYTES);
    if (rc == ACCR_OK) rc = cuda_check(cudaEventRecord(s.done, s.stream), "server: event");
    s.status = rc;
    lk.lock();
    if (rc != ACCR_OK) {
        complete(s, now_ns());
        return 2;
    }
    return 1;
}

void accr_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool any_busy = false, finished = false;
        for (Slot &s : slots) {
            if (!s.busy) continue;
            lk.unlock();
            cudaError_t e = cudaEventQuery(s.done);
            lk.lock();
            if (e == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            if (e != cudaSuccess) s.status = cuda_check(e, "server: batch");
            complete(s, now_ns());
            finished = true;
        }
        if (finished) cv_done.notify_all();
        for (Slot &s : slots) {
            if (s.busy || pending.empty()) continue;
            const int r = launch(s, lk);
            if (r == 0) break;
            if (r == 1) any_busy = true;
            else finished = true;  // failed batch: its waiters must wake up
        }
        if (finished) cv_done.notify_all();
        if (stop && pending.empty() && !any_busy) break;
        if (any_busy) {
            // batches in flight: poll their events again shortly
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else {
            cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return stop || !pending.empty(); });
        }
    }
}

extern "C" ACCR_API int accr_server_create(uint64_t budget, int32_t nstreams, int32_t max_batch,
                                           accr_server **out) {
    ACCR_TRACE("accr_server_create");
    clear_error();
    if (!out) return set_error(ACCR_EINVAL, "accr_server_create: server is NULL");
    *out = nullptr;
    if (budget == 0 || nstreams < 1 || nstreams > 64 || max_batch < 1 || max_batch > (1 << 20))
        return set_error(ACCR_EINVAL, "accr_server_create: bad budget / nstreams / max_batch");
    accr_server *S = new accr_server();
    cudaGetDevice(&S->device);
    S->budget = budget;
    S->max_batch = max_batch;
    S->slots.resize((size_t)nstreams);
    const size_t rb = sizeof(uint64_t) * ACCR_MAX_CLAUSES * (size_t)max_batch;
    for (Slot &s : S->slots) {
        int rc = cuda_check(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking), "server: stream");
        if (rc == ACCR_OK) rc = cuda_check(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming), "server: event");
        if (rc == ACCR_OK) rc = cuda_check(cudaMallocHost(&s.host_res, rb), "server: pinned results");
        if (rc != ACCR_OK) {
            accr_server_destroy(S);
            return rc;
        }
    }
    S->sched = std::thread([S] { S->run(); });
    *out = S;
    return ACCR_OK;
}

extern "C" ACCR_API int accr_submit(accr_server *S, const accr_region *region, uint64_t *ticket) {
    ACCR_TRACE("accr_submit");
    clear_error();
    if (!S || !region || !ticket) return set_error(ACCR_EINVAL, "accr_submit: NULL argument");
    int rc = check_region(*region);
    if (rc != ACCR_OK) return rc;
    Req q;
    q.region = *region;
    // The caller may reuse or free its prior values as soon as this returns:
    // keep a copy of each, read by the scheduler thread when the batch forms.
    q.has_init = 0;
    for (int c = 0; c < ACCR_MAX_CLAUSES; ++c) {
        q.init[c] = 0;
        if (c < region->nclauses && region->clauses[c].init) {
            memcpy(&q.init[c], region->clauses[c].init, (size_t)type_bytes(region->clauses[c].acc_type));
            q.has_init |= 1u << c;
        }
        q.region.clauses[c].init = nullptr;
    }
    q.bytes = region->n * (int64_t)type_bytes(region->in_type);
    if (fault_take(ACCR_FAULT_ADMIT)) return set_error(ACCR_EBUDGET, "accr_submit: injected admission rejection");
    if ((uint64_t)q.bytes > S->budget)
        return set_error(ACCR_EBUDGET, "accr_submit: region of %lld bytes exceeds the budget of %llu",
                         (long long)q.bytes, (unsigned long long)S->budget);
    q.submit_ns = now_ns();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return set_error(ACCR_EINVAL, "accr_submit: server is stopping");
        q.ticket = S->next_ticket++;
        S->pending.push_back(q);
    }
    S->cv_work.notify_one();
    *ticket = q.ticket;
    return ACCR_OK;
}

extern "C" ACCR_API int accr_poll(accr_server *S, uint64_t ticket, accr_result *out, int64_t timeout_us) {
    ACCR_TRACE("accr_poll");
    clear_error();
    if (!S || !out) return set_error(ACCR_EINVAL, "accr_poll: NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto ready = [&] { return S->done.count(ticket) != 0; };
    if (!ready()) {
        if (timeout_us == 0) return ACCR_EAGAIN;
        if (timeout_us < 0) {
            S->cv_done.wait(lk, ready);
        } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
            return set_error(ACCR_ETIMEDOUT, "accr_poll: ticket %llu not ready after %lld us",
                             (unsigned long long)ticket, (long long)timeout_us);
        }
    }
    auto it = S->done.find(ticket);
    *out = it->second;
    S->done.erase(it);
    return out->status;
}

extern "C" ACCR_API int accr_server_destroy(accr_server *S) {
    ACCR_TRACE("accr_server_destroy");
    clear_error();
    if (!S) return ACCR_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->sched.joinable()) S->sched.join();
    for (Slot &s : S->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.host_res) cudaFreeHost(s.host_res);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    delete S;
    return ACCR_OK;
}

// ---- open-loop client ------------------------------------------------------------

namespace accr {
int reduce_grid(int in_type, int nc, int64_t n);
int reduce_launch(const void *in, int64_t n, int in_type, const ClauseDev *cl, int nc, int two_level,
                  Partial *partials, unsigned *counter, int grid, cudaStream_t s);
}  // namespace accr

static void wait_until(int64_t t) {
    while (now_ns() < t) {
    }
}

extern "C" ACCR_API int accr_server_replay(accr_server *S, const accr_region *regions, const double *arrival_s,
                                           int64_t n, uint32_t flags, accr_stream_t stream,
                                           accr_result *results) {
    ACCR_TRACE("accr_server_replay");
    clear_error();
    if (n < 0 || (n > 0 && (!regions || !arrival_s || !results)))
        return set_error(ACCR_EINVAL, "accr_server_replay: bad arguments");
    if (flags & ~ACCR_PLAIN) return set_error(ACCR_EINVAL, "accr_server_replay: bad flags");
    const int64_t t0 = now_ns();
    if (!(flags & ACCR_PLAIN)) {
        if (!S) return set_error(ACCR_EINVAL, "accr_server_replay: server is NULL");
        std::vector<uint64_t> tickets((size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            wait_until(t0 + (int64_t)(arrival_s[i] * 1e9));
            int rc = accr_submit(S, &regions[i], &tickets[i]);
            if (rc != ACCR_OK) return rc;
        }
        int first_err = ACCR_OK;
        for (int64_t i = 0; i < n; ++i) {
            int rc = accr_poll(S, tickets[i], &results[i], -1);
            if (rc != ACCR_OK && first_err == ACCR_OK) first_err = rc;
            results[i].submit_ns = t0 + (int64_t)(arrival_s[i] * 1e9);  // latency from the arrival time
        }
        return first_err;
    }
    // sequential plain launches: one single-region launch per request, in order
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *dres = nullptr, *hres = nullptr;
    int rc = cuda_check(cudaMalloc(&dres, sizeof(uint64_t) * ACCR_MAX_CLAUSES), "replay: results");
    if (rc == ACCR_OK) rc = cuda_check(cudaMallocHost(&hres, sizeof(uint64_t) * ACCR_MAX_CLAUSES), "replay: pinned");
    for (int64_t i = 0; i < n && rc == ACCR_OK; ++i) {
        const accr_region &g = regions[i];
        const int64_t arrive = t0 + (int64_t)(arrival_s[i] * 1e9);
        wait_until(arrive);
        const int64_t start = now_ns();
        accr_clause cl[ACCR_MAX_CLAUSES];
        for (int c = 0; c < g.nclauses && c < ACCR_MAX_CLAUSES; ++c) {
            cl[c] = g.clauses[c];
            cl[c].out = &dres[c];
        }
        rc = accr_reduce(g.in, g.n, g.in_type, cl, g.nclauses, g.flags & ACCR_COMPENSATED, stream);
        if (rc == ACCR_OK)
            rc = cuda_check(cudaMemcpyAsync(hres, dres, sizeof(uint64_t) * ACCR_MAX_CLAUSES, cudaMemcpyDeviceToHost, s),
                            "replay: result copy");
        if (rc == ACCR_OK) rc = cuda_check(cudaStreamSynchronize(s), "replay: sync");
        accr_result &r = results[i];
        memset(&r, 0, sizeof r);
        r.status = rc;
        r.nclauses = g.nclauses;
        for (int c = 0; c < g.nclauses && c < ACCR_MAX_CLAUSES; ++c) {
            uint64_t v = hres[c];
            if (type_bytes(g.clauses[c].acc_type) == 4) v &= 0xffffffffull;
            r.value[c] = v;
        }
        r.submit_ns = arrive;
        r.launch_ns = start;
        r.done_ns = now_ns();
    }
    if (dres) cudaFree(dres);
    if (hres) cudaFreeHost(hres);
    return rc;
}
