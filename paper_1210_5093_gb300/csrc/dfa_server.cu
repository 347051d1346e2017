// Serving loop: a host worker thread that keeps compiled DFAs resident,
// admits requests while the device bytes in flight stay within a budget,
// groups waiting requests into batches and launches each batch on one of
// `max_inflight` streams, so batches formed from requests that arrive while
// earlier batches run overlap them on the device (continuous batching).
// Each batch is one persistent launch of the batched match kernel.
#include <cuda_runtime.h>

#include <algorithm>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "dfa_internal.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

constexpr uint32_t kMaxBatch = 4096;      // requests per launch
// A queue shorter than kAheadBytes is held back (to grow into a larger, more
// efficient batch) only while the device already has work: at least
// kLaunchAhead batches and kAheadBytes of input in flight, a few milliseconds
// of matching.  Below that every request is launched at once; a queue of
// kAheadBytes or more is launched whenever a stream is free.
constexpr uint32_t kLaunchAhead = 2;
constexpr uint64_t kAheadBytes = 512ull << 20;
constexpr size_t kMaxPending = 1u << 20;  // queued requests before EAGAIN

// First-fit allocator over the device arena (offsets, 256-byte granules).
class Arena {
   public:
    void reset(uint64_t size) {
        free_.clear();
        free_[0] = size;
    }
    bool alloc(uint64_t n, uint64_t* off) {
        n = (n + 255) & ~255ull;
        if (n == 0) n = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                uint64_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t n) {
        n = (n + 255) & ~255ull;
        if (n == 0) n = 256;
        auto it = free_.emplace(off, n).first;
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
    }

   private:
    std::map<uint64_t, uint64_t> free_;
};

struct Req {
    uint64_t ticket;
    const dfa_t* dfa;
    const uint8_t* host;
    uint64_t len;
    double t_submit;
    uint64_t dev_off;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t copied = nullptr;  // the batch's input copies have landed (on copy_stream)
    bool busy = false;
    std::vector<Req> reqs;
    uint8_t* ws = nullptr;
    uint64_t ws_bytes = 0;
    uint8_t* pinned = nullptr;  // descriptor staging + results
    uint64_t pinned_bytes = 0;
    dfa_result_t* dev_out = nullptr;
    int status = DFA_OK;
};

}  // namespace

struct dfa_server_s {
    int device = 0;
    uint64_t budget = 0;
    uint8_t* arena_mem = nullptr;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Req> pending;
    std::deque<dfa_completion_t> done;
    std::vector<Slot> slots;
    std::thread worker;
    // Every batch's input copies go on this one stream, in launch order, so the
    // copies of the oldest batch finish first and its matching (on its own
    // stream, after an event wait) overlaps the copies of the batches behind
    // it.  Copies spread over the batches' own streams would share the link
    // and delay every batch's matching until all their copies had landed.
    cudaStream_t copy_stream = nullptr;
    bool stop = false;
    uint64_t next_ticket = 1;
    uint64_t pending_bytes = 0;  // bytes of the queued requests (under mu)
    dfa_server_stats_t st{};
    int fatal = DFA_OK;
    dfa_match_opts_t opts{};  // lookahead and placement window of every batch (under mu)

    void run();
    bool reap();
    bool launch_one();
};

bool dfa_server_s::reap() {
    bool any = false;
    for (Slot& s : slots) {
        if (!s.busy) continue;
        cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaErrorNotReady) continue;
        int status = q == cudaSuccess ? s.status : DFA_ECUDA;
        if (q != cudaSuccess) cudaGetLastError();
        const double t = now_s();
        const dfa_result_t* res = reinterpret_cast<const dfa_result_t*>(s.pinned);
        std::lock_guard<std::mutex> g(mu);
        for (size_t i = 0; i < s.reqs.size(); ++i) {
            dfa_completion_t c;
            std::memset(&c, 0, sizeof c);
            c.ticket = s.reqs[i].ticket;
            if (status == DFA_OK) c.result = res[i];
            else c.result.status = status;
            c.submit_s = s.reqs[i].t_submit;
            c.done_s = t;
            done.push_back(c);
            arena.release(s.reqs[i].dev_off, s.reqs[i].len);
            st.bytes_in_flight -= s.reqs[i].len;
            st.bytes_matched += s.reqs[i].len;
            st.completed++;
        }
        s.reqs.clear();
        s.busy = false;
        any = true;
    }
    if (any) done_cv.notify_all();
    return any;
}

// Per-slot buffers are sized at creation for a full batch (kSlotWs device,
// kSlotPinned pinned host bytes) and doubled when a batch needs more: each
// regrowth frees memory, which waits for the whole device and stalls every
// batch in flight.
constexpr uint64_t kSlotWs = 64ull << 20, kSlotPinned = 1ull << 20;

static int grow(uint8_t** p, uint64_t* cap, uint64_t need, bool pinned) {
    if (*cap >= need) return DFA_OK;
    uint64_t n = std::max<uint64_t>(need, 2 * *cap);
    if (*p) { if (pinned) cudaFreeHost(*p); else cudaFree(*p); }
    *p = nullptr;
    *cap = 0;
    cudaError_t e = pinned ? cudaMallocHost(p, n) : cudaMalloc(p, n);
    if (e != cudaSuccess) { cudaGetLastError(); *p = nullptr; return DFA_ENOMEM; }
    *cap = n;
    return DFA_OK;
}

bool dfa_server_s::launch_one() {
    Slot* slot = nullptr;
    uint32_t busy = 0;
    for (Slot& s : slots) {
        if (s.busy) ++busy;
        else if (!slot) slot = &s;
    }
    if (!slot) return false;
    std::vector<Req> batch;
    dfa_match_opts_t bo;
    {
        std::lock_guard<std::mutex> g(mu);
        bo = opts;
        // admission in arrival order while the arena has room; one batch takes
        // at most budget / slots bytes, so that every slot can be in flight and
        // one batch's copies overlap another's matching
        // and at most kAheadBytes: larger batches fill slowly (latency), and
        // measured host-to-device copies of 1 GiB batches gathered from many
        // request buffers ran at half the rate of 512 MiB batches
        const uint64_t batch_cap =
            std::max<uint64_t>(std::min<uint64_t>(budget / slots.size(), kAheadBytes), 1);
        if (busy >= kLaunchAhead && st.bytes_in_flight >= kAheadBytes &&
            pending_bytes < std::min(batch_cap, kAheadBytes) && pending.size() < kMaxBatch)
            return false;  // let the queue grow while the device is busy
        uint64_t batch_bytes = 0;
        while (!pending.empty() && batch.size() < kMaxBatch) {
            Req r = pending.front();
            if (!batch.empty() && batch_bytes + r.len > batch_cap) break;
            uint64_t off = 0;
            if (!arena.alloc(r.len, &off)) break;
            batch_bytes += r.len;
            r.dev_off = off;
            st.bytes_in_flight += r.len;
            if (st.bytes_in_flight > st.max_bytes_in_flight) st.max_bytes_in_flight = st.bytes_in_flight;
            pending_bytes -= r.len;
            pending.pop_front();
            batch.push_back(r);
        }
    }
    if (batch.empty()) return false;
    const uint32_t n = (uint32_t)batch.size();
    std::vector<const dfa_t*> dfas(n);
    std::vector<const uint8_t*> strs(n);
    std::vector<uint64_t> lens(n);
    for (uint32_t i = 0; i < n; ++i) {
        dfas[i] = batch[i].dfa;
        strs[i] = arena_mem + batch[i].dev_off;
        lens[i] = batch[i].len;
    }
    // one launch per part (tables in shared memory / through L2)
    std::vector<dfam::Prepared> parts;
    std::vector<uint64_t> ws_off;
    uint64_t ws_total = 0;
    int rc = dfam::prepare_parts(n, dfas.data(), strs.data(), lens.data(), &bo, &parts, &ws_off,
                                 &ws_total);
    // device: [part workspaces | results]; pinned host: [results | descriptor staging per part]
    const uint64_t out_off = (ws_total + 255) & ~255ull;
    std::vector<uint64_t> stage_off;
    uint64_t pinned_need = (12ull * n + 255) & ~255ull;
    for (const dfam::Prepared& p : parts) {
        stage_off.push_back(pinned_need);
        pinned_need += (dfam::desc_span(p) + 255) & ~255ull;
    }
    if (rc == DFA_OK) rc = grow(&slot->ws, &slot->ws_bytes, out_off + 12ull * n, false);
    if (rc == DFA_OK) rc = grow(&slot->pinned, &slot->pinned_bytes, pinned_need, true);
    if (rc == DFA_OK) {
        cudaStream_t s = slot->stream;
        // the batch's launch descriptors, then its input, all on the copy
        // stream: the matching stream then holds no host-to-device copy that
        // could queue behind a later batch's input on the copy engine
        for (size_t k = 0; k < parts.size() && rc == DFA_OK; ++k)
            rc = dfam::upload_desc_async(parts[k], slot->ws + ws_off[k], slot->pinned + stage_off[k],
                                         copy_stream);
        for (uint32_t i = 0; i < n && rc == DFA_OK; ++i)
            if (lens[i] && cudaMemcpyAsync(arena_mem + batch[i].dev_off, batch[i].host, lens[i],
                                           cudaMemcpyHostToDevice, copy_stream) != cudaSuccess)
                rc = DFA_ECUDA;
        if (rc == DFA_OK && (cudaEventRecord(slot->copied, copy_stream) != cudaSuccess ||
                             cudaStreamWaitEvent(s, slot->copied, 0) != cudaSuccess))
            rc = DFA_ECUDA;
        slot->dev_out = reinterpret_cast<dfa_result_t*>(slot->ws + out_off);
        for (size_t k = 0; k < parts.size() && rc == DFA_OK; ++k)
            rc = dfam::launch_prepared(parts[k], slot->ws + ws_off[k], slot->dev_out, s);
        if (rc == DFA_OK &&
            cudaMemcpyAsync(slot->pinned, slot->dev_out, 12ull * n, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
            rc = DFA_ECUDA;
        if (cudaEventRecord(slot->done, s) != cudaSuccess) rc = DFA_ECUDA;
    }
    slot->status = rc;
    slot->reqs = std::move(batch);
    slot->busy = true;
    {
        std::lock_guard<std::mutex> g(mu);
        st.launches++;
        uint64_t busy = 0;
        for (const Slot& x : slots) busy += x.busy ? 1 : 0;
        if (busy > st.max_concurrent) st.max_concurrent = busy;
    }
    if (rc != DFA_OK) {
        cudaGetLastError();
        cudaStreamSynchronize(copy_stream);  // no copy into the batch's arena space is left
        cudaStreamSynchronize(slot->stream);
    }
    return true;
}

void dfa_server_s::run() {
    cudaSetDevice(device);
    while (true) {
        bool progressed = reap();
        progressed |= launch_one();
        std::unique_lock<std::mutex> lk(mu);
        bool idle = true;
        for (const Slot& s : slots) idle &= !s.busy;
        if (stop && pending.empty() && idle) break;
        if (!progressed) {
            if (idle && pending.empty()) cv.wait_for(lk, std::chrono::milliseconds(2));
            else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    }
}

extern "C" {

int dfa_server_create(uint64_t budget, uint32_t max_inflight, dfa_server_t** out) {
    return dfam::no_throw([&]() -> int {
        if (!out || budget == 0) return DFA_EINVAL;
        *out = nullptr;
        if (max_inflight == 0) max_inflight = 8;
        if (max_inflight > 64) max_inflight = 64;
        dfa_server_s* s = new (std::nothrow) dfa_server_s();
        if (!s) return DFA_ENOMEM;
        if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return DFA_ECUDA; }
        if (cudaMalloc(&s->arena_mem, budget) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return DFA_ENOMEM;
        }
        s->budget = budget;
        s->opts.lookahead = 1;
        s->arena.reset(budget);
        s->slots.resize(max_inflight);
        bool ok = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
        for (Slot& sl : s->slots)
            ok = ok && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming) == cudaSuccess;
        for (Slot& sl : s->slots)
            ok = ok && grow(&sl.ws, &sl.ws_bytes, kSlotWs, false) == DFA_OK &&
                 grow(&sl.pinned, &sl.pinned_bytes, kSlotPinned, true) == DFA_OK;
        if (!ok) {
            cudaGetLastError();
            for (Slot& x : s->slots) {
                if (x.ws) cudaFree(x.ws);
                if (x.pinned) cudaFreeHost(x.pinned);
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.done) cudaEventDestroy(x.done);
                if (x.copied) cudaEventDestroy(x.copied);
            }
            if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
            cudaFree(s->arena_mem);
            delete s;
            return DFA_ECUDA;
        }
        s->worker = std::thread([s] { s->run(); });
        *out = s;
        return DFA_OK;
    });
}

int dfa_server_set_opts(dfa_server_t* s, const dfa_match_opts_t* opts) {
    return dfam::no_throw([&]() -> int {
        if (!s) return DFA_EINVAL;
        dfa_match_opts_t o{};
        o.lookahead = 1;
        if (opts) {
            if (opts->num_chunks || opts->multiplicity || opts->match_begin_event ||
                opts->match_end_event || opts->lookahead > dfam::kMaxLookahead ||
                opts->boundary_window > dfam::kMaxBoundaryWindow)
                return DFA_EINVAL;
            o.lookahead = opts->lookahead;
            o.boundary_window = opts->boundary_window;
        }
        std::lock_guard<std::mutex> g(s->mu);
        s->opts = o;
        return DFA_OK;
    });
}

int dfa_server_submit(dfa_server_t* s, const dfa_t* dfa, const uint8_t* str, uint64_t len,
                      uint64_t* ticket) {
    return dfam::no_throw([&]() -> int {
        if (!s || !dfa || !ticket || (len && !str)) return DFA_EINVAL;
        if (!dfa->on_device) return DFA_EHOSTONLY;
        std::lock_guard<std::mutex> g(s->mu);
        if (len > s->budget) {
            s->st.rejected++;
            return DFA_EBUDGET;
        }
        if (s->pending.size() >= kMaxPending) return DFA_EAGAIN;
        Req r{s->next_ticket++, dfa, str, len, now_s(), 0};
        s->pending.push_back(r);
        s->pending_bytes += len;
        s->st.submitted++;
        *ticket = r.ticket;
        s->cv.notify_one();
        return DFA_OK;
    });
}

int dfa_server_poll(dfa_server_t* s, dfa_completion_t* out, uint32_t max, uint32_t* n) {
    return dfam::no_throw([&]() -> int {
        if (!s || !n || (max && !out)) return DFA_EINVAL;
        std::lock_guard<std::mutex> g(s->mu);
        uint32_t k = 0;
        while (k < max && !s->done.empty()) {
            out[k++] = s->done.front();
            s->done.pop_front();
        }
        *n = k;
        return DFA_OK;
    });
}

int dfa_server_drain(dfa_server_t* s, double timeout_s) {
    if (!s) return DFA_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                           std::chrono::duration<double>(timeout_s));
    while (s->st.completed < s->st.submitted) {
        if (s->done_cv.wait_until(lk, until) == std::cv_status::timeout &&
            s->st.completed < s->st.submitted)
            return DFA_ETIMEOUT;
    }
    return DFA_OK;
}

int dfa_server_stats(const dfa_server_t* s, dfa_server_stats_t* out) {
    if (!s || !out) return DFA_EINVAL;
    std::lock_guard<std::mutex> g(const_cast<dfa_server_s*>(s)->mu);
    *out = s->st;
    return DFA_OK;
}

void dfa_server_destroy(dfa_server_t* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ws) cudaFree(sl.ws);
        if (sl.pinned) cudaFreeHost(sl.pinned);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.copied) cudaEventDestroy(sl.copied);
    }
    if (s->copy_stream) {
        cudaStreamSynchronize(s->copy_stream);
        cudaStreamDestroy(s->copy_stream);
    }
    if (s->arena_mem) cudaFree(s->arena_mem);
    delete s;
}

}  // extern "C"
