// serve.cpp — topk_serve_*: a request loop with admission by HBM budget and
// continuous batching (host runtime; the selections run in the library's
// kernels).  The paper has no serving form; every request is one selection of
// Section 2 / Section 4.1.
//
// One worker thread owns every CUDA call.  Per turn it
//   1. retires finished slots (event query; no blocking wait), records the
//      latency of each request in them and returns their bytes to the budget;
//   2. admits requests from the head of the FIFO while a slot is free and the
//      bytes in flight stay within the budget: a run of small requests
//      (<= BATCH_ROW_MAX keys, one key type) becomes one batched launch,
//      a large request one topk_select, each on the slot's own stream, so
//      work of different requests overlaps on the device;
//   3. sleeps on a condition variable when nothing is queued or running.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using topk::BATCH_ROW_MAX;

constexpr uint32_t MAX_BATCH_ROWS = 2048;
constexpr uint64_t RESERVE_N = 1ull << 26;  // selection size each slot's scratch is reserved for
constexpr uint64_t REQUEST_OVERHEAD = 4096; // state and bookkeeping per request
constexpr uint64_t CTX_FIXED_BYTES = 256 + 64 * 4 + 4096 + 4096 * 4; // a context's error word, counters, state, histogram

uint64_t steady_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Pending {
    topk_request r;
    uint64_t ticket;
    uint64_t bytes;
    uint64_t arrival;
    bool budget_wait = false; // counted once when it first waited for room in the budget
};

struct Slot {
    topk_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Pending> work;
    uint64_t bytes = 0;
    char* h_ptrs = nullptr; // pinned staging of the batched pointer arrays
    char* d_ptrs = nullptr;
    uint32_t* h_err = nullptr; // pinned copy of the context's error word, read after each dispatch
    uint64_t held = 0;         // device bytes the slot holds outside any request
};

// Device memory a slot holds outside the requests' own buffers: its
// context's scratch blocks and fixed words, and the batched pointer arrays.
uint64_t slot_held(const Slot& slot) {
    const topk_ctx* c = slot.ctx;
    if (!c) return 0;
    return (uint64_t)c->scratch.bytes + c->freq.bytes + c->aux.bytes + CTX_FIXED_BYTES + 52ull * MAX_BATCH_ROWS;
}

uint64_t request_bytes(const topk_request& r) {
    const int w = topk::dtype_bytes(r.dtype);
    return r.n * (uint64_t)w + r.k * (uint64_t)(w + 4) + (uint64_t)w + 4 + REQUEST_OVERHEAD;
}

} // namespace

struct topk_server {
    int device = 0;
    uint64_t budget = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::unordered_map<uint64_t, int> status; // ticket -> topk_status, or -1 while pending
    uint64_t next_ticket = 1;
    uint64_t inflight = 0;
    bool stop = false;
    std::thread worker;
    // statistics
    std::vector<uint64_t> latencies;
    topk_serve_report st{};
    uint64_t first_arrival = 0, last_done = 0;
};

namespace {

// Enqueues the work of one slot (called by the worker, lock not held).
topk_status dispatch(topk_server* s, Slot& slot) {
    const std::vector<Pending>& w = slot.work;
    cudaStream_t st = slot.stream;
    topk_status rs = TOPK_OK;
    if (w.size() == 1 && w[0].r.n > BATCH_ROW_MAX) {
        const topk_request& r = w[0].r;
        rs = topk_select(slot.ctx, r.d_keys, r.n, r.k, r.dtype, r.d_out_keys, r.d_out_idx, r.d_kth_key,
                         r.d_kth_idx, nullptr, st);
    } else {
        const uint32_t rows = (uint32_t)w.size();
        char* h = slot.h_ptrs;
        for (uint32_t i = 0; i < rows; ++i) {
            const topk_request& r = w[i].r;
            reinterpret_cast<const void**>(h)[i] = r.d_keys;
            reinterpret_cast<void**>(h + 8ull * rows)[i] = r.d_out_keys;
            reinterpret_cast<uint32_t**>(h + 16ull * rows)[i] = r.d_out_idx;
            reinterpret_cast<void**>(h + 24ull * rows)[i] = r.d_kth_key;
            reinterpret_cast<uint32_t**>(h + 32ull * rows)[i] = r.d_kth_idx;
            reinterpret_cast<uint64_t*>(h + 40ull * rows)[i] = r.n;
            reinterpret_cast<uint32_t*>(h + 48ull * rows)[i] = (uint32_t)r.k;
        }
        const size_t bytes = 52ull * rows;
        if (cudaMemcpyAsync(slot.d_ptrs, h, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) rs = TOPK_ECUDA;
        if (rs == TOPK_OK) rs = topk::batched_by_pointers(slot.ctx, w[0].r.dtype, rows, slot.d_ptrs, st);
    }
    // the device status travels with the work: no blocking read when it retires
    if (rs == TOPK_OK && cudaMemcpyAsync(slot.h_err, slot.ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                         st) != cudaSuccess)
        rs = TOPK_ECUDA;
    if (cudaEventRecord(slot.done, st) != cudaSuccess && rs == TOPK_OK) rs = TOPK_ECUDA;
    return rs;
}

void worker_main(topk_server* s) {
    cudaSetDevice(s->device);
    while (true) {
        bool any_busy = false;
        // 1. retire finished slots
        for (Slot& slot : s->slots) {
            if (!slot.busy) continue;
            const cudaError_t q = cudaEventQuery(slot.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            topk_status rs = q == cudaSuccess ? static_cast<topk_status>(*slot.h_err) : TOPK_ECUDA;
            if (q != cudaSuccess) cudaGetLastError();
            if (rs != TOPK_OK && q == cudaSuccess) { // clear it before the slot's next work (stream order)
                *slot.h_err = 0;
                cudaMemsetAsync(slot.ctx->d_err, 0, sizeof(uint32_t), slot.stream);
            }
            const uint64_t now = steady_ns();
            std::lock_guard<std::mutex> lock(s->mu);
            for (const Pending& p : slot.work) {
                s->status[p.ticket] = rs;
                if (rs == TOPK_OK) {
                    s->st.completed++;
                    s->st.keys += p.r.n;
                    s->latencies.push_back(now > p.arrival ? now - p.arrival : 0);
                } else {
                    s->st.failed++;
                }
            }
            s->last_done = now;
            s->inflight -= slot.bytes;
            slot.bytes = 0;
            slot.work.clear();
            slot.busy = false;
            s->cv_done.notify_all();
        }
        // 2. admit from the head of the queue onto free slots
        std::vector<Slot*> launch;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            for (Slot& slot : s->slots) {
                if (slot.busy) continue;
                if (s->queue.empty()) break;
                Pending& head = s->queue.front();
                if (s->inflight + head.bytes > s->budget) { // FIFO: wait for room
                    if (!head.budget_wait) {
                        head.budget_wait = true;
                        s->st.budget_waits++;
                    }
                    break;
                }
                const bool small = head.r.n <= BATCH_ROW_MAX;
                const topk_dtype dt = head.r.dtype;
                do {
                    s->inflight += s->queue.front().bytes;
                    slot.bytes += s->queue.front().bytes;
                    slot.work.push_back(s->queue.front());
                    s->queue.pop_front();
                } while (small && !s->queue.empty() && slot.work.size() < MAX_BATCH_ROWS &&
                         s->queue.front().r.n <= BATCH_ROW_MAX && s->queue.front().r.dtype == dt &&
                         s->inflight + s->queue.front().bytes <= s->budget);
                s->st.peak_inflight_bytes = std::max(s->st.peak_inflight_bytes, s->inflight);
                if (small) {
                    s->st.batches++;
                    s->st.batched_requests += slot.work.size();
                }
                slot.busy = true;
                launch.push_back(&slot);
            }
            if (launch.empty() && !any_busy) {
                if (s->stop && s->queue.empty()) return;
                if (s->queue.empty()) {
                    s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty(); });
                    continue;
                }
            }
        }
        for (Slot* slot : launch) {
            const topk_status rs = dispatch(s, *slot);
            const uint64_t held = slot_held(*slot); // a larger request may have grown the slot's scratch
            if (held != slot->held) {
                std::lock_guard<std::mutex> lock(s->mu);
                s->st.reserved_bytes += held - slot->held;
                slot->held = held;
            }
            if (rs != TOPK_OK) { // nothing (more) will complete on this slot's event: retire now
                cudaStreamSynchronize(slot->stream);
                cudaGetLastError();
                std::lock_guard<std::mutex> lock(s->mu);
                for (const Pending& p : slot->work) {
                    s->status[p.ticket] = rs;
                    s->st.failed++;
                }
                s->inflight -= slot->bytes;
                slot->bytes = 0;
                slot->work.clear();
                slot->busy = false;
                s->cv_done.notify_all();
            }
        }
        // slots are busy: poll again soon (a sleep would cost tens of
        // microseconds of timer slack on every completion)
        if (launch.empty()) std::this_thread::yield();
    }
}

} // namespace

extern "C" {

topk_status topk_serve_create(topk_server** out, int device, uint64_t hbm_budget, uint32_t max_slots) {
    if (!out || max_slots == 0 || max_slots > 64 || hbm_budget == 0) return TOPK_EINVAL;
    *out = nullptr;
    topk_server* s = new topk_server();
    s->device = device;
    s->budget = hbm_budget;
    s->slots.resize(max_slots);
    topk_status rs = TOPK_OK;
    if (cudaSetDevice(device) != cudaSuccess) rs = TOPK_EINVAL;
    for (Slot& slot : s->slots) {
        if (rs != TOPK_OK) break;
        if ((rs = topk_ctx_create(&slot.ctx, device)) != TOPK_OK) break;
        // scratch for the largest work a slot usually gets (a selection of
        // 2^26 keys, a batch of MAX_BATCH_ROWS rows, 64-bit keys), so that
        // growing it -- which synchronises the device -- stays rare
        if ((rs = topk_ctx_reserve(slot.ctx, RESERVE_N, TOPK_U64)) != TOPK_OK) break;
        if ((rs = topk::batched_reserve(slot.ctx, TOPK_U64, MAX_BATCH_ROWS)) != TOPK_OK) break;
        if (cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void**>(&slot.h_ptrs), 52ull * MAX_BATCH_ROWS) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void**>(&slot.h_err), sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&slot.d_ptrs), 52ull * MAX_BATCH_ROWS) != cudaSuccess)
            rs = TOPK_ENOMEM;
    }
    if (rs != TOPK_OK) {
        topk_serve_destroy(s);
        return rs;
    }
    for (Slot& slot : s->slots) {
        slot.held = slot_held(slot);
        s->st.reserved_bytes += slot.held;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return TOPK_OK;
}

topk_status topk_serve_submit(topk_server* s, const topk_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket) return TOPK_EINVAL;
    const topk_request& r = *req;
    const int w = topk::dtype_bytes(r.dtype);
    if (w == 0 || !r.d_keys || !r.d_out_keys || !r.d_out_idx || !r.d_kth_key || !r.d_kth_idx || r.k < 1 ||
        r.k > r.n || r.n > 0xFFFFFFFFull)
        return TOPK_EINVAL;
    Pending p;
    p.r = r;
    p.bytes = request_bytes(r);
    const uint64_t now = steady_ns();
    p.arrival = r.arrival_ns ? r.arrival_ns : now;
    std::lock_guard<std::mutex> lock(s->mu);
    s->st.submitted++;
    if (p.bytes > s->budget) {
        s->st.rejected++;
        return TOPK_EBUDGET;
    }
    p.ticket = s->next_ticket++;
    *ticket = p.ticket;
    s->status[p.ticket] = -1;
    if (s->first_arrival == 0 || p.arrival < s->first_arrival) s->first_arrival = p.arrival;
    s->queue.push_back(p);
    s->cv_work.notify_one();
    return TOPK_OK;
}

topk_status topk_serve_poll(topk_server* s, uint64_t ticket, int* done) {
    if (!s || !done) return TOPK_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->status.find(ticket);
    if (it == s->status.end()) return TOPK_EINVAL;
    *done = it->second >= 0;
    return TOPK_OK;
}

topk_status topk_serve_wait(topk_server* s, uint64_t ticket, uint64_t timeout_ns) {
    if (!s) return TOPK_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->status.find(ticket);
    if (it == s->status.end()) return TOPK_EINVAL;
    const bool ok = s->cv_done.wait_for(lock, std::chrono::nanoseconds(timeout_ns),
                                        [&] { return s->status[ticket] >= 0; });
    if (!ok) return TOPK_ETIMEOUT;
    return static_cast<topk_status>(s->status[ticket]);
}

topk_status topk_serve_stats(topk_server* s, topk_serve_report* out) {
    if (!s || !out) return TOPK_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->st;
    if (!s->latencies.empty()) {
        std::vector<uint64_t> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto at = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5))]; };
        out->p50_ns = at(0.50);
        out->p99_ns = at(0.99);
        out->max_ns = v.back();
    }
    if (s->last_done > s->first_arrival && s->first_arrival)
        out->elapsed_s = (double)(s->last_done - s->first_arrival) * 1e-9;
    return TOPK_OK;
}

topk_status topk_serve_replay(topk_server* s, const topk_request* reqs, const int64_t* done_before, uint64_t count,
                              uint64_t* tickets, uint64_t* lag_ns) {
    if (!s || (count && (!reqs || !done_before || !tickets))) return TOPK_EINVAL;
    int64_t waited = -1; // every request of index <= waited has finished
    for (uint64_t i = 0; i < count; ++i) {
        const int64_t need = done_before[i];
        if (need >= (int64_t)i) return TOPK_EINVAL; // only earlier requests can be waited for
        while (waited < need) {
            ++waited;
            if (tickets[waited] == 0) continue; // rejected at submission
            const topk_status st = topk_serve_wait(s, tickets[waited], 60ull * 1000 * 1000 * 1000);
            if (st == TOPK_ETIMEOUT) return TOPK_ETIMEOUT;
        }
        uint64_t now = steady_ns();
        while (now < reqs[i].arrival_ns) now = steady_ns();
        if (lag_ns) lag_ns[i] = now - (reqs[i].arrival_ns ? reqs[i].arrival_ns : now);
        if (topk_serve_submit(s, &reqs[i], &tickets[i]) != TOPK_OK) tickets[i] = 0;
    }
    return TOPK_OK;
}

uint64_t topk_serve_now_ns(topk_server* s) {
    (void)s;
    return steady_ns();
}

void topk_serve_destroy(topk_server* s) {
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    cudaSetDevice(s->device);
    for (Slot& slot : s->slots) {
        if (slot.stream) cudaStreamSynchronize(slot.stream);
        if (slot.done) cudaEventDestroy(slot.done);
        if (slot.stream) cudaStreamDestroy(slot.stream);
        if (slot.h_ptrs) cudaFreeHost(slot.h_ptrs);
        if (slot.h_err) cudaFreeHost(slot.h_err);
        if (slot.d_ptrs) cudaFree(slot.d_ptrs);
        if (slot.ctx) topk_ctx_destroy(slot.ctx);
    }
    delete s;
}

} // extern "C"
