// Amplitude serving with continuous admission.
//
// A server owns one device arena (its HBM budget, allocated once) and a few
// CUDA streams ("slots"). Requests (a plan plus host bitstrings) queue on the
// host; a dispatcher thread admits them in arrival order whenever a slot is
// free and the arena can hold the plan's tables (kept resident across
// requests, least recently used evicted first) plus at least one boundary.
// Admitted requests run concurrently on their slots; the dispatcher polls
// their completion events (no device-side waits), copies the amplitudes out
// of pinned staging and wakes the waiters. The paper's driver reuses plan and
// workspace caches across its 2051 contractions (Sec. 5.2); this is the same
// reuse for a stream of independent requests.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tb_plan.h"
#include "tb_run.h"
#include "tc_pass.cuh"
#include "tbsweep.h"

using namespace tb;
using namespace tb::rt;

namespace {

using clk = std::chrono::steady_clock;

// First-fit allocator over [0, size) with 256-byte granularity.
class Arena {
  public:
    void reset(int64_t size) {
        size_ = size;
        free_.clear();
        free_[0] = size;
        used_ = 0;
    }
    int64_t alloc(int64_t bytes) {
        bytes = align_up(std::max<int64_t>(bytes, 1), 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const int64_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                sizes_[off] = bytes;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off) {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        int64_t len = s->second;
        sizes_.erase(s);
        used_ -= len;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += len;
                return;
            }
        }
        free_[off] = len;
    }
    int64_t largest_free() const {
        int64_t m = 0;
        for (const auto& f : free_) m = std::max(m, f.second);
        return m;
    }
    int64_t used() const { return used_; }

  private:
    int64_t size_ = 0, used_ = 0;
    std::map<int64_t, int64_t> free_;   // offset -> length
    std::map<int64_t, int64_t> sizes_;  // allocated offset -> length
};

struct TableEntry {
    int64_t off = -1;
    int refs = 0;
    uint64_t last_use = 0;
};

struct Request {
    int64_t ticket = 0;
    const tb_plan* plan = nullptr;
    std::vector<uint8_t> bits;  // host copy
    int64_t nb = 0;
    double* out = nullptr;      // caller's host buffer
    clk::time_point t_submit, t_admit, t_done;
    int slot = -1;
    int64_t region_off = -1, stage_off = -1;
    int status = TB_OK;
    bool done = false;
};

}  // namespace

struct tb_server {
    int device = 0;
    int64_t budget = 0;
    void* arena_base = nullptr;
    Arena arena;
    uint8_t* pinned = nullptr;  // host staging: bitstrings in, amplitudes out
    int64_t pinned_bytes = 0;
    Arena pinned_arena;
    std::vector<cudaStream_t> slots;
    std::vector<cudaEvent_t> slot_done;
    std::vector<std::shared_ptr<Request>> running;  // per slot
    std::unordered_map<uint64_t, TableEntry> tables;  // by plan uid
    uint64_t use_clock = 0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<int64_t, std::shared_ptr<Request>> all;
    int64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;

    // statistics
    int64_t completed = 0, amplitudes = 0, peak_running = 0, peak_used = 0;
    std::vector<double> latencies;
};

namespace {

// Bytes a request needs beyond its plan's tables: staged bitstrings and
// amplitudes plus k boundaries (per_b each).
// The last 256 bytes hold the request's fault word (bounded device waits
// that gave up), copied back with the amplitudes.
int64_t staging_len(const Plan& P, int64_t nb) { return align_up(nb * P.n, 256) + align_up(16 * nb, 256) + 256; }

void release_request(tb_server* S, Request& R) {
    if (R.region_off >= 0) S->arena.release(R.region_off);
    if (R.stage_off >= 0) S->pinned_arena.release(R.stage_off);
    R.region_off = R.stage_off = -1;
    auto it = S->tables.find(R.plan->p.uid);
    if (it != S->tables.end()) {
        it->second.refs--;
        it->second.last_use = ++S->use_clock;
    }
}

void finish(tb_server* S, int k) {
    auto R = S->running[k];
    S->running[k].reset();
    if (R->status == TB_OK) {
        const cudaError_t e = cudaEventQuery(S->slot_done[k]);
        if (e != cudaSuccess) R->status = fail(TB_ECUDA, std::string("request failed: ") + cudaGetErrorString(e));
    }
    if (R->status == TB_OK) {
        int faults = 0;
        std::memcpy(&faults, S->pinned + R->stage_off + staging_len(R->plan->p, R->nb) - 256, sizeof(int));
        faults = note_faults(faults);
        if (faults != 0)
            R->status = fail(TB_ETIMEOUT, "a bounded device wait gave up; the amplitudes are not valid");
    }
    if (R->status == TB_OK)
        std::memcpy(R->out, S->pinned + R->stage_off + align_up(R->nb * R->plan->p.n, 256), (size_t)(16 * R->nb));
    release_request(S, *R);
    R->t_done = clk::now();
    R->done = true;
    if (R->status == TB_OK) {
        S->completed++;
        S->amplitudes += R->nb;
        S->latencies.push_back(std::chrono::duration<double>(R->t_done - R->t_submit).count());
    }
    S->cv_done.notify_all();
}

// Allocate device bytes, evicting resident tables nobody uses (LRU first).
int64_t alloc_evicting(tb_server* S, int64_t bytes) {
    for (;;) {
        const int64_t off = S->arena.alloc(bytes);
        if (off >= 0) return off;
        uint64_t best = UINT64_MAX;
        uint64_t victim = 0;
        for (const auto& kv : S->tables)
            if (kv.second.refs == 0 && kv.second.last_use < best) {
                best = kv.second.last_use;
                victim = kv.first;
            }
        if (best == UINT64_MAX) return -1;
        S->arena.release(S->tables[victim].off);
        S->tables.erase(victim);
    }
}

// Try to start the request on slot k; false if memory is not available now.
bool admit(tb_server* S, const std::shared_ptr<Request>& Rp, int k) {
    Request& R = *Rp;
    const Plan& P = R.plan->p;
    const CallLayout c = call_layout(P);
    // pinned staging
    const int64_t st_len = staging_len(P, R.nb);
    const int64_t st_off = S->pinned_arena.alloc(st_len);
    if (st_off < 0) return false;
    // resident tables (pinned by a reference so that eviction skips them)
    TableEntry& te = S->tables[P.uid];
    te.refs++;
    te.last_use = ++S->use_clock;
    if (te.off < 0) {
        const int64_t off = alloc_evicting(S, P.lay.total);
        if (off < 0) {
            if (--te.refs == 0) S->tables.erase(P.uid);
            S->pinned_arena.release(st_off);
            return false;
        }
        te.off = off;
        uint8_t* dst = static_cast<uint8_t*>(S->arena_base) + te.off;
        if (cudaMemcpyAsync(dst, P.blob.data(), (size_t)P.lay.total, cudaMemcpyHostToDevice, S->slots[k]) != cudaSuccess ||
            cudaStreamSynchronize(S->slots[k]) != cudaSuccess) {
            S->arena.release(te.off);
            S->tables.erase(P.uid);
            S->pinned_arena.release(st_off);
            R.status = fail(TB_ECUDA, "table upload failed");
            return true;
        }
    }
    // device region: staged inputs/outputs and as many boundaries as fit
    int64_t kb = c.per_b ? std::min<int64_t>(R.nb, max_batch(P, c)) : 0;
    int64_t reg = -1;
    for (;;) {
        reg = alloc_evicting(S, st_len + kb * c.per_b);
        if (reg >= 0 || kb <= 1) break;
        kb = (kb + 1) / 2;
    }
    if (reg < 0) {
        te.refs--;
        S->pinned_arena.release(st_off);
        return false;
    }
    R.region_off = reg;
    R.stage_off = st_off;
    R.slot = k;
    R.t_admit = clk::now();
    uint8_t* arena = static_cast<uint8_t*>(S->arena_base);
    uint8_t* d_bits = arena + reg;
    double* d_out = reinterpret_cast<double*>(arena + reg + align_up(R.nb * P.n, 256));
    uint8_t* h_bits = S->pinned + st_off;
    std::memcpy(h_bits, R.bits.data(), R.bits.size());
    cudaStream_t st = S->slots[k];
    int rc = TB_OK;
    if (cudaMemcpyAsync(d_bits, h_bits, R.bits.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = fail(TB_ECUDA, "bitstring upload failed");
    int* d_fault = reinterpret_cast<int*>(arena + reg + st_len - 256);
    if (rc == TB_OK && cudaMemsetAsync(d_fault, 0, sizeof(int), st) != cudaSuccess)
        rc = fail(TB_ECUDA, "fault word reset failed");
    if (rc == TB_OK) {
        uint8_t* tab = arena + te.off;
        const int64_t region_off = (reg + st_len) - te.off;
        rc = run_device(P, d_bits, R.nb, tab, region_off + kb * c.per_b, region_off, d_out, st, d_fault);
    }
    if (rc == TB_OK &&
        (cudaMemcpyAsync(h_bits + align_up(R.nb * P.n, 256), d_out, (size_t)(16 * R.nb), cudaMemcpyDeviceToHost,
                         st) != cudaSuccess ||
         cudaMemcpyAsync(h_bits + st_len - 256, d_fault, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess))
        rc = fail(TB_ECUDA, "amplitude download failed");
    if (cudaEventRecord(S->slot_done[k], st) != cudaSuccess && rc == TB_OK) rc = fail(TB_ECUDA, "event record failed");
    R.status = rc;
    S->running[k] = Rp;
    S->peak_used = std::max(S->peak_used, S->arena.used());
    int64_t nrun = 0;
    for (const auto& r : S->running) nrun += r ? 1 : 0;
    S->peak_running = std::max(S->peak_running, nrun);
    return true;
}

void dispatcher(tb_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool any = false;
        for (size_t k = 0; k < S->running.size(); ++k) {
            if (!S->running[k]) continue;
            const cudaError_t e = cudaEventQuery(S->slot_done[k]);
            if (e == cudaErrorNotReady) {
                any = true;
                continue;
            }
            finish(S, (int)k);
        }
        while (!S->queue.empty()) {  // arrival order: the head waits for room
            int k = -1;
            for (size_t i = 0; i < S->running.size(); ++i)
                if (!S->running[i]) { k = (int)i; break; }
            if (k < 0) break;
            auto R = S->queue.front();
            if (!admit(S, R, k)) break;
            S->queue.pop_front();
            if (R->status != TB_OK && !S->running[k]) {  // failed before launch
                R->done = true;
                S->cv_done.notify_all();
            }
            any = true;
        }
        if (S->stop && S->queue.empty() && !any) break;
        if (any) S->cv_work.wait_for(lk, std::chrono::microseconds(50));
        else S->cv_work.wait(lk);
    }
}

std::atomic<uint64_t> g_plan_uid{1};

}  // namespace

namespace tb {
uint64_t next_plan_uid() { return g_plan_uid++; }
}  // namespace tb

extern "C" {

int tb_server_create(const tb_server_opts* opts, tb_server** out) {
    if (!out) return fail(TB_EINVAL, "out is NULL");
    *out = nullptr;
    tb_server_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.hbm_budget_bytes <= 0) o.hbm_budget_bytes = (int64_t)16 << 30;
    if (o.slots <= 0) o.slots = 4;
    if (o.slots > 64) return fail(TB_EINVAL, "at most 64 slots");
    if (o.pinned_bytes <= 0) o.pinned_bytes = (int64_t)64 << 20;
    tb_server* S = nullptr;
    try {
        S = new tb_server;
    } catch (const std::bad_alloc&) {
        return fail(TB_ENOMEM, "host allocation failed");
    }
    S->device = o.device;
    S->budget = align_up(o.hbm_budget_bytes, 256);
    S->pinned_bytes = align_up(o.pinned_bytes, 256);
    int rc = TB_OK;
    if (cudaSetDevice(S->device) != cudaSuccess) rc = fail(TB_ECUDA, "cudaSetDevice failed");
    if (rc == TB_OK && cudaMalloc(&S->arena_base, (size_t)S->budget) != cudaSuccess)
        rc = fail(TB_ENOMEM, "cannot allocate the HBM budget of " + std::to_string(S->budget) + " bytes");
    if (rc == TB_OK && cudaHostAlloc(reinterpret_cast<void**>(&S->pinned), (size_t)S->pinned_bytes,
                                     cudaHostAllocDefault) != cudaSuccess)
        rc = fail(TB_ENOMEM, "cannot allocate pinned staging");
    for (int k = 0; k < o.slots && rc == TB_OK; ++k) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            rc = fail(TB_ECUDA, "stream or event creation failed");
            break;
        }
        S->slots.push_back(st);
        S->slot_done.push_back(ev);
    }
    if (rc != TB_OK) {
        for (auto e : S->slot_done) cudaEventDestroy(e);
        for (auto st : S->slots) cudaStreamDestroy(st);
        if (S->pinned) cudaFreeHost(S->pinned);
        if (S->arena_base) cudaFree(S->arena_base);
        delete S;
        return rc;
    }
    S->arena.reset(S->budget);
    S->pinned_arena.reset(S->pinned_bytes);
    S->running.resize(S->slots.size());
    S->worker = std::thread(dispatcher, S);
    *out = S;
    return TB_OK;
}

int tb_server_submit(tb_server* S, const tb_plan* plan, const uint8_t* bits, int64_t nb, double* out,
                     int64_t* ticket) {
    if (!S || !plan || !bits || !out || !ticket || nb <= 0) return fail(TB_EINVAL, "NULL argument or nb <= 0");
    const Plan& P = plan->p;
    if (P.h > MAX_H) return fail(TB_EDOMAIN, "boundary wider than 2^33 entries");
    if (P.open_k) return fail(TB_EINVAL, "open plans are evaluated by tb_amplitudes / tb_amplitudes_device");
    for (int64_t i = 0; i < nb * P.n; ++i)
        if (bits[i] > 1) return fail(TB_EINVAL, "bitstring entries must be 0 or 1");
    const CallLayout c = call_layout(P);
    if (align_up(P.lay.total, 256) + staging_len(P, nb) + c.per_b > S->budget)
        return fail(TB_ENOMEM, "request needs more than the server's HBM budget");
    if (staging_len(P, nb) > S->pinned_bytes) return fail(TB_ENOMEM, "request needs more than the pinned staging");
    std::shared_ptr<Request> R;
    try {
        R = std::make_shared<Request>();
        R->bits.assign(bits, bits + nb * P.n);
    } catch (const std::bad_alloc&) {
        return fail(TB_ENOMEM, "host allocation failed");
    }
    R->plan = plan;
    R->nb = nb;
    R->out = out;
    R->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        R->ticket = S->next_ticket++;
        S->all[R->ticket] = R;
        S->queue.push_back(R);
    }
    S->cv_work.notify_one();
    *ticket = R->ticket;
    return TB_OK;
}

int tb_server_wait(tb_server* S, int64_t ticket, double timeout_s, tb_request_stats* stats) {
    if (!S) return fail(TB_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(TB_EINVAL, "unknown ticket");
    auto R = it->second;
    auto ready = [&] { return R->done; };
    if (timeout_s < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready))
        return fail(TB_ETIMEOUT, "request still running");
    if (stats) {
        stats->latency_s = std::chrono::duration<double>(R->t_done - R->t_submit).count();
        stats->queue_s = R->t_admit.time_since_epoch().count()
                             ? std::chrono::duration<double>(R->t_admit - R->t_submit).count()
                             : 0.0;
        stats->run_s = stats->latency_s - stats->queue_s;
        stats->status = R->status;
        stats->slot = R->slot;
    }
    S->all.erase(it);
    return R->status;
}

int tb_server_stats(tb_server* S, tb_server_stats_t* out) {
    if (!S || !out) return fail(TB_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = S->completed;
    out->amplitudes = S->amplitudes;
    out->peak_concurrent = S->peak_running;
    out->peak_bytes_in_use = S->peak_used;
    out->queued = (int64_t)S->queue.size();
    std::vector<double> l = S->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (double)(l.size() - 1) + 0.5))]; };
        out->p50_latency_s = q(0.50);
        out->p99_latency_s = q(0.99);
        double m = 0;
        for (double x : l) m += x;
        out->mean_latency_s = m / (double)l.size();
    }
    return TB_OK;
}

void tb_server_destroy(tb_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();  // finishes every queued request first
    cudaSetDevice(S->device);
    for (auto e : S->slot_done) cudaEventDestroy(e);
    for (auto st : S->slots) cudaStreamDestroy(st);
    if (S->pinned) cudaFreeHost(S->pinned);
    if (S->arena_base) cudaFree(S->arena_base);
    delete S;
}

}  // extern "C"
