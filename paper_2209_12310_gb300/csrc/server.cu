// server.cu -- continuous-batching hull server (ch_server_* / ch_submit / ch_poll).
//
// A server owns one device arena carved from its memory budget, an engine
// thread and kSlots (3) CUDA streams.  ch_submit only appends a request to the
// admission queue (O(1), never touches the GPU, never copies: the caller's
// buffer is read when the request is admitted into a batch and must stay
// valid until ch_poll answers for it).  The engine thread repeatedly
//   1. retires finished batches (result counts first, then the index lists,
//      both copied back asynchronously and observed through CUDA events),
//   2. forms a new batch from the queue head while a free stream slot exists
//      and the arena has a contiguous block for the batch (admission by
//      memory: a request waits until memory frees up),
//   3. copies the batch's points in and enqueues the batched hull on it (no
//      host wait; sets the batched kernels leave to the single-hull path are
//      finished when the batch retires).
// Batch slots on separate streams let new batches start while earlier ones
// are still on the GPU, so one batch's copies overlap another's kernels and
// requests that arrive during a batch do not wait for it; a batch takes at
// most 1 / kSlots of the arena's points so that the slots' batches fit side
// by side.  Every request's result is computed by the same kernels as
// ch_hull on that request alone.
#include "ch_internal.cuh"
#include "host.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace ch {
namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t ticket = 0;
    const float* host = nullptr;
    int64_t n = 0;
    int state = 0;          // 0 queued, 1 running, 2 done, 3 failed
    int status = CH_OK;
    int64_t h = 0;
    std::vector<int32_t> result;
    double t_submit = 0, t_done = 0;
};

// First-fit allocator of contiguous byte ranges inside the device arena.
class Arena {
  public:
    void init(size_t bytes) { free_[0] = bytes; size_ = bytes; }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, o = it->first + bytes;
                free_.erase(it);
                if (rest) free_[o] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_.emplace(off, bytes).first;
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
    size_t size() const { return size_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0;
};

struct Slot {
    bool busy = false;
    int phase = 0;   // 1: waiting for counts, 2: waiting for indices
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t te[4] = {};        // timing: copies in start / end, hull and counts end, indices end
    double t_form = 0;             // host time the batch was formed
    int64_t batch_points = 0;
    int redo_sets = 0;             // sets the batched kernels left to the single-hull path
    std::vector<Req*> reqs;
    std::vector<int64_t> off;       // host copy of the batch offsets
    int64_t* h_off = nullptr;       // pinned offsets (k + 1)
    int64_t* h_n = nullptr;         // pinned result counts (k)
    unsigned char* h_redo = nullptr;  // pinned flags of sets left to the single-hull path (k)
    bool redone = false;
    int32_t* h_idx = nullptr;       // pinned result indices
    size_t h_idx_cap = 0;
    size_t cap_k = 0;
    size_t arena_off = 0, arena_bytes = 0;
};

constexpr size_t kMaxQueue = 1u << 17;
constexpr int kBatchTrace = 8;
constexpr size_t kMaxTrace = 1u << 20;   // batches traced at most
constexpr int kMaxBatch = 4096;
constexpr int kSlots = 3;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }
size_t batch_bytes(int64_t points, size_t k) {
    return align256(8 * (size_t)points) + align256(4 * (size_t)points) + align256(8 * (k + 1)) +
           align256(8 * k);
}

}  // namespace

struct Server {
    int device = 0;
    size_t budget = 0;
    char* arena_base = nullptr;
    Arena arena;
    int64_t max_points = 0;     // largest batch the reserved workspace covers
    Slot slots[kSlots];
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req*> queue;
    std::unordered_map<uint64_t, Req*> reqs;
    uint64_t next_ticket = 1;
    std::atomic<bool> stop{false};
    std::thread engine;
    std::vector<double> lat_ms;
    std::vector<double> trace;   // per batch: kBatchTrace values (ch_server_trace)
    int64_t served_points = 0, completed = 0;
    double t_first = 0, t_last = 0;
    int fatal = CH_OK;

    void run();
    bool retire(Slot& sl);
    bool launch(Slot& sl);
};

bool Server::retire(Slot& sl) {
    if (!sl.busy) return false;
    const cudaError_t q = cudaEventQuery(sl.ev);
    if (q == cudaErrorNotReady) return false;
    if (q != cudaSuccess) {
        std::lock_guard<std::mutex> lk(mu);
        for (Req* r : sl.reqs) { r->state = 3; r->status = CH_ECUDA; }
        fatal = CH_ECUDA;
        sl.busy = false;
        return true;
    }
    const size_t k = sl.reqs.size();
    char* base = arena_base + sl.arena_off;
    const int64_t total = sl.off[k];
    int32_t* d_idx = (int32_t*)(base + align256(8 * (size_t)total));
    if (sl.phase == 1 && !sl.redone) {   // sets the batched kernels left to the single-hull path
        sl.redone = true;
        bool any = false;
        for (size_t i = 0; i < k; ++i) any |= sl.h_redo[i] != 0;
        if (any) {
            float* d_pts = (float*)base;
            int64_t* d_n = (int64_t*)(base + align256(8 * (size_t)total) + align256(4 * (size_t)total) +
                                      align256(8 * (k + 1)));
            if (hull_batched_redo(d_pts, sl.h_off, (int32_t)k, d_idx, d_n, sl.h_redo, sl.s) != CH_OK)
                cudaMemsetAsync(d_n, 0xFF, 8 * k, sl.s);
            cudaMemcpyAsync(sl.h_n, d_n, 8 * k, cudaMemcpyDeviceToHost, sl.s);
            cudaEventRecord(sl.ev, sl.s);
            sl.redo_sets = 0;
            for (size_t i = 0; i < k; ++i) sl.redo_sets += sl.h_redo[i] != 0;
            return true;
        }
    }
    if (sl.phase == 1) {
        size_t hsum = 0;
        for (size_t i = 0; i < k; ++i) hsum += sl.h_n[i] > 0 ? (size_t)sl.h_n[i] : 0;
        if (hsum > sl.h_idx_cap) {
            if (sl.h_idx) cudaFreeHost(sl.h_idx);
            sl.h_idx_cap = std::max(hsum, 2 * sl.h_idx_cap);
            if (cudaMallocHost((void**)&sl.h_idx, sl.h_idx_cap * sizeof(int32_t)) != cudaSuccess) {
                sl.h_idx = nullptr;
                sl.h_idx_cap = 0;
            }
        }
        size_t o = 0;
        for (size_t i = 0; i < k && sl.h_idx; ++i) {
            const int64_t h = sl.h_n[i];
            if (h > 0) {
                cudaMemcpyAsync(sl.h_idx + o, d_idx + sl.off[i], 4 * (size_t)h, cudaMemcpyDeviceToHost, sl.s);
                o += (size_t)h;
            }
        }
        cudaEventRecord(sl.te[3], sl.s);
        cudaEventRecord(sl.ev, sl.s);
        sl.phase = 2;
        return true;
    }
    // phase 2: results are on the host
    const double t = now_s();
    std::lock_guard<std::mutex> lk(mu);
    size_t o = 0;
    for (size_t i = 0; i < k; ++i) {
        Req* r = sl.reqs[i];
        const int64_t h = sl.h_n[i];
        if (h < 0 || !sl.h_idx) {
            r->state = 3;
            r->status = h < 0 ? (int)h : CH_ENOMEM;
        } else {
            r->h = h;
            r->result.assign(sl.h_idx + o, sl.h_idx + o + h);
            o += (size_t)h;
            r->state = 2;
        }
        r->t_done = t;
        lat_ms.push_back((t - r->t_submit) * 1e3);
        served_points += r->n;
        ++completed;
        t_last = t;
    }
    if (trace.size() < kMaxTrace * kBatchTrace) {
        float h2d = 0.f, hull = 0.f, idx = 0.f;
        if (cudaEventElapsedTime(&h2d, sl.te[0], sl.te[1]) != cudaSuccess) h2d = -1.f;
        if (cudaEventElapsedTime(&hull, sl.te[1], sl.te[2]) != cudaSuccess) hull = -1.f;
        if (cudaEventElapsedTime(&idx, sl.te[2], sl.te[3]) != cudaSuccess) idx = -1.f;
        const double v[kBatchTrace] = {(sl.t_form - t_first) * 1e3, (double)k, (double)sl.batch_points,
                                       (double)h2d, (double)hull, (double)idx, (t - sl.t_form) * 1e3,
                                       (double)sl.redo_sets};
        trace.insert(trace.end(), v, v + kBatchTrace);
    }
    arena.release(sl.arena_off, sl.arena_bytes);
    sl.reqs.clear();
    sl.busy = false;
    sl.phase = 0;
    return true;
}

bool Server::launch(Slot& sl) {
    if (sl.busy) return false;
    std::vector<Req*> batch;
    int64_t points = 0;
    size_t off = 0, bytes = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        // FIFO admission: take queue-head requests while the batch still fits
        // the workspace and a contiguous arena block exists for it.  A batch
        // takes at most 1 / kSlots of the arena's points (a single request
        // may take more), so that the other slots' batches fit beside it.
        const int64_t cap = std::max<int64_t>(max_points / kSlots, 1);
        while (!queue.empty() && (int)batch.size() < kMaxBatch) {
            Req* r = queue.front();
            const int64_t np = points + r->n;
            if (np > max_points || (!batch.empty() && np > cap)) break;
            if (batch_bytes(np, batch.size() + 1) > arena.size()) break;
            batch.push_back(r);
            points = np;
            queue.pop_front();
        }
        if (batch.empty()) return false;
        // shrink until an arena block is available (memory is freed by retire)
        while (!batch.empty()) {
            bytes = batch_bytes(points, batch.size());
            if (arena.alloc(bytes, &off)) break;
            Req* r = batch.back();
            batch.pop_back();
            points -= r->n;
            queue.push_front(r);
        }
        if (batch.empty()) return false;
        for (Req* r : batch) r->state = 1;
    }
    const size_t k = batch.size();
    if (sl.cap_k < k) {
        if (sl.h_off) cudaFreeHost(sl.h_off);
        if (sl.h_n) cudaFreeHost(sl.h_n);
        if (sl.h_redo) cudaFreeHost(sl.h_redo);
        sl.cap_k = std::max<size_t>(k, 256);
        cudaMallocHost((void**)&sl.h_off, 8 * (sl.cap_k + 1));
        cudaMallocHost((void**)&sl.h_n, 8 * sl.cap_k);
        cudaMallocHost((void**)&sl.h_redo, sl.cap_k);
    }
    sl.off.assign(k + 1, 0);
    for (size_t i = 0; i < k; ++i) sl.off[i + 1] = sl.off[i] + batch[i]->n;
    std::memcpy(sl.h_off, sl.off.data(), 8 * (k + 1));
    char* base = arena_base + off;
    float* d_pts = (float*)base;
    int32_t* d_idx = (int32_t*)(base + align256(8 * (size_t)points));
    int64_t* d_off = (int64_t*)(base + align256(8 * (size_t)points) + align256(4 * (size_t)points));
    int64_t* d_n = (int64_t*)((char*)d_off + align256(8 * (k + 1)));
    sl.t_form = now_s();
    sl.batch_points = points;
    sl.redo_sets = 0;
    cudaEventRecord(sl.te[0], sl.s);
    for (size_t i = 0; i < k; ++i)
        cudaMemcpyAsync(d_pts + 2 * sl.off[i], batch[i]->host, 8 * (size_t)batch[i]->n, cudaMemcpyHostToDevice,
                        sl.s);
    cudaMemcpyAsync(d_off, sl.h_off, 8 * (k + 1), cudaMemcpyHostToDevice, sl.s);
    cudaEventRecord(sl.te[1], sl.s);
    std::memset(sl.h_redo, 0, k);
    sl.redone = false;
    // no host synchronisation: the batch overlaps with the other slot's
    const int st = hull_batched_impl(d_pts, d_off, (int32_t)k, d_idx, d_n, sl.h_off, sl.s, false, sl.h_redo);
    if (st != CH_OK) cudaMemsetAsync(d_n, 0xFF, 8 * k, sl.s);   // -1 = CH_EINVAL per set
    cudaMemcpyAsync(sl.h_n, d_n, 8 * k, cudaMemcpyDeviceToHost, sl.s);
    cudaEventRecord(sl.te[2], sl.s);
    cudaEventRecord(sl.ev, sl.s);
    sl.reqs = std::move(batch);
    sl.arena_off = off;
    sl.arena_bytes = bytes;
    sl.phase = 1;
    sl.busy = true;
    return true;
}

void Server::run() {
    cudaSetDevice(device);
    while (!stop.load()) {
        bool progress = false;
        for (auto& sl : slots) progress |= retire(sl);
        for (auto& sl : slots) progress |= launch(sl);
        if (!progress) {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

}  // namespace ch

using namespace ch;

extern "C" {

int ch_server_create(size_t budget_bytes, int device, void** srv) {
    if (!srv || budget_bytes < (64u << 20)) return CH_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return CH_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    Server* S = new Server();
    S->device = device;
    S->budget = budget_bytes;
    // Split of the budget: per point a batch needs 12 bytes of arena (points
    // in, indices out) and about ws bytes of single-hull workspace on each
    // slot stream (sets left to that path).  Each slot's batched workspace,
    // reserved below for batches of up to max_points points in kMaxBatch sets,
    // comes on top of the budget.
    const double ws_pp = (double)ch_workspace_bytes(1 << 20) / (double)(1 << 20);
    const double per_point = 12.0 + (double)kSlots * ws_pp;
    S->max_points = (int64_t)((double)budget_bytes / per_point);
    const size_t arena_bytes = align256((size_t)(12.0 * (double)S->max_points) + (size_t)kMaxBatch * 64 + (1u << 20));
    int st = CH_OK;
    if (cudaMalloc((void**)&S->arena_base, arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        st = CH_ENOMEM;
    }
    for (int i = 0; st == CH_OK && i < kSlots; ++i) {
        if (cudaStreamCreateWithFlags(&S->slots[i].s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&S->slots[i].ev, cudaEventDisableTiming) != cudaSuccess)
            st = CH_ECUDA;
        for (int e = 0; st == CH_OK && e < 4; ++e)
            if (cudaEventCreate(&S->slots[i].te[e]) != cudaSuccess) st = CH_ECUDA;
        if (st == CH_OK) st = ch_reserve(S->max_points, kMaxBatch, S->slots[i].s);
    }
    if (st != CH_OK) {
        for (auto& sl : S->slots) {
            if (sl.ev) cudaEventDestroy(sl.ev);
            for (cudaEvent_t e : sl.te)
                if (e) cudaEventDestroy(e);
            if (sl.s) cudaStreamDestroy(sl.s);
        }
        if (S->arena_base) cudaFree(S->arena_base);
        delete S;
        cudaSetDevice(prev);
        return st;
    }
    S->arena.init(arena_bytes);
    S->engine = std::thread([S] { S->run(); });
    cudaSetDevice(prev);
    *srv = S;
    return CH_OK;
}

int ch_submit(void* srv, const float* pts_host, int64_t n, uint64_t* ticket) {
    Server* S = (Server*)srv;
    if (!S || !ticket || n < 0 || (n > 0 && !pts_host)) return CH_EINVAL;
    if (((uintptr_t)pts_host & 7u) != 0u) return CH_EINVAL;
    if (n > S->max_points || batch_bytes(n, 1) > S->arena.size()) return CH_ENOMEM;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal != CH_OK) return S->fatal;
    if (S->queue.size() >= kMaxQueue) return CH_EBUSY;
    Req* r = new Req();
    r->ticket = S->next_ticket++;
    r->host = pts_host;
    r->n = n;
    r->t_submit = now_s();
    if (S->t_first == 0) S->t_first = r->t_submit;
    S->reqs[r->ticket] = r;
    S->queue.push_back(r);
    *ticket = r->ticket;
    S->cv.notify_one();
    return CH_OK;
}

int ch_poll(void* srv, uint64_t ticket, int32_t* out_idx_host, int64_t cap, int64_t* out_n) {
    Server* S = (Server*)srv;
    if (!S || !out_n) return CH_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return CH_EINVAL;
    Req* r = it->second;
    if (r->state == 0 || r->state == 1) return CH_PENDING;
    int st = CH_OK;
    if (r->state == 3) {
        st = r->status;
        *out_n = r->status;
    } else {
        *out_n = r->h;
        if (r->h > cap || (r->h > 0 && !out_idx_host)) {
            return CH_EINVAL;   // keep the result; caller may retry with a larger buffer
        }
        if (r->h > 0) std::memcpy(out_idx_host, r->result.data(), 4 * (size_t)r->h);
    }
    S->reqs.erase(it);
    delete r;
    return st;
}

int ch_server_stats(void* srv, double* p50_ms, double* p99_ms, double* points_per_s, int64_t* completed) {
    Server* S = (Server*)srv;
    if (!S) return CH_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> v = S->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
        if (v.empty()) return 0.0;
        const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
        return v[i];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (points_per_s) {
        const double dt = S->t_last - S->t_first;
        *points_per_s = dt > 0 ? (double)S->served_points / dt : 0.0;
    }
    if (completed) *completed = S->completed;
    return CH_OK;
}

int ch_server_trace(void* srv, double* out, int64_t cap) {
    Server* S = (Server*)srv;
    if (!S || cap < 0 || (cap > 0 && !out)) return CH_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    const int64_t n = (int64_t)(S->trace.size() / kBatchTrace);
    const int64_t m = std::min(n, cap);
    if (m > 0) std::memcpy(out, S->trace.data(), sizeof(double) * kBatchTrace * (size_t)m);
    return (int)std::min<int64_t>(n, INT32_MAX);
}

int ch_server_destroy(void* srv) {
    Server* S = (Server*)srv;
    if (!S) return CH_EINVAL;
    S->stop.store(true);
    S->cv.notify_all();
    if (S->engine.joinable()) S->engine.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto& sl : S->slots) {
        if (sl.s) cudaStreamSynchronize(sl.s);
        if (sl.ev) cudaEventDestroy(sl.ev);
        for (cudaEvent_t e : sl.te)
            if (e) cudaEventDestroy(e);
        if (sl.h_off) cudaFreeHost(sl.h_off);
        if (sl.h_n) cudaFreeHost(sl.h_n);
        if (sl.h_redo) cudaFreeHost(sl.h_redo);
        if (sl.h_idx) cudaFreeHost(sl.h_idx);
        for (Req* r : sl.reqs) S->reqs.erase(r->ticket), delete r;
    }
    for (auto& kv : S->reqs) delete kv.second;
    S->reqs.clear();
    if (S->arena_base) cudaFree(S->arena_base);
    for (auto& sl : S->slots) {
        if (!sl.s) continue;
        release_stream_workspace(S->device, sl.s);
        cudaStreamDestroy(sl.s);
    }
    cudaSetDevice(prev);
    delete S;
    return CH_OK;
}

}  // extern "C"
