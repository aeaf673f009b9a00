// api.cu -- C ABI entry points (ch.h): argument checks, workspace management,
// launch sequences and device-timed kernel statistics.
#include "ch_internal.cuh"
#include "launch.h"
#include "host.h"

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

namespace ch {

// ---------------------------------------------------------------------------
// Device information (SM count, resident blocks per SM of every kernel).
struct DevInfo {
    int sms = 0;
    int occ_main = 1, occ_post = 1, occ_lab = 1, occ_sort = 1, occ_chain = 1;
};

static std::mutex g_mu;
static std::map<int, DevInfo> g_dev;

static int device_info(int dev, DevInfo* out) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_dev.find(dev);
    if (it != g_dev.end()) { *out = it->second; return CH_OK; }
    DevInfo di;
    if (cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CH_ECUDA;
    if (configure_hull_kernels() != cudaSuccess) return CH_ECUDA;
    if (configure_filter_kernels() != cudaSuccess) return CH_ECUDA;
    if (configure_post_kernel() != cudaSuccess) return CH_ECUDA;
    if (configure_bucket_kernels() != cudaSuccess) return CH_ECUDA;
    if (configure_star_kernel() != cudaSuccess) return CH_ECUDA;
    if (occupancy_filter(&di.occ_main, &di.occ_lab) != cudaSuccess) return CH_ECUDA;
    if (occupancy_post(&di.occ_post) != cudaSuccess) return CH_ECUDA;
    if (occupancy_sort(&di.occ_sort) != cudaSuccess) return CH_ECUDA;
    if (occupancy_chain(&di.occ_chain) != cudaSuccess) return CH_ECUDA;
    di.occ_main = std::max(1, di.occ_main);
    di.occ_post = std::max(1, di.occ_post);
    di.occ_lab = std::max(1, di.occ_lab);
    di.occ_sort = std::max(1, di.occ_sort);
    di.occ_chain = std::max(1, di.occ_chain);
    g_dev[dev] = di;
    *out = di;
    return CH_OK;
}

// ---------------------------------------------------------------------------
// Workspace layout for one hull of up to n points.
static size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

Layout make_layout(long long n) {
    Layout L{};
    L.cap = n + 16;
    L.sort_tiles = (L.cap + kSortTile - 1) / kSortTile;
    L.bmax = L.cap / kBkAvg + 4 * kBkMinQ + 8;
    // chain tiles: sorted records (one per kChainTile) or bucket chains (one
    // per kBkGroup buckets of each queue), whichever needs more
    L.ctcap = std::max((L.cap + kChainTile - 1) / kChainTile + 4, L.bmax / kBkGroup + 8);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t r = o;
        o = align_up(o + bytes);
        return r;
    };
    // zeroed at allocation: the control block, the sort's look-back status
    // words and the merge tree's arrival counters (each kernel leaves them
    // in that state for the next call)
    L.off_ctl = take(sizeof(Ctl));
    L.off_status = take(8 * (size_t)kDigits * L.sort_tiles);
    L.off_counters = take(4 * (size_t)kMaxLevels * L.ctcap);
    L.off_star_bins = take(star_bins_bytes());   // the star and post passes leave them at zero
    L.zero_bytes = o;
    L.off_kA = take(4 * (size_t)L.cap);
    L.off_kB = take(4 * (size_t)L.cap);
    L.off_vA = take(8 * (size_t)L.cap);
    L.off_vB = take(8 * (size_t)L.cap);
    L.off_cu = take(4 * (size_t)L.ctcap * kChainTile);
    L.off_cv = take(4 * (size_t)L.ctcap * kChainTile);
    L.off_ci = take(4 * (size_t)L.ctcap * kChainTile);
    L.off_clen = take(4 * (size_t)L.ctcap);
    L.off_bcount = take(4 * (size_t)L.bmax);
    L.off_bcur = take(4 * (size_t)L.bmax);
    L.off_bstart = take(4 * (size_t)L.bmax);
    L.off_bsum = take(4 * ((size_t)L.bmax / 1024 + 2 + 2 * (size_t)kBkCoarseMax + 1));   // block sums, cursors, tiles
    L.off_blen = take(4 * (size_t)L.bmax);
    L.off_bu = take(4 * (size_t)L.bmax * kBkChain);
    L.off_bv = take(4 * (size_t)L.bmax * kBkChain);
    L.off_bi = take(4 * (size_t)L.bmax * kBkChain);
    L.total = o;
    return L;
}

struct Workspace {
    char* base = nullptr;
    size_t bytes = 0;
    long long n_cap = -1;
    // staging for the host-buffer entry point
    char* stage = nullptr;
    size_t stage_bytes = 0;
    // the star pass's branch: a stream of its own, forked from and joined
    // back into the caller's stream by two events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

static std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

void drop_graphs(int dev, cudaStream_t s);

static int grow_workspace(Workspace& ws, long long n, cudaStream_t s, int dev) {
    if (n <= ws.n_cap) return CH_OK;
    drop_graphs(dev, s);
    const long long want = std::max(n, (long long)(ws.n_cap > 0 ? ws.n_cap + ws.n_cap / 4 : n));
    const Layout L = make_layout(want);
    if (ws.base) {
        cudaStreamSynchronize(s);
        if (ws.side) cudaStreamSynchronize(ws.side);
        cudaFree(ws.base);
        ws.base = nullptr;
        ws.bytes = 0;
        ws.n_cap = -1;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, L.total) != cudaSuccess) {
        cudaGetLastError();
        return CH_ENOMEM;
    }
    if (cudaMemsetAsync(p, 0, L.zero_bytes, s) != cudaSuccess) {
        cudaFree(p);
        return CH_ECUDA;
    }
    ws.base = (char*)p;
    ws.bytes = L.total;
    ws.n_cap = want;
    return CH_OK;
}

int get_workspace(int dev, cudaStream_t s, long long n, char** base, Layout* L) {
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace& ws = g_ws[std::make_pair(dev, s)];
    const int st = grow_workspace(ws, n, s, dev);
    if (st != CH_OK) return st;
    *base = ws.base;
    *L = make_layout(ws.n_cap);
    return CH_OK;
}

static void free_workspace(Workspace& w, cudaStream_t s) {
    cudaStreamSynchronize(s);
    if (w.side) cudaStreamSynchronize(w.side);
    if (w.base) cudaFree(w.base);
    if (w.stage) cudaFree(w.stage);
    if (w.ev_fork) cudaEventDestroy(w.ev_fork);
    if (w.ev_join) cudaEventDestroy(w.ev_join);
    if (w.side) cudaStreamDestroy(w.side);
    w = Workspace();
}

void release_stream_workspace(int dev, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ws.find(std::make_pair(dev, s));
    drop_batched_graphs(dev, s);
    release_batched_stream(dev, s);
    if (it == g_ws.end()) return;
    drop_graphs(dev, s);
    free_workspace(it->second, s);
    g_ws.erase(it);
}

// The star pass's stream and events of (dev, s), created on first use;
// false when they cannot be (the hull then runs without the star pass).
static bool get_side(int dev, cudaStream_t s, cudaStream_t* side, cudaEvent_t* fork, cudaEvent_t* join) {
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace& ws = g_ws[std::make_pair(dev, s)];
    if (!ws.side) {
        cudaStream_t st = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
            if (st) cudaStreamDestroy(st);
            if (a) cudaEventDestroy(a);
            cudaGetLastError();
            return false;
        }
        ws.side = st;
        ws.ev_fork = a;
        ws.ev_join = b;
    }
    *side = ws.side;
    *fork = ws.ev_fork;
    *join = ws.ev_join;
    return true;
}

static int get_stage(int dev, cudaStream_t s, size_t bytes, char** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace& ws = g_ws[std::make_pair(dev, s)];
    if (ws.stage_bytes < bytes) {
        if (ws.stage) {
            cudaStreamSynchronize(s);
            cudaFree(ws.stage);
            ws.stage = nullptr;
            ws.stage_bytes = 0;
        }
        void* p = nullptr;
        const size_t want = std::max(bytes, ws.stage_bytes + ws.stage_bytes / 4);
        if (cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            return CH_ENOMEM;
        }
        ws.stage = (char*)p;
        ws.stage_bytes = want;
    }
    *out = ws.stage;
    return CH_OK;
}

// ---------------------------------------------------------------------------
// Device-timed statistics: CUDA events recorded on the launching stream.
struct ProfPending {
    const char* name;
    cudaEvent_t a, b;
};
static bool g_prof = false;
static std::mutex g_prof_mu;
static std::vector<ProfPending> g_pending;
static std::vector<cudaEvent_t> g_event_pool;
static std::map<std::string, std::pair<long long, double>> g_acc;
static std::vector<std::string> g_names;   // stable storage for names returned to callers

bool prof_enabled() { return g_prof; }

static cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfScope::ProfScope(const char* name, cudaStream_t s) : name_(name), s_(s), a_(nullptr) {
    if (!g_prof) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    a_ = take_event();
    cudaEventRecord((cudaEvent_t)a_, s_);
}

ProfScope::~ProfScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t b = take_event();
    cudaEventRecord(b, s_);
    g_pending.push_back(ProfPending{name_, (cudaEvent_t)a_, b});
}

static void prof_drain() {
    for (auto& p : g_pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        auto& acc = g_acc[p.name];
        acc.first += 1;
        acc.second += ms;
        g_event_pool.push_back(p.a);
        g_event_pool.push_back(p.b);
    }
    g_pending.clear();
}

// ---------------------------------------------------------------------------
// The launch sequence of one hull (n >= 1) on an allocated workspace, in two
// parts: the filter (init .. post), after which small survivor sets are done,
// and the large-survivor path (buckets, the sort fallback, the chain merge).
// `cond`, when non-zero, is a graph condition the post pass raises when the
// second part has work (see the CUDA-graph cache below).
struct HullLaunch {
    DevInfo di;
    Ctl* ctl;
    uint32_t *kA, *kB;
    uint64_t *vA, *vB;
    int head;
    long long ntiles;
    // the star pass (dense data): its branch and its buffers; side is null
    // when the input is too small for it
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    void* star_bins;
};

// Inputs below this many warp tiles skip the star pass.
constexpr long long kStarMinTiles = 256;

// owner: the caller's stream, whose workspace (and star branch) the launches use.
static int hull_setup(const float* pts, long long n, int dev, cudaStream_t owner, char* base, const Layout& L,
                      HullLaunch* h) {
    int st = device_info(dev, &h->di);
    if (st != CH_OK) return st;
    h->ctl = (Ctl*)(base + L.off_ctl);
    h->kA = (uint32_t*)(base + L.off_kA);
    h->kB = (uint32_t*)(base + L.off_kB);
    h->vA = (uint64_t*)(base + L.off_vA);
    h->vB = (uint64_t*)(base + L.off_vB);
    h->head = (((uintptr_t)pts & 15u) != 0u && n > 0) ? 1 : 0;
    h->ntiles = (n - h->head) / kWarpTilePts;
    h->star_bins = base + L.off_star_bins;
    h->side = nullptr;
    h->ev_fork = h->ev_join = nullptr;
    if (h->ntiles >= kStarMinTiles && !get_side(dev, owner, &h->side, &h->ev_fork, &h->ev_join)) h->side = nullptr;
    return CH_OK;
}

static void enqueue_filter_part(const float* pts, long long n, int32_t* out_idx, int64_t* out_n, cudaStream_t s,
                                const HullLaunch& h, unsigned long long cond) {
    const long long samples = sample_tiles_host(h.ntiles);
    const int grid_sample = (int)std::max<long long>(1, std::min<long long>(256, (samples + 7) / 8));
    // Raw survivors of the fused pass live in the B buffers until the post
    // pass has turned them into sort records in the A buffers.
    uint64_t* raw_xy = h.vB;
    uint32_t* raw_idx = h.kB;
    const unsigned switch_at = (unsigned)std::max<long long>(1 << 16, n >> 5);
    { ProfScope p("init", s); launch_init(h.ctl, 0, s); }
    { ProfScope p("sample", s); launch_sample(pts, n, h.head, h.ntiles, h.ctl, grid_sample, s); }
    // The star pass needs only the sample octagon: it runs on its own branch
    // beside the main pass, and the post pass waits for both.  The main pass
    // is enqueued first, so that its blocks are placed before the star pass's.
    const bool star = h.side != nullptr;
    if (star) cudaEventRecord(h.ev_fork, s);
    {
        ProfScope p("main_filter", s);
        launch_main(pts, n, h.head, h.ntiles, h.ctl, raw_xy, raw_idx, switch_at, h.kA, h.vA,
                    h.di.sms * h.di.occ_main, s);
    }
    if (star) {
        cudaStreamWaitEvent(h.side, h.ev_fork, 0);
        {
            ProfScope p("star", h.side);
            launch_star(pts, n, h.head, h.ntiles, h.ctl, h.star_bins, h.di.sms, h.side);
        }
        cudaEventRecord(h.ev_join, h.side);
        cudaStreamWaitEvent(s, h.ev_join, 0);
    }
    {
        ProfScope p("post", s);
        launch_post(pts, n, h.head, h.ntiles, h.ctl, raw_xy, raw_idx, h.kA, h.vA, out_idx, out_n,
                    star ? h.star_bins : nullptr, cond, h.di.sms * h.di.occ_post, s);
    }
}

static void enqueue_large_part(const float* pts, long long n, int32_t* out_idx, int64_t* out_n, cudaStream_t s,
                               char* base, const Layout& L, const HullLaunch& h) {
    Ctl* ctl = h.ctl;
    unsigned long long* status = (unsigned long long*)(base + L.off_status);
    launch_bucket_pass(ctl, h.kA, h.vA, h.kB, h.vB, (unsigned*)(base + L.off_bcount), (unsigned*)(base + L.off_bcur),
                       (unsigned*)(base + L.off_bstart), (unsigned*)(base + L.off_bsum), (int*)(base + L.off_bu), (int*)(base + L.off_bv),
                       (int*)(base + L.off_bi), (int*)(base + L.off_blen), (unsigned)L.bmax, h.di.sms, s);
    {
        ProfScope p("sort", s);
        const int grid_sort = h.di.sms * h.di.occ_sort;
        launch_sort_hist(h.kA, ctl, h.di.sms, s);
        launch_sort_pass(h.kA, h.vA, h.kB, h.vB, ctl, status, 0, grid_sort, s);
        launch_sort_pass(h.kB, h.vB, h.kA, h.vA, ctl, status, 1, grid_sort, s);
        launch_sort_pass(h.kA, h.vA, h.kB, h.vB, ctl, status, 2, grid_sort, s);
    }
    {
        ProfScope p("hull_chains", s);
        launch_chain(ctl, h.kB, h.vB, (const int*)(base + L.off_bu), (const int*)(base + L.off_bv),
                     (const int*)(base + L.off_bi), (const int*)(base + L.off_blen), (int*)(base + L.off_cu),
                     (int*)(base + L.off_cv), (int*)(base + L.off_ci), (int*)(base + L.off_clen),
                     (int*)(base + L.off_counters), (int)L.ctcap, (int*)h.vA, (int*)h.kA, (int*)h.kB, (int*)h.vB,
                     pts, n, out_idx, out_n, h.di.sms * h.di.occ_chain, s);
    }
}

static int enqueue_hull_direct(const float* pts, long long n, int32_t* out_idx, int64_t* out_n, cudaStream_t s,
                               int dev, char* base, const Layout& L, cudaStream_t owner) {
    HullLaunch h;
    const int st = hull_setup(pts, n, dev, owner, base, L, &h);
    if (st != CH_OK) return st;
    enqueue_filter_part(pts, n, out_idx, out_n, s, h, 0ull);
    enqueue_large_part(pts, n, out_idx, out_n, s, base, L, h);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ECUDA;
}

// Captures the sequence on `cs` with the large-survivor part as the body of
// a conditional (if) node whose condition the post pass raises; replays of
// small-survivor calls then launch only the filter part.  False when any step
// of the capture fails (the caller then captures the plain sequence).
static bool capture_conditional(const float* pts, long long n, int32_t* out_idx, int64_t* out_n, cudaStream_t cs,
                                int dev, char* base, const Layout& L, cudaStream_t owner, cudaGraph_t* out) {
    HullLaunch h;
    if (hull_setup(pts, n, dev, owner, base, L, &h) != CH_OK) return false;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    bool ok = true;
    cudaGraph_t graph = nullptr;
    cudaGraphConditionalHandle cond = 0;
    cudaStream_t bs = nullptr;
    {
        cudaStreamCaptureStatus stc;
        unsigned long long id = 0;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* edata = nullptr;
        size_t ndeps = 0;
        ok = cudaStreamGetCaptureInfo(cs, &stc, &id, &graph, &deps, &edata, &ndeps) == cudaSuccess && graph;
        if (ok) ok = cudaGraphConditionalHandleCreate(&cond, graph, 0u, cudaGraphCondAssignDefault) == cudaSuccess;
    }
    if (ok) {
        enqueue_filter_part(pts, n, out_idx, out_n, cs, h, (unsigned long long)cond);
        cudaStreamCaptureStatus stc;
        unsigned long long id = 0;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* edata = nullptr;
        size_t ndeps = 0;
        ok = cudaStreamGetCaptureInfo(cs, &stc, &id, &graph, &deps, &edata, &ndeps) == cudaSuccess;
        cudaGraphNode_t node = nullptr;
        cudaGraphNodeParams np = {};
        if (ok) {
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = cond;
            np.conditional.type = cudaGraphCondTypeIf;
            np.conditional.size = 1;
            ok = cudaGraphAddNode(&node, graph, deps, edata, ndeps, &np) == cudaSuccess;
        }
        if (ok) ok = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                     cudaSuccess;
        if (ok) ok = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) {
            cudaGraph_t body = np.conditional.phGraph_out[0];
            ok = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
            if (ok) {
                enqueue_large_part(pts, n, out_idx, out_n, bs, base, L, h);
                cudaGraph_t tmp = nullptr;
                ok = cudaStreamEndCapture(bs, &tmp) == cudaSuccess;
            }
        }
    }
    cudaGraph_t g = nullptr;
    const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
    if (bs) cudaStreamDestroy(bs);
    if (!ok || !ended || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    *out = g;
    return true;
}

// ---------------------------------------------------------------------------
// CUDA-graph cache.  A call repeated with the same (device, stream, points,
// n, outputs, workspace) replays one captured graph instead of ~10 separate
// launches.  The first call of a key runs directly; the second captures the
// sequence on a private stream and instantiates it; later ones replay it.
// Disabled while profiling (per-kernel events) and when the caller's stream
// is itself being captured (the launches then become part of that graph).
struct GraphKey {
    int dev;
    cudaStream_t s;
    const void* pts;
    long long n;
    const void* out_idx;
    const void* out_n;
    const void* ws;
    bool operator<(const GraphKey& o) const {
        if (dev != o.dev) return dev < o.dev;
        if (s != o.s) return s < o.s;
        if (pts != o.pts) return pts < o.pts;
        if (n != o.n) return n < o.n;
        if (out_idx != o.out_idx) return out_idx < o.out_idx;
        if (out_n != o.out_n) return out_n < o.out_n;
        return ws < o.ws;
    }
};
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int seen = 0;
    unsigned long long last_use = 0;
};
static std::mutex g_graph_mu;
static std::map<GraphKey, GraphEntry> g_graphs;
static unsigned long long g_graph_clock = 0;
static constexpr size_t kGraphCacheMax = 64;

static void drop_graphs_locked(int dev, cudaStream_t s) {
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        if (it->first.dev == dev && it->first.s == s) {
            if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

void drop_graphs(int dev, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    drop_graphs_locked(dev, s);
}

int enqueue_hull_nograph(const float* pts, long long n, int32_t* out_idx, int64_t* out_n, cudaStream_t s,
                         int dev) {
    char* base = nullptr;
    Layout L;
    const int st = get_workspace(dev, s, n, &base, &L);
    if (st != CH_OK) return st;
    return enqueue_hull_direct(pts, n, out_idx, out_n, s, dev, base, L, s);
}

int enqueue_hull(const float* pts, long long n, int32_t* out_idx, int64_t* out_n, cudaStream_t s, int dev) {
    DevInfo di;
    int st = device_info(dev, &di);
    if (st != CH_OK) return st;
    // The workspace must exist (and keep its address) before a graph names it.
    char* base = nullptr;
    Layout L;
    st = get_workspace(dev, s, n, &base, &L);
    if (st != CH_OK) return st;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (g_prof || cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return enqueue_hull_direct(pts, n, out_idx, out_n, s, dev, base, L, s);
    const GraphKey key{dev, s, pts, n, out_idx, out_n, base};
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        GraphEntry& e = g_graphs[key];
        e.last_use = ++g_graph_clock;
        if (e.exec) exec = e.exec;
        else if (e.seen++ == 0) return enqueue_hull_direct(pts, n, out_idx, out_n, s, dev, base, L, s);
    }
    if (exec) return cudaGraphLaunch(exec, s) == cudaSuccess ? CH_OK : CH_ECUDA;
    // Second call of this key: capture on a private stream, then replay.
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return enqueue_hull_direct(pts, n, out_idx, out_n, s, dev, base, L, s);
    }
    cudaGraph_t graph = nullptr;
    bool ok = capture_conditional(pts, n, out_idx, out_n, cs, dev, base, L, s, &graph);
    if (!ok) {   // plain capture of the whole sequence
        ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            st = enqueue_hull_direct(pts, n, out_idx, out_n, cs, dev, base, L, s);
            ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && st == CH_OK && graph;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (!ok) {
        cudaGetLastError();
        return enqueue_hull_direct(pts, n, out_idx, out_n, s, dev, base, L, s);
    }
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        if (g_graphs.size() > kGraphCacheMax) {   // evict the least recently used entry
            auto victim = g_graphs.begin();
            for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it)
                if (it->second.last_use < victim->second.last_use) victim = it;
            if (victim->second.exec) cudaGraphExecDestroy(victim->second.exec);
            g_graphs.erase(victim);
        }
        g_graphs[key].exec = exec;
    }
    return cudaGraphLaunch(exec, s) == cudaSuccess ? CH_OK : CH_ECUDA;
}

int check_points_args(const float* pts, long long n) {
    if (n < 0 || n > CH_MAX_POINTS) return CH_EINVAL;
    if (n > 0 && !pts) return CH_EINVAL;
    if (((uintptr_t)pts & 7u) != 0u) return CH_EINVAL;
    return CH_OK;
}

}  // namespace ch

using namespace ch;

extern "C" {

int ch_hull(const float* pts, int64_t n, int32_t* out_idx, int64_t* out_n, void* stream) {
    int st = check_points_args(pts, n);
    if (st != CH_OK) return st;
    if (!out_n || (n > 0 && !out_idx)) return CH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return cudaMemsetAsync(out_n, 0, sizeof(int64_t), s) == cudaSuccess ? CH_OK : CH_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    return enqueue_hull(pts, n, out_idx, out_n, s, dev);
}

int ch_filter(const float* pts, int64_t n, int32_t* out_ext8, uint8_t* out_labels, int64_t* out_counts4,
              void* stream) {
    int st = check_points_args(pts, n);
    if (st != CH_OK) return st;
    if (!out_ext8) return CH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        if (cudaMemsetAsync(out_ext8, 0xFF, 8 * sizeof(int32_t), s) != cudaSuccess) return CH_ECUDA;
        if (out_counts4 && cudaMemsetAsync(out_counts4, 0, 4 * sizeof(int64_t), s) != cudaSuccess)
            return CH_ECUDA;
        return CH_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    DevInfo di;
    if ((st = device_info(dev, &di)) != CH_OK) return st;
    char* base = nullptr;
    Layout L;
    if ((st = get_workspace(dev, s, n, &base, &L)) != CH_OK) return st;
    Ctl* ctl = (Ctl*)(base + L.off_ctl);
    const int head = (((uintptr_t)pts & 15u) != 0u) ? 1 : 0;
    const long long ntiles = (n - head) / kWarpTilePts;
    uint32_t* kA = (uint32_t*)(base + L.off_kA);
    uint64_t* vA = (uint64_t*)(base + L.off_vA);
    { ProfScope p("init", s); launch_init(ctl, 1, s); }
    {
        ProfScope p("main_filter", s);
        launch_main(pts, n, head, ntiles, ctl, nullptr, nullptr, 0xFFFFFFFFu, kA, vA, di.sms * di.occ_main, s);
    }
    if (out_labels || out_counts4) {
        ProfScope p("labels", s);
        launch_labels(pts, n, ctl, out_labels, di.sms * di.occ_lab, s);
    }
    launch_filter_output(ctl, n, out_ext8, out_counts4, s);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ECUDA;
}

int ch_hull_host(const float* pts, int64_t n, int32_t* out_idx, int64_t* out_n, void* stream) {
    int st = check_points_args(pts, n);
    if (st != CH_OK) return st;
    if (!out_n || (n > 0 && !out_idx)) return CH_EINVAL;
    if (n == 0) { *out_n = 0; return CH_OK; }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    const size_t pts_bytes = align_up(8 * (size_t)n), idx_bytes = align_up(4 * (size_t)n);
    char* stage = nullptr;
    if ((st = get_stage(dev, s, pts_bytes + idx_bytes + 256, &stage)) != CH_OK) return st;
    float* dpts = (float*)stage;
    int32_t* didx = (int32_t*)(stage + pts_bytes);
    int64_t* dn = (int64_t*)(stage + pts_bytes + idx_bytes);
    if (cudaMemcpyAsync(dpts, pts, 8 * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess) return CH_ECUDA;
    if ((st = enqueue_hull(dpts, n, didx, dn, s, dev)) != CH_OK) return st;
    int64_t h = 0;
    if (cudaMemcpyAsync(&h, dn, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CH_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CH_ECUDA;
    *out_n = h;
    if (h > 0) {
        if (cudaMemcpyAsync(out_idx, didx, 4 * (size_t)h, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return CH_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return CH_ECUDA;
    }
    return CH_OK;
}

int ch_reserve(int64_t n, int32_t k, void* stream) {
    if (n < 0 || k < 0) return CH_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    DevInfo di;
    int st = device_info(dev, &di);
    if (st != CH_OK) return st;
    char* base;
    Layout L;
    st = get_workspace(dev, (cudaStream_t)stream, std::max<int64_t>(n, 1), &base, &L);
    if (st != CH_OK) return st;
    return reserve_batched(dev, (cudaStream_t)stream, n, k);
}

size_t ch_workspace_bytes(int64_t n) { return n < 0 ? 0 : make_layout(n).total; }

int ch_hull_counters(void* stream, int64_t* out, int cap) {
    if (!out || cap < 0) return CH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_ws.find(std::make_pair(dev, s));
        if (it == g_ws.end() || !it->second.base) return CH_EINVAL;
        base = it->second.base;
    }
    Ctl c;
    if (cudaMemcpyAsync(&c, base, sizeof(Ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CH_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CH_ECUDA;
    const int64_t v[] = {
        (int64_t)c.count_raw,
        (int64_t)c.count,
        (int64_t)c.mode,
        (int64_t)(c.bk_state == 2 ? 2 : c.bk_state == 1 ? 1 : 0),
        (int64_t)c.status,
        (int64_t)(c.star_final ? c.star_k : 0),
    };
    const int nv = (int)(sizeof(v) / sizeof(v[0]));
    for (int i = 0; i < nv && i < cap; ++i) out[i] = v[i];
    return nv;
}

#if defined(CH_TRACE) || defined(CH_TIMELINE)
// Debug builds: the phase timeline of the most recent call on the first
// workspace (%globaltimer ns; 14 phases, first start and last end of each).
int ch_trace_timeline(unsigned long long* out28) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_ws.empty() || !g_ws.begin()->second.base) return CH_EINVAL;
    Ctl c;
    if (cudaMemcpy(&c, g_ws.begin()->second.base, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return CH_ECUDA;
    for (int i = 0; i < 14; ++i) {
        out28[2 * i] = c.tl[i][0];
        out28[2 * i + 1] = c.tl[i][1];
    }
    return CH_OK;
}
#endif

int ch_release(void) {
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        for (auto& kv : g_graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        g_graphs.clear();
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : g_ws) free_workspace(kv.second, kv.first.second);
    g_ws.clear();
    release_batched();
    return CH_OK;
}

const char* ch_strerror(int status) {
    switch (status) {
        case CH_OK: return "ok";
        case CH_PENDING: return "pending";
        case CH_EINVAL: return "invalid argument";
        case CH_ERANGE: return "coordinate outside the integer domain [0, 2^24)";
        case CH_ENOMEM: return "out of memory or over budget";
        case CH_ECUDA: return "CUDA error";
        case CH_ETIMEOUT: return "device wait timed out";
        case CH_EBUSY: return "busy, retry";
        default: return "unknown status";
    }
}

int ch_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof = on != 0;
    return CH_OK;
}

int ch_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    g_acc.clear();
    return CH_OK;
}

int ch_profile_read(const char** names, int64_t* launches, double* total_ms, int cap) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    g_names.clear();
    for (auto& kv : g_acc) g_names.push_back(kv.first);
    int i = 0;
    for (auto& kv : g_acc) {
        if (i < cap) {
            if (names) names[i] = g_names[i].c_str();
            if (launches) launches[i] = kv.second.first;
            if (total_ms) total_ms[i] = kv.second.second;
        }
        ++i;
    }
    return (int)g_acc.size();
}

}  // extern "C"
