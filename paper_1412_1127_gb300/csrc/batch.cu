// batch.cu -- many independent regions in one persistent launch.
//
// The paper charges every kernel call a launch cost (Methodology: cudaLaunch,
// cudaSetupArgument, cudaConfigureCall) and notes applications that pay it
// per loop (Hotspot, Pathfinder in Sec. 4.2).  Here a whole batch of
// reduction regions -- each with the semantics of accr_reduce -- runs in one
// launch:
//
//   * a region of at most `small_bytes` is folded whole by one warp
//     (lanes stream 16-byte vectors, shuffle merge, lane 0 writes);
//   * a longer region is cut into tiles of `tile_bytes`; CTAs of a persistent
//     grid fold tiles independently; a tile's partial goes to scratch and the
//     region's last tile to finish (a per-region counter) merges the region's
//     partials in tile order and writes its variables.
//
// The split is a function of each region's own element type and length, so a
// region's result has the same bits alone and inside any batch.  The host
// builds the plan (descriptors, tile -> region map, warp-region list) and
// uploads it in one copy; accr_batch_create additionally captures the launch
// in a CUDA graph that later launches replay.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "debug.cuh"
#include "fold.cuh"

namespace accr {

// Defined in reduce.cu (the single-region path, used by the unbatched form).
int reduce_grid(int in_type, int nc, int64_t n);
int reduce_launch(const void *in, int64_t n, int in_type, const ClauseDev *cl, int nc, int two_level,
                  Partial *partials, unsigned *counter, int grid, cudaStream_t s);

// Vectors in flight: picked by the autotuner (paper_1412_1127_gb300/autotune.py,
// "vectors" in tuning.json), which builds and times the candidates; the build
// passes the chosen widths in.
#ifndef ACCR_BATCH_BU
#define ACCR_BATCH_BU 4
#endif
#ifndef ACCR_BATCH_SU
#define ACCR_BATCH_SU 8
#endif
#ifndef ACCR_BATCH_MINB
#define ACCR_BATCH_MINB 4
#endif
constexpr int BB = 256;              // threads per CTA (4 CTAs per SM: one CTA's merge between tiles overlaps the others' streaming)
constexpr int BU = ACCR_BATCH_BU;    // 16-byte vectors per thread per iteration (tiles)
constexpr int SU = ACCR_BATCH_SU;    // 16-byte vectors per lane per iteration (warp regions)
constexpr int MINB = ACCR_BATCH_MINB;  // CTAs per SM the register budget is set for

// A region's descriptor carries at most two clauses: a region with three or
// four is planned as two descriptors over the same elements.
constexpr int RD_CLAUSES = 2;
struct RegionDev {
    const void *in;
    int64_t n;
    int64_t tile0;  // first tile of a tiled region; -1 for a warp region
    int32_t in_type;
    int32_t nc;     // 1 or 2
    ClauseDev cl[RD_CLAUSES];
};
static_assert(sizeof(RegionDev) == 112, "RegionDev layout");

struct BatchArgs {
    const RegionDev *regions;
    const int2 *tiles;           // [T] (region, tile index in region), in queue order
    const int32_t *small;        // [S] warp regions, in queue order
    int64_t T, S;
    int64_t R;                   // descriptors (bound of the region indices)
    int64_t slots;               // partial slots (tiles of all tiled descriptors)
    int64_t tile_bytes;
    Partial *partials;           // [sum of tiles][RD_CLAUSES], slot tile0 + k
    unsigned *counters;          // [R] tiles done per region; zero on entry and exit
    unsigned *queue;             // [3] next tile, next warp region, CTAs done
};

__device__ __forceinline__ uint4 ld_batch(const uint4 *p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

__device__ __forceinline__ Partial ld_partial_cg(const Partial *p) {
    uint4 v = __ldcg(reinterpret_cast<const uint4 *>(p));
    Partial q;
    q.a = ((uint64_t)v.y << 32) | v.x;
    q.c = __uint_as_float(v.z);
    q.pad = 0;
    return q;
}

// One tile of a tiled region, folded by the whole CTA.
template <typename T, int NC>
__device__ __noinline__ void tile_fold(const BatchArgs &p, const RegionDev *d, int r, int64_t k,
                                          Acc (*sh)[BB / 32], int *s_last) {
    constexpr bool E64 = sizeof(T) == 8;
    constexpr int EPV = 16 / (int)sizeof(T);
    const int64_t TE = p.tile_bytes / (int64_t)sizeof(T);
    const int64_t n = d->n;
    const int64_t tile0 = d->tile0;
    const int64_t t = tile0 + k;  // this tile's partial slot
    const int64_t lo = k * TE;
    const int64_t len = (n - lo) < TE ? (n - lo) : TE;
    const int64_t ntiles = (n + TE - 1) / TE;
    const T *in = (const T *)d->in + lo;
    if (!ACCR_DCHECK(k >= 0 && k < ntiles, DS_BATCH_TILE)) return;  // the same for the whole CTA

    int w[NC];
    uint64_t id[NC];
    Acc A[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        w[c] = d->cl[c].wcode;
        id[c] = d->cl[c].ident;
        A[c].a = id[c];
        A[c].c = 0.f;
    }
    const int64_t mis = (int64_t)(((16 - ((uintptr_t)in & 15)) & 15) / sizeof(T));
    const int64_t head = mis < len ? mis : len;
    const uint4 *vin = (const uint4 *)(in + head);
    const int64_t nvec = (len - head) / EPV;
    const int64_t tail0 = head + nvec * EPV;
    if (threadIdx.x < head) {
        T x = in[threadIdx.x];
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_one<T>(w[c], A[c], x);
    }
    if (tail0 + threadIdx.x < len) {
        T x = in[tail0 + threadIdx.x];
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_one<T>(w[c], A[c], x);
    }
    int64_t v = threadIdx.x;
    for (; v + (BU - 1) * BB < nvec; v += BB * BU) {
        uint4 b[BU];
#pragma unroll
        for (int u = 0; u < BU; ++u) b[u] = ld_batch(vin + v + u * BB);
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_vec<T, BU>(w[c], A[c], b);
    }
#pragma unroll
    for (int u = 0; u < BU; ++u) {
        const int64_t vv = v + u * BB;
        if (vv < nvec) {
            uint4 b = ld_batch(vin + vv);
#pragma unroll
            for (int c = 0; c < NC; ++c) fold_vec<T, 1>(w[c], A[c], &b);
        }
    }
    cta_merge<NC, BB>(w, id, E64, A, sh);

    if (ntiles == 1) {
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
                store_var(d->cl[c], 0, finish(d->cl[c], E64, n == 0, to_final(w[c], A[c])));
        }
        return;
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            Partial q;
            q.a = A[c].a;
            q.c = A[c].c;
            q.pad = 0;
            if (ACCR_DCHECK(t >= 0 && t < p.slots, DS_BATCH_SLOT)) p.partials[t * RD_CLAUSES + c] = q;
        }
        __threadfence();
        const unsigned old = atomicAdd(&p.counters[r], 1u);
        *s_last = (old == (unsigned)(ntiles - 1));
    }
    __syncthreads();
    const int last = *s_last;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const bool slots_ok = ACCR_DCHECK(tile0 >= 0 && tile0 + ntiles <= p.slots, DS_BATCH_SLOT);
    int fw[NC];
    uint64_t fid[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        fw[c] = final_code(w[c]);
        fid[c] = final_ident(d->cl[c]);
        A[c].a = fid[c];
        A[c].c = 0.f;
        for (int64_t j = threadIdx.x; slots_ok && j < ntiles; j += BB) {
            Partial q = ld_partial_cg(&p.partials[(tile0 + j) * RD_CLAUSES + c]);
            Acc Q;
            Q.a = q.a;
            Q.c = q.c;
            merge(fw[c], E64, A[c], to_final(w[c], Q));
        }
    }
    cta_merge<NC, BB>(fw, fid, E64, A, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) store_var(d->cl[c], 0, finish(d->cl[c], E64, false, A[c]));
        p.counters[r] = 0u;
    }
}

// A whole short region folded by one warp.
template <typename T, int NC>
__device__ __noinline__ void warp_fold(const RegionDev *d, int lane) {
    constexpr bool E64 = sizeof(T) == 8;
    constexpr int EPV = 16 / (int)sizeof(T);
    const int64_t n = d->n;
    const T *in = (const T *)d->in;
    int w[NC];
    Acc A[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        w[c] = d->cl[c].wcode;
        A[c].a = d->cl[c].ident;
        A[c].c = 0.f;
    }
    const int64_t mis = (int64_t)(((16 - ((uintptr_t)in & 15)) & 15) / sizeof(T));
    const int64_t head = mis < n ? mis : n;
    const uint4 *vin = (const uint4 *)(in + head);
    const int64_t nvec = (n - head) / EPV;
    const int64_t tail0 = head + nvec * EPV;
    if (lane < head) {
        T x = in[lane];
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_one<T>(w[c], A[c], x);
    }
    if (tail0 + lane < n) {
        T x = in[tail0 + lane];
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_one<T>(w[c], A[c], x);
    }
    int64_t v = lane;
    for (; v + (SU - 1) * 32 < nvec; v += 32 * SU) {
        uint4 b[SU];
#pragma unroll
        for (int u = 0; u < SU; ++u) b[u] = ld_batch(vin + v + u * 32);
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_vec<T, SU>(w[c], A[c], b);
    }
#pragma unroll
    for (int u = 0; u < SU; ++u) {
        const int64_t vv = v + u * 32;
        if (vv < nvec) {
            uint4 b = ld_batch(vin + vv);
#pragma unroll
            for (int c = 0; c < NC; ++c) fold_vec<T, 1>(w[c], A[c], &b);
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        warp_merge(w[c], E64, A[c]);
        if (lane == 0) store_var(d->cl[c], 0, finish(d->cl[c], E64, n == 0, to_final(w[c], A[c])));
    }
}

// Regions in a batch carry one or two clauses; a region with three or four
// is split on the host into two descriptors over the same elements.
#define ACCR_DISPATCH_TYPE_NC(type, nc, FN, ...)                          \
    switch ((type) * 2 + (nc) - 1) {                                      \
    case 0: FN<int32_t, 1>(__VA_ARGS__); break;                           \
    case 1: FN<int32_t, 2>(__VA_ARGS__); break;                           \
    case 2: FN<int64_t, 1>(__VA_ARGS__); break;                           \
    case 3: FN<int64_t, 2>(__VA_ARGS__); break;                           \
    case 4: FN<float, 1>(__VA_ARGS__); break;                             \
    case 5: FN<float, 2>(__VA_ARGS__); break;                             \
    case 6: FN<double, 1>(__VA_ARGS__); break;                            \
    default: FN<double, 2>(__VA_ARGS__); break;                           \
    }

__device__ __forceinline__ void batch_body(const BatchArgs &p, const RegionDev *regions, const int2 *tiles,
                                           const int32_t *small) {
    __shared__ Acc sh[RD_CLAUSES][BB / 32];
    __shared__ int s_last;
    __shared__ long long s_q;
    // tiles of long regions, one CTA per tile, taken from a queue (largest
    // first within each element-type group); the next index is fetched while
    // the current tile is folded
    if (threadIdx.x == 0) s_q = (long long)atomicAdd(&p.queue[0], 1u);
    __syncthreads();
    long long q = s_q;
    __syncthreads();
    while (q < p.T) {
        if (threadIdx.x == 0) s_q = (long long)atomicAdd(&p.queue[0], 1u);
        const int2 tk = tiles[q];
        if (ACCR_DCHECK(tk.x >= 0 && tk.x < p.R, DS_BATCH_REGION)) {  // the same for the whole CTA
            const RegionDev *d = regions + tk.x;
            const int type = d->in_type, nc = d->nc;
            ACCR_DISPATCH_TYPE_NC(type, nc, tile_fold, p, d, tk.x, (int64_t)tk.y, sh, &s_last);
        }
        __syncthreads();
        q = s_q;
        __syncthreads();
    }
    // short regions, one warp per region, from a second queue
    const int lane = threadIdx.x & 31;
    long long s = 0;
    if (lane == 0) s = (long long)atomicAdd(&p.queue[1], 1u);
    s = __shfl_sync(0xffffffffu, s, 0);
    while (s < p.S) {
        long long nx = 0;
        if (lane == 0) nx = (long long)atomicAdd(&p.queue[1], 1u);
        const int32_t ri = small[s];
        if (ACCR_DCHECK(ri >= 0 && ri < p.R, DS_BATCH_REGION)) {
            const RegionDev *d = regions + ri;
            const int type = d->in_type, nc = d->nc;
            ACCR_DISPATCH_TYPE_NC(type, nc, warp_fold, d, lane);
        }
        s = __shfl_sync(0xffffffffu, nx, 0);
    }
    // the last CTA to finish returns the queues to zero for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&p.queue[2], 1u) == gridDim.x - 1) {
            p.queue[0] = 0u;
            p.queue[1] = 0u;
            p.queue[2] = 0u;
        }
    }
}

__global__ void __launch_bounds__(BB, MINB) batch_kernel(const __grid_constant__ BatchArgs p) {
    batch_body(p, p.regions, p.tiles, p.small);
}

// A small plan (a batch of a few regions, as the served loop forms) travels
// in the kernel's parameters instead of through a host-to-device copy ahead
// of the launch; the descriptors are read from the parameter space.
constexpr int INL_REGIONS = 16, INL_TILES = 1024, INL_SMALL = 16;
struct BatchArgsInline {
    BatchArgs b;  // its plan pointers are unused
    RegionDev regions[INL_REGIONS];
    int2 tiles[INL_TILES];
    int32_t small[INL_SMALL];
};
static_assert(sizeof(BatchArgsInline) < 32000, "kernel parameters are limited to 32764 bytes");

__global__ void __launch_bounds__(BB, MINB) batch_kernel_inline(const __grid_constant__ BatchArgsInline p) {
    batch_body(p.b, p.regions, p.tiles, p.small);
}

// ---- host: plans -------------------------------------------------------------------

static std::atomic<int64_t> g_small_bytes{ACCR_SMALL_BYTES};
static std::atomic<int64_t> g_tile_bytes{ACCR_TILE_BYTES};

struct HostPlan {
    std::vector<RegionDev> regions;
    std::vector<int2> tiles;      // queue order
    std::vector<int32_t> small;   // queue order
    int64_t ntiles = 0;           // partial slots
    int64_t tile_bytes = ACCR_TILE_BYTES;
    int64_t tile_override = 0;    // > 0: this plan's tile size instead of the process-wide one
    // layout of the device copy
    size_t off_tiles = 0, off_small = 0, off_partials = 0, plan_bytes = 0, total_bytes = 0;
};

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The calling thread's plan for one-shot batches: its vectors keep their
// capacity from call to call, so planning a batch of the same size again
// allocates nothing and touches no new pages.
static HostPlan &thread_plan(int64_t tile_override) {
    static thread_local HostPlan P;
    P.tile_override = tile_override;
    return P;
}

static int log2_floor(uint64_t v) { return v ? 63 - __builtin_clzll(v) : 0; }

// ---- host: planner threads ----------------------------------------------------------
//
// Planning a batch of many regions (lowering each region's clauses, sorting
// the work queues, writing the plan into pinned staging) takes a few hundred
// microseconds on one host core for 20,000 regions, longer than the batch's
// kernel.  Large plans are therefore cut into contiguous ranges of regions that
// a small pool of host threads plans in parallel; the result is the same plan,
// entry for entry, as the serial one.
class PlanPool {
public:
    explicit PlanPool(int workers) {
        for (int i = 0; i < workers; ++i) th_.emplace_back([this] { loop(); });
    }
    ~PlanPool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (std::thread &t : th_) t.join();
    }
    int threads() const { return (int)th_.size() + 1; }
    // Runs f(0) .. f(n - 1) on the pool's threads and the caller's; returns
    // when all have finished.  One job at a time.
    void run(int n, const std::function<void(int)> &f) {
        std::lock_guard<std::mutex> one(run_mu_);
        Job j;
        j.fn = &f;
        j.n = n;
        {
            std::lock_guard<std::mutex> lk(mu_);
            cur_ = &j;
            ++gen_;
        }
        cv_.notify_all();
        const int mine = work(j);
        std::unique_lock<std::mutex> lk(mu_);
        cur_ = nullptr;  // no thread attaches to this job any more
        j.done += mine;
        done_cv_.wait(lk, [&] { return j.done == j.n && j.active == 0; });
    }

private:
    struct Job {
        const std::function<void(int)> *fn = nullptr;
        int n = 0;
        std::atomic<int> next{0};
        int done = 0;    // items finished (under mu_)
        int active = 0;  // pool threads attached (under mu_)
    };
    static int work(Job &j) {
        int mine = 0;
        for (int i = j.next.fetch_add(1); i < j.n; i = j.next.fetch_add(1)) {
            (*j.fn)(i);
            ++mine;
        }
        return mine;
    }
    void loop() {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
            if (stop_) return;
            seen = gen_;
            Job *j = cur_;
            if (!j) continue;
            ++j->active;
            lk.unlock();
            const int mine = work(*j);
            lk.lock();
            j->done += mine;
            --j->active;
            done_cv_.notify_all();
        }
    }
    std::vector<std::thread> th_;
    std::mutex run_mu_, mu_;
    std::condition_variable cv_, done_cv_;
    Job *cur_ = nullptr;
    uint64_t gen_ = 0;
    bool stop_ = false;
};

constexpr int64_t PAR_MIN_REGIONS = 4096;  // smaller plans stay on the calling thread
constexpr int PLAN_THREADS = 4;            // pool threads besides the caller

static PlanPool &plan_pool() {
    static PlanPool *pool = new PlanPool(PLAN_THREADS);  // lives until exit
    return *pool;
}

// Runs f over `chunks` chunks: in the pool if the plan is large, else here.
static void plan_for(int64_t R, int chunks, const std::function<void(int)> &f) {
    if (chunks <= 1 || R < PAR_MIN_REGIONS) {
        for (int c = 0; c < chunks; ++c) f(c);
        return;
    }
    plan_pool().run(chunks, f);
}

static int check_region_ptr(const void *in, int64_t n, int t, int64_t r) {
    if (n < 0) return set_error(ACCR_EINVAL, "region %lld: n < 0", (long long)r);
    if (n > 0 && !in) return set_error(ACCR_EINVAL, "region %lld: in is NULL", (long long)r);
    if (((uintptr_t)in & (uintptr_t)(type_bytes(t) - 1)) != 0)
        return set_error(ACCR_EINVAL, "region %lld: in is not aligned to its element size", (long long)r);
    return ACCR_OK;
}

// Lowered clauses of recent region kinds, reused when a region has the same
// element type, flags, operators, variable types and prior values as one of
// them (only the outputs then differ): batches are usually many regions of a
// few kinds, and lowering dominated the host cost of a plan.
struct ClauseMemo {
    struct Entry {
        bool valid = false;
        int in_type = 0, nc = 0;
        unsigned flags = 0;
        int op[ACCR_MAX_CLAUSES], acc[ACCR_MAX_CLAUSES];
        const void *init[ACCR_MAX_CLAUSES];
        ClauseDev dev[ACCR_MAX_CLAUSES];
        bool same(const accr_region &g) const {
            if (!valid || g.in_type != in_type || g.nclauses != nc || g.flags != flags) return false;
            for (int c = 0; c < nc; ++c)
                if (g.clauses[c].op != op[c] || g.clauses[c].acc_type != acc[c] || g.clauses[c].init != init[c])
                    return false;
            return true;
        }
    };
    Entry e[4];
    int next = 0;
};

static int lower_region(const accr_region &g, int64_t r, ClauseMemo &m, ClauseDev *cl) {
    for (const ClauseMemo::Entry &x : m.e) {
        if (!x.same(g)) continue;
        for (int c = 0; c < x.nc; ++c) {
            if (!g.clauses[c].out) return set_error(ACCR_EINVAL, "region %lld: clause %d: out is NULL", (long long)r, c);
            cl[c] = x.dev[c];
            cl[c].out = g.clauses[c].out;
        }
        return ACCR_OK;
    }
    int rc = lower_clauses(g.in_type, g.clauses, g.nclauses, g.flags, cl);
    if (rc != ACCR_OK) return rc;
    ClauseMemo::Entry &x = m.e[m.next];
    m.next = (m.next + 1) & 3;
    x.valid = true;
    x.in_type = g.in_type;
    x.nc = g.nclauses;
    x.flags = g.flags;
    for (int c = 0; c < x.nc; ++c) {
        x.op[c] = g.clauses[c].op;
        x.acc[c] = g.clauses[c].acc_type;
        x.init[c] = g.clauses[c].init;
        x.dev[c] = cl[c];
    }
    return ACCR_OK;
}

// ---- host: plans -------------------------------------------------------------------

constexpr int NKEY = 8 * 64;

// Queue key: grouped by (element type, clause count) so that neighbouring work
// runs the same code, largest first within a group so that the small pieces
// fill in at the end.
static int key_of(int in_type, int nc, int64_t bytes) {
    return (in_type * 2 + (nc - 1)) * 64 + (63 - log2_floor((uint64_t)(bytes > 0 ? bytes : 1)));
}

// One contiguous range of source items (regions or segments) of a plan.
struct PlanChunk {
    int64_t s0 = 0, s1 = 0;  // source items
    int64_t d0 = 0, nd = 0;  // its descriptors
    int64_t slots = 0;       // partial slots (tiles) of its tiled descriptors
    std::vector<int64_t> tpos, spos;  // per key: counts, then queue positions
    int rc = ACCR_OK;
    std::string msg;
};

// The caller's region descriptors.
struct RegionSource {
    const accr_region *regs;
    int ndesc(int64_t i) const { return regs[i].nclauses > RD_CLAUSES ? 2 : 1; }
    // Lowers item i into out[0..ndesc); returns ACCR_OK or an error code.
    int fill(int64_t i, RegionDev *out, ClauseMemo &m) const {
        const accr_region &g = regs[i];
        if (g.flags & ~ACCR_COMPENSATED) return set_error(ACCR_EINVAL, "region %lld: bad flags", (long long)i);
        ClauseDev cl[ACCR_MAX_CLAUSES];
        int rc = lower_region(g, i, m, cl);
        if (rc != ACCR_OK) return rc;
        rc = check_region_ptr(g.in, g.n, g.in_type, i);
        if (rc != ACCR_OK) return rc;
        put(out, g.in, g.n, g.in_type, cl, g.nclauses);
        return ACCR_OK;
    }
    // Descriptors over the same elements: clauses 0-1, then 2-3.
    static void put(RegionDev *out, const void *in, int64_t n, int in_type, const ClauseDev *cl, int nc) {
        for (int c0 = 0, j = 0; c0 < nc; c0 += RD_CLAUSES, ++j) {
            RegionDev &d = out[j];
            d.in = in;
            d.n = n;
            d.tile0 = 0;
            d.in_type = in_type;
            d.nc = (nc - c0) < RD_CLAUSES ? (nc - c0) : RD_CLAUSES;
            d.cl[0] = cl[c0];
            if (d.nc > 1) d.cl[1] = cl[c0 + 1];
            else memset(&d.cl[1], 0, sizeof d.cl[1]);
        }
    }
};

// Segments [off[s], off[s+1]) of one array, one variable per segment.
struct SegmentSource {
    const void *values;
    const int64_t *off;
    int in_type, nc;
    int64_t eb;
    const ClauseDev *base;  // lowered clauses; out = the arrays' starts
    int ndesc(int64_t) const { return nc > RD_CLAUSES ? 2 : 1; }
    int fill(int64_t s, RegionDev *out, ClauseMemo &) const {
        const int64_t lo = off[s], hi = off[s + 1];
        if (lo < 0 || hi < lo)
            return set_error(ACCR_EINVAL, "segmented: offsets not non-decreasing at %lld", (long long)s);
        const void *in = (const char *)values + lo * eb;
        int rc = check_region_ptr(in, hi - lo, in_type, s);
        if (rc != ACCR_OK) return rc;
        if (hi > lo && !values) return set_error(ACCR_EINVAL, "segmented: values is NULL");
        ClauseDev cl[ACCR_MAX_CLAUSES];
        for (int c = 0; c < nc; ++c) {
            cl[c] = base[c];
            cl[c].out = (char *)base[c].out + s * type_bytes(base[c].acc_type);
        }
        RegionSource::put(out, in, hi - lo, in_type, cl, nc);
        return ACCR_OK;
    }
};

// Builds the plan of n source items: each descriptor goes to the warp list
// or to tiles by its own type and length, and both queues are ordered by key
// (a counting sort).  Large plans run in chunks on the planner threads; the
// queues come out in the same order as a serial pass would give (by key, then
// descriptor, then tile).
template <typename Src>
static int plan_chunked(const Src &src, int64_t n, HostPlan &P) {
    const int64_t small_b = g_small_bytes.load(), tile_b = P.tile_override > 0 ? P.tile_override : g_tile_bytes.load();
    P.tile_bytes = tile_b;
    const int nch = n >= PAR_MIN_REGIONS ? 2 * plan_pool().threads() : 1;
    std::vector<PlanChunk> ch((size_t)nch);
    for (int c = 0; c < nch; ++c) {
        ch[c].s0 = n * c / nch;
        ch[c].s1 = n * (c + 1) / nch;
    }
    // descriptors per chunk (a region with three or four clauses has two)
    plan_for(n, nch, [&](int c) {
        int64_t nd = 0;
        for (int64_t i = ch[c].s0; i < ch[c].s1; ++i) nd += src.ndesc(i);
        ch[c].nd = nd;
    });
    int64_t D = 0;
    for (PlanChunk &k : ch) {
        k.d0 = D;
        D += k.nd;
    }
    if (D > INT32_MAX / 2) return set_error(ACCR_EINVAL, "batch: too many regions");
    P.regions.resize((size_t)D);
    // lower every item into its descriptors; count queue entries per key
    plan_for(n, nch, [&](int c) {
        PlanChunk &k = ch[c];
        k.tpos.assign(NKEY, 0);
        k.spos.assign(NKEY, 0);
        k.slots = 0;
        ClauseMemo memo;
        int64_t d = k.d0;
        for (int64_t i = k.s0; i < k.s1; ++i) {
            const int nd = src.ndesc(i);
            const int rc = src.fill(i, &P.regions[(size_t)d], memo);
            if (rc != ACCR_OK) {
                k.rc = rc;
                k.msg = accr_last_error();
                return;
            }
            for (int j = 0; j < nd; ++j, ++d) {
                RegionDev &x = P.regions[(size_t)d];
                const int64_t eb = type_bytes(x.in_type);
                if (x.n * eb <= small_b) {
                    x.tile0 = -1;
                    k.spos[key_of(x.in_type, x.nc, x.n * eb)]++;
                } else {
                    const int64_t te = tile_b / eb, nt = (x.n + te - 1) / te;
                    x.tile0 = k.slots;  // chunk-relative until the bases are known
                    k.slots += nt;
                    k.tpos[key_of(x.in_type, x.nc, tile_b)] += nt - 1;
                    k.tpos[key_of(x.in_type, x.nc, (x.n - (nt - 1) * te) * eb)]++;
                }
            }
        }
    });
    for (PlanChunk &k : ch)
        if (k.rc != ACCR_OK) return set_error(k.rc, "%s", k.msg.c_str());
    // tile bases per chunk; queue positions per (key, chunk)
    std::vector<int64_t> base((size_t)nch);
    int64_t slots = 0;
    for (int c = 0; c < nch; ++c) {
        base[c] = slots;
        slots += ch[c].slots;
    }
    if (slots > INT32_MAX) return set_error(ACCR_EINVAL, "batch: more than 2^31 tiles");
    int64_t tp = 0, sp = 0;
    for (int key = 0; key < NKEY; ++key) {
        for (PlanChunk &k : ch) {
            const int64_t t = k.tpos[key], u = k.spos[key];
            k.tpos[key] = tp;
            k.spos[key] = sp;
            tp += t;
            sp += u;
        }
    }
    P.ntiles = slots;
    P.tiles.resize((size_t)tp);
    P.small.resize((size_t)sp);
    plan_for(n, nch, [&](int c) {
        PlanChunk &k = ch[c];
        for (int64_t d = k.d0; d < k.d0 + k.nd; ++d) {
            RegionDev &x = P.regions[(size_t)d];
            const int64_t eb = type_bytes(x.in_type);
            if (x.tile0 < 0) {
                P.small[(size_t)k.spos[key_of(x.in_type, x.nc, x.n * eb)]++] = (int32_t)d;
                continue;
            }
            x.tile0 += base[c];
            const int64_t te = tile_b / eb, nt = (x.n + te - 1) / te;
            const int kfull = key_of(x.in_type, x.nc, tile_b);
            const int klast = key_of(x.in_type, x.nc, (x.n - (nt - 1) * te) * eb);
            for (int64_t t = 0; t < nt; ++t)
                P.tiles[(size_t)k.tpos[t + 1 < nt ? kfull : klast]++] = make_int2((int)d, (int)t);
        }
    });
    P.off_tiles = align_up(sizeof(RegionDev) * P.regions.size(), 256);
    P.off_small = align_up(P.off_tiles + sizeof(int2) * P.tiles.size(), 256);
    P.plan_bytes = P.off_small + 4 * P.small.size();
    P.off_partials = align_up(P.plan_bytes, 256);
    P.total_bytes = P.off_partials + sizeof(Partial) * RD_CLAUSES * (size_t)P.ntiles + 256;
    return ACCR_OK;
}

// Copies the plan (descriptors, tile queue, warp queue) into dst, in pieces
// on the planner threads when it is large.
static void write_plan(const HostPlan &P, char *dst) {
    struct Piece {
        char *to;
        const char *from;
        size_t bytes;
    };
    const Piece parts[3] = {{dst, (const char *)P.regions.data(), sizeof(RegionDev) * P.regions.size()},
                            {dst + P.off_tiles, (const char *)P.tiles.data(), sizeof(int2) * P.tiles.size()},
                            {dst + P.off_small, (const char *)P.small.data(), 4 * P.small.size()}};
    const int64_t R = (int64_t)P.regions.size();
    const int pieces = R >= PAR_MIN_REGIONS ? 2 * plan_pool().threads() : 1;
    plan_for(R, pieces, [&](int c) {
        for (const Piece &q : parts) {
            const size_t lo = q.bytes * (size_t)c / (size_t)pieces, hi = q.bytes * (size_t)(c + 1) / (size_t)pieces;
            if (hi > lo) memcpy(q.to + lo, q.from + lo, hi - lo);
        }
    });
}

static int plan_from_regions(const accr_region *regs, int64_t R, HostPlan &P) {
    if (R < 0 || (R > 0 && !regs)) return set_error(ACCR_EINVAL, "batch: bad region array");
    if (R > INT32_MAX / 2) return set_error(ACCR_EINVAL, "batch: too many regions");
    RegionSource src{regs};
    return plan_chunked(src, R, P);
}

static int plan_from_segments(const void *values, const int64_t *off, int64_t nseg, int in_type,
                              const accr_clause *clauses, int nc, unsigned flags, HostPlan &P) {
    if (nseg < 0 || (nseg > 0 && !off)) return set_error(ACCR_EINVAL, "segmented: bad offsets");
    if (nseg > INT32_MAX / 2) return set_error(ACCR_EINVAL, "segmented: too many segments");
    ClauseDev base[ACCR_MAX_CLAUSES];
    int rc = lower_clauses(in_type, clauses, nc, flags & ACCR_COMPENSATED, base);
    if (rc != ACCR_OK) return rc;
    SegmentSource src{values, off, in_type, nc, (int64_t)type_bytes(in_type), base};
    return plan_chunked(src, nseg, P);
}

static int batch_grid(const HostPlan &P) {
    static std::mutex mu;
    static int cached[64] = {0};
    const DeviceInfo &dinfo = device_info();
    int maxg;
    {
        std::lock_guard<std::mutex> lk(mu);
        int &slot = cached[dinfo.id & 63];
        if (!slot) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, BB, 0);
            slot = (per_sm < 1 ? 1 : per_sm) * dinfo.sms;
        }
        maxg = slot;
    }
    const int64_t T = (int64_t)P.tiles.size(), S = (int64_t)P.small.size();
    int64_t want = std::max<int64_t>(T, (S + BB / 32 - 1) / (BB / 32));
    if (want < 1) want = 1;
    return (int)std::min<int64_t>(want, maxg);
}

static BatchArgs args_for(const HostPlan &P, char *dev, unsigned *counters) {
    BatchArgs a;
    a.regions = (const RegionDev *)dev;
    a.tiles = (const int2 *)(dev + P.off_tiles);
    a.small = (const int32_t *)(dev + P.off_small);
    a.T = (int64_t)P.tiles.size();
    a.S = (int64_t)P.small.size();
    a.R = (int64_t)P.regions.size();
    a.slots = P.ntiles;
    a.tile_bytes = P.tile_bytes;
    a.partials = (Partial *)(dev + P.off_partials);
    a.queue = counters;         // 4 words: the queues
    a.counters = counters + 4;  // then one per region
    return a;
}

// ---- host: per-stream buffers of the one-shot path ----------------------------------

struct StreamBufs {
    char *dev = nullptr;
    size_t dev_bytes = 0;
    unsigned *counters = nullptr;
    size_t ncounters = 0;
    char *stage[2] = {nullptr, nullptr};
    size_t stage_bytes[2] = {0, 0};
    cudaEvent_t stage_done[2] = {nullptr, nullptr};
    int next = 0;
    std::mutex mu;  // one planner per stream at a time
};
static std::mutex g_bufs_mu;
static std::map<std::pair<int, uintptr_t>, StreamBufs *> g_bufs;

static StreamBufs *bufs_for(accr_stream_t stream) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_bufs_mu);
    auto key = std::make_pair(dev, (uintptr_t)stream);
    auto it = g_bufs.find(key);
    if (it != g_bufs.end()) return it->second;
    StreamBufs *b = new StreamBufs();
    g_bufs.emplace(key, b);
    return b;
}

static int run_once(HostPlan &P, unsigned flags, accr_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const size_t R = P.regions.size();
    if (R == 0) return ACCR_OK;
    log_msg(2, "batch: %zu descriptors, %zu tiles of %lld bytes, %zu warp regions", R, P.tiles.size(),
            (long long)P.tile_bytes, P.small.size());
    StreamBufs *B = bufs_for(stream);
    std::lock_guard<std::mutex> lk(B->mu);
    // device plan + partials
    if ((B->dev_bytes < P.total_bytes || B->ncounters < R + 4) && fault_take(ACCR_FAULT_ALLOC))
        return set_error(ACCR_ENOMEM, "batch: injected allocation failure");
    if (B->dev_bytes < P.total_bytes || B->ncounters < R + 4) {
        int rc = cuda_check(cudaStreamSynchronize(s), "batch: grow sync");
        if (rc != ACCR_OK) return rc;
        if (B->dev_bytes < P.total_bytes) {
            if (B->dev) cudaFree(B->dev);
            B->dev = nullptr;
            B->dev_bytes = 0;
            size_t want = std::max(P.total_bytes, (size_t)1 << 20);
            if (cudaMalloc(&B->dev, want) != cudaSuccess) {
                cudaGetLastError();
                return set_error(ACCR_ENOMEM, "batch: cudaMalloc of %zu bytes failed", want);
            }
            B->dev_bytes = want;
        }
        if (B->ncounters < R + 4) {
            if (B->counters) cudaFree(B->counters);
            B->counters = nullptr;
            B->ncounters = 0;
            size_t want = std::max(R + 4, (size_t)65536);
            if (cudaMalloc(&B->counters, want * 4) != cudaSuccess) {
                cudaGetLastError();
                return set_error(ACCR_ENOMEM, "batch: cudaMalloc of counters failed");
            }
            rc = cuda_check(cudaMemset(B->counters, 0, want * 4), "batch: clear counters");
            if (rc != ACCR_OK) return rc;
            B->ncounters = want;
        }
    }
    if (R <= (size_t)INL_REGIONS && P.tiles.size() <= (size_t)INL_TILES && P.small.size() <= (size_t)INL_SMALL) {
        static BatchArgsInline ai;  // built under B->mu; launched by value
        static std::mutex inl_mu;
        std::lock_guard<std::mutex> il(inl_mu);
        ai.b = args_for(P, B->dev, B->counters);
        ai.b.regions = nullptr;
        ai.b.tiles = nullptr;
        ai.b.small = nullptr;
        ai.b.partials = (Partial *)B->dev;  // the partial slots start the device buffer
        std::copy(P.regions.begin(), P.regions.end(), ai.regions);
        std::copy(P.tiles.begin(), P.tiles.end(), ai.tiles);
        std::copy(P.small.begin(), P.small.end(), ai.small);
        int rc = launch_guard("batch_kernel");
        if (rc != ACCR_OK) return rc;
        batch_kernel_inline<<<batch_grid(P), BB, 0, s>>>(ai);
        rc = launched("batch_kernel");
        if (rc != ACCR_OK) return rc;
        if (flags & ACCR_SYNC) return cuda_check(cudaStreamSynchronize(s), "batch: sync");
        return ACCR_OK;
    }
    // pinned staging (double-buffered; wait until the copy that last used it is done)
    const int i = B->next;
    B->next ^= 1;
    if (!B->stage_done[i]) {
        int rc = cuda_check(cudaEventCreateWithFlags(&B->stage_done[i], cudaEventDisableTiming), "batch: event");
        if (rc != ACCR_OK) return rc;
    } else {
        int rc = cuda_check(cudaEventSynchronize(B->stage_done[i]), "batch: staging wait");
        if (rc != ACCR_OK) return rc;
    }
    if (B->stage_bytes[i] < P.plan_bytes) {
        if (B->stage[i]) cudaFreeHost(B->stage[i]);
        B->stage[i] = nullptr;
        B->stage_bytes[i] = 0;
        size_t want = std::max(P.plan_bytes, (size_t)1 << 20);
        if (cudaMallocHost(&B->stage[i], want) != cudaSuccess) {
            cudaGetLastError();
            return set_error(ACCR_ENOMEM, "batch: cudaMallocHost of %zu bytes failed", want);
        }
        B->stage_bytes[i] = want;
    }
    write_plan(P, B->stage[i]);
    int rc = cuda_check(cudaMemcpyAsync(B->dev, B->stage[i], P.plan_bytes, cudaMemcpyHostToDevice, s),
                        "batch: plan upload");
    if (rc != ACCR_OK) return rc;
    rc = cuda_check(cudaEventRecord(B->stage_done[i], s), "batch: event record");
    if (rc != ACCR_OK) return rc;
    BatchArgs a = args_for(P, B->dev, B->counters);
    if ((rc = launch_guard("batch_kernel")) != ACCR_OK) return rc;
    batch_kernel<<<batch_grid(P), BB, 0, s>>>(a);
    rc = launched("batch_kernel");
    if (rc != ACCR_OK) return rc;
    if (flags & ACCR_SYNC) return cuda_check(cudaStreamSynchronize(s), "batch: sync");
    return ACCR_OK;
}

int batch_launch_regions(const accr_region *regions, int64_t nregions, accr_stream_t stream, int64_t tile_bytes) {
    HostPlan &P = thread_plan(tile_bytes);
    int rc = plan_from_regions(regions, nregions, P);
    if (rc != ACCR_OK) return rc;
    return run_once(P, 0, stream);
}

}  // namespace accr

// ---- prepared batches -----------------------------------------------------------------

struct accr_batch {
    int device = 0;
    char *dev = nullptr;
    unsigned *counters = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    int64_t nregions = 0;
};

using namespace accr;

// The unbatched form: one single-region launch per region, in order.
static int run_plain(const accr_region *regs, int64_t R, unsigned flags, accr_stream_t stream) {
    if (R < 0 || (R > 0 && !regs)) return set_error(ACCR_EINVAL, "batch: bad region array");
    cudaStream_t s = (cudaStream_t)stream;
    for (int64_t r = 0; r < R; ++r) {
        const accr_region &g = regs[r];
        if (g.flags & ~ACCR_COMPENSATED) return set_error(ACCR_EINVAL, "region %lld: bad flags", (long long)r);
        ClauseDev cl[ACCR_MAX_CLAUSES];
        int rc = lower_clauses(g.in_type, g.clauses, g.nclauses, g.flags, cl);
        if (rc != ACCR_OK) return rc;
        rc = check_region_ptr(g.in, g.n, g.in_type, r);
        if (rc != ACCR_OK) return rc;
        const int grid = reduce_grid(g.in_type, g.nclauses, g.n);
        Scratch *scr = scratch_for(stream, (size_t)g.nclauses * grid * sizeof(Partial));
        if (!scr) return ACCR_ENOMEM;
        rc = reduce_launch(g.in, g.n, g.in_type, cl, g.nclauses, 0, (Partial *)scr->buf, scr->counters, grid, s);
        if (rc != ACCR_OK) return rc;
    }
    if (flags & ACCR_SYNC) return cuda_check(cudaStreamSynchronize(s), "batch: sync");
    return ACCR_OK;
}

extern "C" ACCR_API int accr_batch_reduce(const accr_region *regions, int64_t nregions, uint32_t flags,
                                          accr_stream_t stream) {
    ACCR_TRACE("accr_batch_reduce");
    clear_error();
    if (flags & ~(ACCR_SYNC | ACCR_PLAIN))
        return set_error(ACCR_EINVAL, "accr_batch_reduce: unsupported flags 0x%x", flags);
    if (flags & ACCR_PLAIN) return run_plain(regions, nregions, flags, stream);
    HostPlan &P = thread_plan(0);
    int rc = plan_from_regions(regions, nregions, P);
    if (rc != ACCR_OK) return rc;
    return run_once(P, flags, stream);
}

extern "C" ACCR_API int accr_segmented_reduce(const void *values, const int64_t *offsets, int64_t nseg,
                                              int32_t in_type, const accr_clause *clauses, int32_t nclauses,
                                              uint32_t flags, accr_stream_t stream) {
    ACCR_TRACE("accr_segmented_reduce");
    clear_error();
    if (flags & ~(ACCR_SYNC | ACCR_COMPENSATED))
        return set_error(ACCR_EINVAL, "accr_segmented_reduce: unsupported flags 0x%x", flags);
    HostPlan &P = thread_plan(0);
    int rc = plan_from_segments(values, offsets, nseg, in_type, clauses, nclauses, flags, P);
    if (rc != ACCR_OK) return rc;
    return run_once(P, flags, stream);
}

extern "C" ACCR_API int accr_batch_create(const accr_region *regions, int64_t nregions, uint32_t flags,
                                          accr_batch **out) {
    ACCR_TRACE("accr_batch_create");
    clear_error();
    if (!out) return set_error(ACCR_EINVAL, "accr_batch_create: batch is NULL");
    *out = nullptr;
    if (flags != 0) return set_error(ACCR_EINVAL, "accr_batch_create: unsupported flags 0x%x", flags);
    HostPlan P;
    int rc = plan_from_regions(regions, nregions, P);
    if (rc != ACCR_OK) return rc;
    accr_batch *b = new accr_batch();
    cudaGetDevice(&b->device);
    b->nregions = nregions;
    auto fail = [&](int code) {
        accr_batch_destroy(b);
        return code;
    };
    const size_t R = P.regions.size() + 4;  // queues + one counter per region
    if (cudaMalloc(&b->dev, P.total_bytes) != cudaSuccess || cudaMalloc(&b->counters, R * 4) != cudaSuccess) {
        cudaGetLastError();
        set_error(ACCR_ENOMEM, "accr_batch_create: cudaMalloc failed");
        return fail(ACCR_ENOMEM);
    }
    std::vector<char> host(P.plan_bytes);
    write_plan(P, host.data());
    if ((rc = cuda_check(cudaMemcpy(b->dev, host.data(), P.plan_bytes, cudaMemcpyHostToDevice), "accr_batch_create: upload")) != ACCR_OK)
        return fail(rc);
    if ((rc = cuda_check(cudaMemset(b->counters, 0, R * 4), "accr_batch_create: counters")) != ACCR_OK) return fail(rc);
    if ((rc = cuda_check(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming), "accr_batch_create: event")) != ACCR_OK)
        return fail(rc);
    if (P.regions.empty()) {
        *out = b;
        return ACCR_OK;
    }
    // capture the persistent launch once; accr_batch_launch replays it
    cudaStream_t cs;
    if ((rc = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "accr_batch_create: stream")) != ACCR_OK)
        return fail(rc);
    BatchArgs a = args_for(P, b->dev, b->counters);
    const int grid = batch_grid(P);
    rc = cuda_check(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "accr_batch_create: capture");
    if (rc == ACCR_OK) {
        batch_kernel<<<grid, BB, 0, cs>>>(a);
        cudaError_t le = cudaGetLastError();
        cudaError_t ce = cudaStreamEndCapture(cs, &b->graph);
        rc = cuda_check(le != cudaSuccess ? le : ce, "accr_batch_create: end capture");
    }
    if (rc == ACCR_OK) rc = cuda_check(cudaGraphInstantiate(&b->exec, b->graph, 0), "accr_batch_create: instantiate");
    cudaStreamDestroy(cs);
    if (rc != ACCR_OK) return fail(rc);
    *out = b;
    return ACCR_OK;
}

extern "C" ACCR_API int accr_batch_launch(accr_batch *b, accr_stream_t stream) {
    ACCR_TRACE("accr_batch_launch");
    clear_error();
    if (!b) return set_error(ACCR_EINVAL, "accr_batch_launch: batch is NULL");
    if (!b->exec) return ACCR_OK;  // empty batch
    int rc = launch_guard("accr_batch_launch");
    if (rc != ACCR_OK) return rc;
    rc = cuda_check(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "accr_batch_launch");
    if (rc != ACCR_OK) return rc;
    rc = launched("batch_kernel (graph)");
    if (rc != ACCR_OK) return rc;
    return cuda_check(cudaEventRecord(b->done, (cudaStream_t)stream), "accr_batch_launch: event");
}

extern "C" ACCR_API int accr_batch_destroy(accr_batch *b) {
    ACCR_TRACE("accr_batch_destroy");
    clear_error();
    if (!b) return ACCR_OK;
    int rc = ACCR_OK;
    if (b->done) rc = cuda_check(cudaEventSynchronize(b->done), "accr_batch_destroy: wait");
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->done) cudaEventDestroy(b->done);
    if (b->dev) cudaFree(b->dev);
    if (b->counters) cudaFree(b->counters);
    delete b;
    return rc;
}

extern "C" ACCR_API int accr_batch_tiling(int64_t small_bytes, int64_t tile_bytes, int64_t *old_small,
                                          int64_t *old_tile) {
    clear_error();
    if (small_bytes < 0 || tile_bytes < 0 || small_bytes % 16 || tile_bytes % 16 ||
        (tile_bytes != 0 && tile_bytes < 4096))
        return set_error(ACCR_EINVAL, "accr_batch_tiling: sizes must be multiples of 16, tile >= 4096");
    if (old_small) *old_small = g_small_bytes.load();
    if (old_tile) *old_tile = g_tile_bytes.load();
    if (small_bytes) g_small_bytes.store(small_bytes);
    if (tile_bytes) g_tile_bytes.store(tile_bytes);
    return ACCR_OK;
}
