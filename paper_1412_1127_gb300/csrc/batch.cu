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
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "fold.cuh"

namespace accr {

// Defined in reduce.cu (the single-region path, used by the unbatched form).
int reduce_grid(int in_type, int nc, int64_t n);
int reduce_launch(const void *in, int64_t n, int in_type, const ClauseDev *cl, int nc, int two_level,
                  Partial *partials, unsigned *counter, int grid, cudaStream_t s);

constexpr int BB = 256;  // threads per CTA (4 CTAs per SM: one CTA's merge between tiles overlaps the others' streaming)
constexpr int BU = 4;    // 16-byte vectors per thread per iteration (tiles)
constexpr int SU = 8;    // 16-byte vectors per lane per iteration (warp regions)

struct RegionDev {
    const void *in;
    int64_t n;
    int64_t tile0;  // first tile of a tiled region; -1 for a warp region
    int32_t in_type;
    int32_t nc;
    ClauseDev cl[ACCR_MAX_CLAUSES];
};
static_assert(sizeof(RegionDev) == 192, "RegionDev layout");

struct BatchArgs {
    const RegionDev *regions;
    const int2 *tiles;           // [T] (region, tile index in region), in queue order
    const int32_t *small;        // [S] warp regions, in queue order
    int64_t T, S;
    int64_t tile_bytes;
    Partial *partials;           // [sum of tiles][ACCR_MAX_CLAUSES], slot tile0 + k
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
            p.partials[t * ACCR_MAX_CLAUSES + c] = q;
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
    int fw[NC];
    uint64_t fid[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        fw[c] = final_code(w[c]);
        fid[c] = final_ident(d->cl[c]);
        A[c].a = fid[c];
        A[c].c = 0.f;
        for (int64_t j = threadIdx.x; j < ntiles; j += BB) {
            Partial q = ld_partial_cg(&p.partials[(tile0 + j) * ACCR_MAX_CLAUSES + c]);
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
    __shared__ Acc sh[ACCR_MAX_CLAUSES][BB / 32];
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
        const RegionDev *d = regions + tk.x;
        const int type = d->in_type, nc = d->nc;
        ACCR_DISPATCH_TYPE_NC(type, nc, tile_fold, p, d, tk.x, (int64_t)tk.y, sh, &s_last);
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
        const RegionDev *d = regions + small[s];
        const int type = d->in_type, nc = d->nc;
        ACCR_DISPATCH_TYPE_NC(type, nc, warp_fold, d, lane);
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

__global__ void __launch_bounds__(BB, 4) batch_kernel(const __grid_constant__ BatchArgs p) {
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

__global__ void __launch_bounds__(BB, 4) batch_kernel_inline(const __grid_constant__ BatchArgsInline p) {
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

static int log2_floor(uint64_t v) {
    int b = 0;
    while (v >>= 1) ++b;
    return b;
}

// Assigns each region to the warp list or to tiles, by its own type and
// length, and orders both queues: grouped by (element type, clause count) so
// that neighbouring work runs the same code, largest first within a group so
// that the small pieces fill in at the end.  (Counting sort on a size bucket.)
static int finish_plan(HostPlan &P) {
    const int64_t small_b = g_small_bytes.load(), tile_b = P.tile_override > 0 ? P.tile_override : g_tile_bytes.load();
    P.tile_bytes = tile_b;
    P.tiles.clear();
    P.small.clear();
    const int64_t R = (int64_t)P.regions.size();
    constexpr int NKEY = 8 * 64;
    std::vector<int64_t> tile_count(NKEY + 1, 0), small_count(NKEY + 1, 0);
    int64_t slots = 0;
    auto key_of = [](const RegionDev &d, int64_t bytes) {
        const int group = d.in_type * 2 + (d.nc - 1);
        return group * 64 + (63 - log2_floor((uint64_t)(bytes > 0 ? bytes : 1)));
    };
    for (int64_t r = 0; r < R; ++r) {
        RegionDev &d = P.regions[r];
        const int64_t eb = type_bytes(d.in_type);
        if (d.n * eb <= small_b) {
            d.tile0 = -1;
            small_count[key_of(d, d.n * eb) + 1]++;
        } else {
            const int64_t te = tile_b / eb;
            const int64_t nt = (d.n + te - 1) / te;
            d.tile0 = slots;
            slots += nt;
            if (slots > INT32_MAX) return set_error(ACCR_EINVAL, "batch: more than 2^31 tiles");
            tile_count[key_of(d, tile_b) + 1] += nt - 1;
            tile_count[key_of(d, (d.n - (nt - 1) * te) * eb) + 1]++;
        }
    }
    for (int k = 0; k < NKEY; ++k) {
        tile_count[k + 1] += tile_count[k];
        small_count[k + 1] += small_count[k];
    }
    P.ntiles = slots;
    P.tiles.resize((size_t)tile_count[NKEY]);
    P.small.resize((size_t)small_count[NKEY]);
    for (int64_t r = 0; r < R; ++r) {
        const RegionDev &d = P.regions[r];
        const int64_t eb = type_bytes(d.in_type);
        if (d.tile0 < 0) {
            P.small[(size_t)small_count[key_of(d, d.n * eb)]++] = (int32_t)r;
        } else {
            const int64_t te = tile_b / eb;
            const int64_t nt = (d.n + te - 1) / te;
            const int kfull = key_of(d, tile_b), klast = key_of(d, (d.n - (nt - 1) * te) * eb);
            for (int64_t k = 0; k < nt; ++k)
                P.tiles[(size_t)tile_count[k + 1 < nt ? kfull : klast]++] = make_int2((int)r, (int)k);
        }
    }
    P.off_tiles = align_up(sizeof(RegionDev) * (size_t)R, 256);
    P.off_small = align_up(P.off_tiles + sizeof(int2) * P.tiles.size(), 256);
    P.plan_bytes = P.off_small + 4 * P.small.size();
    P.off_partials = align_up(P.plan_bytes, 256);
    P.total_bytes = P.off_partials + sizeof(Partial) * ACCR_MAX_CLAUSES * (size_t)P.ntiles + 256;
    return ACCR_OK;
}

static void write_plan(const HostPlan &P, char *dst) {
    memcpy(dst, P.regions.data(), sizeof(RegionDev) * P.regions.size());
    if (!P.tiles.empty()) memcpy(dst + P.off_tiles, P.tiles.data(), sizeof(int2) * P.tiles.size());
    if (!P.small.empty()) memcpy(dst + P.off_small, P.small.data(), 4 * P.small.size());
}

static int check_region_ptr(const void *in, int64_t n, int t, int64_t r) {
    if (n < 0) return set_error(ACCR_EINVAL, "region %lld: n < 0", (long long)r);
    if (n > 0 && !in) return set_error(ACCR_EINVAL, "region %lld: in is NULL", (long long)r);
    if (((uintptr_t)in % (uintptr_t)type_bytes(t)) != 0)
        return set_error(ACCR_EINVAL, "region %lld: in is not aligned to its element size", (long long)r);
    return ACCR_OK;
}

// Appends a region's descriptor; one with three or four clauses becomes two
// descriptors over the same elements (clauses 0-1 and 2-3).
static void push_split(std::vector<RegionDev> &out, const RegionDev &d) {
    if (d.nc <= 2) {
        out.push_back(d);
        return;
    }
    RegionDev a = d, b = d;
    a.nc = 2;
    b.nc = d.nc - 2;
    b.cl[0] = d.cl[2];
    b.cl[1] = d.cl[3];
    out.push_back(a);
    out.push_back(b);
}

static int plan_from_regions(const accr_region *regs, int64_t R, HostPlan &P) {
    if (R < 0 || (R > 0 && !regs)) return set_error(ACCR_EINVAL, "batch: bad region array");
    if (R > INT32_MAX / 2) return set_error(ACCR_EINVAL, "batch: too many regions");
    P.regions.clear();
    P.regions.reserve((size_t)R);
    for (int64_t r = 0; r < R; ++r) {
        const accr_region &g = regs[r];
        if (g.flags & ~ACCR_COMPENSATED) return set_error(ACCR_EINVAL, "region %lld: bad flags", (long long)r);
        RegionDev d;
        memset(&d, 0, sizeof d);
        int rc = lower_clauses(g.in_type, g.clauses, g.nclauses, g.flags, d.cl);
        if (rc != ACCR_OK) return rc;
        rc = check_region_ptr(g.in, g.n, g.in_type, r);
        if (rc != ACCR_OK) return rc;
        d.in = g.in;
        d.n = g.n;
        d.in_type = g.in_type;
        d.nc = g.nclauses;
        push_split(P.regions, d);
    }
    return finish_plan(P);
}

static int plan_from_segments(const void *values, const int64_t *off, int64_t nseg, int in_type,
                              const accr_clause *clauses, int nc, unsigned flags, HostPlan &P) {
    if (nseg < 0 || (nseg > 0 && !off)) return set_error(ACCR_EINVAL, "segmented: bad offsets");
    if (nseg > INT32_MAX / 2) return set_error(ACCR_EINVAL, "segmented: too many segments");
    ClauseDev base[ACCR_MAX_CLAUSES];
    int rc = lower_clauses(in_type, clauses, nc, flags & ACCR_COMPENSATED, base);
    if (rc != ACCR_OK) return rc;
    const int64_t eb = type_bytes(in_type);
    P.regions.clear();
    P.regions.reserve((size_t)nseg * (nc > 2 ? 2 : 1));
    for (int64_t s = 0; s < nseg; ++s) {
        const int64_t lo = off[s], hi = off[s + 1];
        if (lo < 0 || hi < lo) return set_error(ACCR_EINVAL, "segmented: offsets not non-decreasing at %lld", (long long)s);
        RegionDev d;
        memset(&d, 0, sizeof d);
        d.in = (const char *)values + lo * eb;
        rc = check_region_ptr(d.in, hi - lo, in_type, s);
        if (rc != ACCR_OK) return rc;
        if (hi > lo && !values) return set_error(ACCR_EINVAL, "segmented: values is NULL");
        d.n = hi - lo;
        d.in_type = in_type;
        d.nc = nc;
        for (int c = 0; c < nc; ++c) {
            d.cl[c] = base[c];
            d.cl[c].out = (char *)base[c].out + s * type_bytes(base[c].acc_type);
        }
        push_split(P.regions, d);
    }
    return finish_plan(P);
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
    HostPlan P;
    P.tile_override = tile_bytes;
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
    clear_error();
    if (flags & ~(ACCR_SYNC | ACCR_PLAIN))
        return set_error(ACCR_EINVAL, "accr_batch_reduce: unsupported flags 0x%x", flags);
    if (flags & ACCR_PLAIN) return run_plain(regions, nregions, flags, stream);
    HostPlan P;
    int rc = plan_from_regions(regions, nregions, P);
    if (rc != ACCR_OK) return rc;
    return run_once(P, flags, stream);
}

extern "C" ACCR_API int accr_segmented_reduce(const void *values, const int64_t *offsets, int64_t nseg,
                                              int32_t in_type, const accr_clause *clauses, int32_t nclauses,
                                              uint32_t flags, accr_stream_t stream) {
    clear_error();
    if (flags & ~(ACCR_SYNC | ACCR_COMPENSATED))
        return set_error(ACCR_EINVAL, "accr_segmented_reduce: unsupported flags 0x%x", flags);
    HostPlan P;
    int rc = plan_from_segments(values, offsets, nseg, in_type, clauses, nclauses, flags, P);
    if (rc != ACCR_OK) return rc;
    return run_once(P, flags, stream);
}

extern "C" ACCR_API int accr_batch_create(const accr_region *regions, int64_t nregions, uint32_t flags,
                                          accr_batch **out) {
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
