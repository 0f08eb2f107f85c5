// patterns.cu -- three region patterns from the paper's application study
// (IPMACC Sec. 4.2), on the same single-pass reduction machinery:
//
//  * Nearest Neighbor: distances to a query point and the k smallest -- a
//    reduction whose operator keeps a sorted list of k (distance, index)
//    pairs.  Each warp keeps one list in shared memory and tests a whole round
//    of its points against the list's k-th distance at once; distance bounds
//    (a warp's first round, then one taken from a sample of the whole array
//    and published while the scan runs) keep the lists' slow path rare.  The
//    CTA ranks its warps' entries, and the last CTA to finish ranks the few
//    CTA entries that can still be among the k smallest.
//
//  * SRAD: a reduction region whose result feeds a data-parallel region.  The
//    paper's OpenACC code merges the block partials on the CPU and launches
//    the next region; here one cooperative launch does both: the last CTA of
//    the reduction publishes the statistics, every CTA waits for them at a
//    bounded grid barrier and then runs the elementwise pass (for arrays that
//    fit in L2 the second pass reads from L2).  Unfused and two-level host
//    forms are kept for comparison.
//
//  * BFS: a level-synchronous loop that stops when no cell changed.  The
//    OpenACC version reduces a global boolean with ||; the CUDA version
//    initialises the flag and lets threads write only `true`.  Both forms run
//    here with the host driving the levels, and a third keeps every level in
//    one cooperative launch with a bounded grid barrier between levels.
//
// Every cross-CTA wait spins a bounded number of times; on expiry it records
// a code in a status word and the host reports ACCR_ETIMEDOUT.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "common.cuh"
#include "debug.cuh"
#include "fold.cuh"

namespace accr {

constexpr uint32_t kSpinLimit = 20000000u;  // ~seconds of __nanosleep(64) polls

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier for a cooperative launch that also ORs one CTA-uniform flag:
// generation counting, bounded spin.  bar[0] counts arrivals (low 20 bits)
// and raised flags (bits 20 and up); bar[1] holds (generation << 1) | OR of
// the flags, published by the last CTA to arrive, so the flag comes back
// with the release instead of through a word of its own.  Returns 0 if the
// wait ran out, else 1 + the OR of the flags.
__device__ __forceinline__ int grid_barrier_or(unsigned *bar, unsigned &gen, bool flag) {
    __shared__ int s_res;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned my = (gen + 1) & 0x7fffffffu;
        __threadfence();
        const unsigned old = atomicAdd(&bar[0], 1u + (flag ? (1u << 20) : 0u));
        int res = 0;
        if ((old & 0xfffffu) == gridDim.x - 1) {
            const unsigned any = ((old >> 20) != 0u || flag) ? 1u : 0u;
            bar[0] = 0u;
            st_release(&bar[1], (my << 1) | any);
            res = 1 + (int)any;
        } else {
            uint32_t i = 0;
            unsigned v = ld_acquire(&bar[1]);
            while ((v >> 1) != my && ++i <= kSpinLimit) {
                __nanosleep(64);
                v = ld_acquire(&bar[1]);
            }
            if ((v >> 1) == my) res = 1 + (int)(v & 1u);
        }
        s_res = res;
    }
    gen = (gen + 1) & 0x7fffffffu;
    __syncthreads();
    return s_res;
}

// ============================================================================
// Nearest Neighbor: k smallest squared distances
// ============================================================================

constexpr int NK_THREADS = 256;

struct __align__(16) PairSlot {
    int64_t i;
    float d;
    uint32_t pad;
};

__device__ __forceinline__ bool pless(float da, int64_t ia, float db, int64_t ib) {
    return da < db || (da == db && ia < ib);
}

// Streaming 16-byte load of two points (read once: no L1 allocation).
__device__ __forceinline__ float4 ld_pts(const float4 *p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

__device__ __forceinline__ float sqdist(float x, float y, float qx, float qy) {
    const float dx = __fsub_rn(x, qx), dy = __fsub_rn(y, qy);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));  // no fused multiply-add
}

// One list per warp in shared memory, kept sorted in the (distance, index)
// order; its first k entries are the warp's k smallest so far, and every
// lane keeps the k-th (the threshold) in registers.  Entries past the k-th
// never rise above it, so they never matter.  A lane's candidate that beats
// the threshold is found by a ballot; such candidates (rare once the list
// holds real points, or from the start under a bound) go through the
// out-of-line slow path one at a time, lane 0 inserting into the shared list.
struct Thr {
    float d;
    int64_t i;
};

template <int KT>
__device__ __noinline__ Thr warp_insert_slow(float *LD, int64_t *LI, int k, float d, int64_t i, unsigned mask) {
    const int lane = threadIdx.x & 31;
    while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const float cd = __shfl_sync(0xffffffffu, d, src);
        const int64_t ci = (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)i, src);
        if (lane == 0 && pless(cd, ci, LD[k - 1], LI[k - 1])) {
            int j = k - 1;
            while (j > 0 && pless(cd, ci, LD[j - 1], LI[j - 1])) {
                LD[j] = LD[j - 1];
                LI[j] = LI[j - 1];
                --j;
            }
            LD[j] = cd;
            LI[j] = ci;
        }
        __syncwarp();
    }
    Thr t;
    t.d = LD[k - 1];
    t.i = LI[k - 1];
    __syncwarp();
    return t;
}

// The hot path is one compare: d <= the warp's k-th distance admits a
// superset of the winners (ties included); the slow path applies the exact
// (distance, index) order.
template <int KT>
__device__ __forceinline__ void warp_offer(float *LD, int64_t *LI, int k, Thr &thr, float d, int64_t i) {
    const unsigned mask = __ballot_sync(0xffffffffu, d <= thr.d);
    if (mask) thr = warp_insert_slow<KT>(LD, LI, k, d, i, mask);
}

// A distance bound B that at least k distinct points reach may stand in for
// k placeholders (B, no index): every entry of the list at or past (B, no
// index) becomes one (the prefix below it stays), so the list keeps the k
// smallest of what it held and the placeholders.  Returns the new threshold.
template <int KT>
__device__ __noinline__ Thr warp_apply_bound(float *LD, int64_t *LI, int k, float B) {
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int j = 0; j < KT; ++j)
            if (!pless(LD[j], LI[j], B, INT64_MAX)) {
                LD[j] = B;
                LI[j] = INT64_MAX;
            }
    }
    __syncwarp();
    Thr t;
    t.d = LD[k - 1];
    t.i = LI[k - 1];
    __syncwarp();
    return t;
}

// The k-th smallest of one value per lane (k <= 32; every lane gets it).
__device__ __forceinline__ float warp_kth_smallest(float v, int k) {
    const int lane = threadIdx.x & 31;
    float t = INFINITY;
    for (int r = 0; r < k; ++r) {
        float w = v;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) w = fminf(w, __shfl_xor_sync(0xffffffffu, w, o));
        t = w;
        const unsigned who = __ballot_sync(0xffffffffu, v == w);
        if (lane == __ffs(who) - 1) v = INFINITY;  // exactly one lane gives up its value
    }
    return t;
}

// The CTA's KT smallest of its warps' lists (shared memory), written to
// MD/MI: each entry's rank is the number of entries before it in the
// (distance, index) order, equal entries (placeholders) ordered by position,
// so the ranks are distinct and entry r of the result is the one of rank r.
template <int KT, int NT>
__device__ __forceinline__ void cta_merge_warp_lists(const float (*wld)[KT], const int64_t (*wli)[KT], float *MD,
                                                     int64_t *MI) {
    constexpr int NC = (NT / 32) * KT;
    __syncthreads();
    const float *fd = &wld[0][0];
    const int64_t *fi = &wli[0][0];
    for (int c = threadIdx.x; c < NC; c += NT) {
        const float dc = fd[c];
        const int64_t ic = fi[c];
        int rank = 0;
        for (int o = 0; o < NC; ++o) {
            const float dd = fd[o];
            const int64_t io = fi[o];
            rank += (pless(dd, io, dc, ic) || (dd == dc && io == ic && o < c)) ? 1 : 0;
        }
        if (rank < KT) {
            MD[rank] = dc;
            MI[rank] = ic;
        }
    }
    __syncthreads();
}

// The sampled bound.  Every CTA of the scan launch takes NK_SAMPLE
// consecutive points at blockIdx.x * sample_stride (so the sample spreads
// over the whole array) and records its smallest distance; those minima
// belong to distinct points, so the k-th smallest of them is a distance that
// at least k points reach.  The last CTA to record its minimum selects it and
// publishes it as one word (its bits + 1; zero means not yet).  Nobody waits
// for it: each warp polls the word once per round and applies the bound when
// it appears; until then its first round's own k-th smallest lane minimum
// serves as a bound.
constexpr int NK_SAMPLE = NK_THREADS;        // points sampled per CTA (one per thread)
constexpr int64_t NK_BOUND_MIN_N = 1 << 22;  // smaller inputs skip the sampled bound

template <int KT>
__device__ __forceinline__ void flist_insert(float (&D)[KT], float d) {
    if (!(d < D[KT - 1])) return;  // NaN never enters
#pragma unroll
    for (int j = KT - 1; j > 0; --j) D[j] = d < D[j - 1] ? D[j - 1] : (d < D[j] ? d : D[j]);
    D[0] = d < D[0] ? d : D[0];
}

// The k-th smallest of cnt values (one warp; every lane gets it; k <= KT).
template <int KT>
__device__ __forceinline__ float kth_of_values(const float *v, int cnt, int k) {
    const int lane = threadIdx.x & 31;
    float D[KT];
#pragma unroll
    for (int j = 0; j < KT; ++j) D[j] = INFINITY;
    for (int j0 = lane; j0 < cnt; j0 += 32 * 8) {
        float mv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) mv[u] = (j0 + 32 * u < cnt) ? __ldcg(v + j0 + 32 * u) : INFINITY;  // in flight together
#pragma unroll
        for (int u = 0; u < 8; ++u) flist_insert<KT>(D, mv[u]);
    }
    // k rounds of a warp minimum, each taking the head of exactly one lane
    float t = INFINITY;
    for (int r = 0; r < k; ++r) {
        float w = D[0];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) w = fminf(w, __shfl_xor_sync(0xffffffffu, w, o));
        t = w;
        const unsigned who = __ballot_sync(0xffffffffu, D[0] == w);
        if (lane == __ffs(who) - 1) {
#pragma unroll
            for (int j = 0; j < KT - 1; ++j) D[j] = D[j + 1];
            D[KT - 1] = INFINITY;
        }
    }
    return t;
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Last CTA: the k smallest of the G <= 2 NT CTA lists (each sorted) by k
// rounds of a tournament over the lists' heads.  Thread t holds the heads of
// lists t and t + NT and the entry after each (loaded ahead, so the winner of
// a round seldom waits for its next entry); a round takes the CTA-wide
// smallest (distance, index, list) and its list advances.
constexpr int NK_MAX_GRID = 2 * NK_THREADS;  // CTA lists the tournament takes
template <int KT, int NT>
__device__ __noinline__ void final_tournament(const PairSlot *partials, int G, int k, float *MD, int64_t *MI) {
    __shared__ float wd[2][NT / 32];
    __shared__ int64_t wi[2][NT / 32];
    __shared__ int wo[2][NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NONE = 0x7fffffff;  // no list
    auto slot = [&](int L, int j, float &d, int64_t &i) {
        if (L < G && j < k) {
            const uint4 r = __ldcg(reinterpret_cast<const uint4 *>(partials + (int64_t)L * KT + j));
            d = __uint_as_float(r.z);
            i = (int64_t)(((uint64_t)r.y << 32) | r.x);
        } else {
            d = INFINITY;
            i = INT64_MAX;
        }
    };
    const int L0 = threadIdx.x, L1 = threadIdx.x + NT;
    float h0, n0, h1, n1;
    int64_t g0, m0, g1, m1;
    slot(L0, 0, h0, g0);
    slot(L1, 0, h1, g1);
    slot(L0, 1, n0, m0);
    slot(L1, 1, n1, m1);
    int p0 = 0, p1 = 0;
    for (int r = 0; r < k; ++r) {
        const bool second = pless(h1, g1, h0, g0);  // ties: the lower list
        float d = second ? h1 : h0;
        int64_t i = second ? g1 : g0;
        int o = (second ? L1 : L0) < G ? (second ? L1 : L0) : NONE;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            const float od = __shfl_xor_sync(0xffffffffu, d, s);
            const int64_t oi = (int64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)i, s);
            const int oo = __shfl_xor_sync(0xffffffffu, o, s);
            if (pless(od, oi, d, i) || (od == d && oi == i && oo < o)) d = od, i = oi, o = oo;
        }
        if (lane == 0) wd[r & 1][warp] = d, wi[r & 1][warp] = i, wo[r & 1][warp] = o;
        __syncthreads();
        d = wd[r & 1][0], i = wi[r & 1][0], o = wo[r & 1][0];
#pragma unroll
        for (int w = 1; w < NT / 32; ++w) {
            const float od = wd[r & 1][w];
            const int64_t oi = wi[r & 1][w];
            const int oo = wo[r & 1][w];
            if (pless(od, oi, d, i) || (od == d && oi == i && oo < o)) d = od, i = oi, o = oo;
        }
        if (threadIdx.x == 0) MD[r] = d, MI[r] = i;
        if (o == L0) {  // the winner's list advances; the entry after the new head is loaded ahead
            h0 = n0, g0 = m0, ++p0;
            slot(L0, p0 + 1, n0, m0);
        } else if (o == L1) {
            h1 = n1, g1 = m1, ++p1;
            slot(L1, p1 + 1, n1, m1);
        }
    }
    __syncthreads();
}

// With sample_stride > 0 every CTA samples, the last one publishes the
// sampled bound in bstate[1], and warps pick it up as described above.
// bstate[0] counts the CTAs that recorded their sample minimum; the last CTA
// of the launch returns both words to zero.
template <int KT, int NT>
__global__ void __launch_bounds__(NT, 2) nearest_kernel(const float *__restrict__ pts, int64_t n, float qx, float qy,
                                                     int k, int64_t *idx_out, float *d_out, PairSlot *partials,
                                                     unsigned *counter, int64_t sample_stride, float *minima,
                                                     unsigned *bstate) {
    __shared__ float wld[NT / 32][KT];
    __shared__ int64_t wli[NT / 32][KT];
    __shared__ float MD[KT];
    __shared__ int64_t MI[KT];
    __shared__ float s_min[NT / 32];
    __shared__ int am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *LD = wld[warp];
    int64_t *LI = wli[warp];
    if (lane < KT) {
        LD[lane] = INFINITY;
        LI[lane] = INT64_MAX;
    }
    __syncwarp();
    Thr thr;
    thr.d = INFINITY;
    thr.i = INT64_MAX;
    // points are float2; the vector part starts at a 16-byte boundary
    const int64_t head = (((uintptr_t)pts & 15) != 0 && n > 0) ? 1 : 0;
    const float4 *v4 = (const float4 *)(pts + 2 * head);
    const int64_t npairs = (n - head) / 2;
    const int64_t nth = (int64_t)gridDim.x * NT;
    // Full rounds: NU 16-byte loads (2 points each) per lane, every one in
    // range, so no per-point bounds test; the round's smallest distance is
    // compared once with the warp's k-th, and only a round in which some lane
    // beats it tests its points.  The trip count is uniform across each warp
    // so that the votes see 32 lanes.
    constexpr int NU = 16;
    const int64_t vstep = nth * NU;
    int64_t vb = (int64_t)blockIdx.x * (NT * NU) + warp * 32;
    float4 q[NU];
    bool full = vb + (NU - 1) * NT + 31 < npairs;  // uniform across the warp
    if (full) {  // the first round's loads go out before the sample
        const float4 *p = v4 + vb + lane;
#pragma unroll
        for (int u = 0; u < NU; ++u) q[u] = ld_pts(p + u * NT);
    }
    bool poll = false;
    if (sample_stride > 0) {
        const float2 sp = __ldg((const float2 *)pts + (int64_t)blockIdx.x * sample_stride + threadIdx.x);
        float m = sqdist(sp.x, sp.y, qx, qy);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_min[warp] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            float cm = s_min[0];
#pragma unroll
            for (int w = 1; w < NT / 32; ++w) cm = fminf(cm, s_min[w]);  // fminf passes over NaN
            minima[blockIdx.x] = cm;
            __threadfence();
            am_last = atomicAdd(&bstate[0], 1u) == gridDim.x - 1u;
        }
        __syncthreads();
        if (am_last && warp == 0) {
            __threadfence();
            const float t = kth_of_values<KT>(minima, (int)gridDim.x, k);
            if (lane == 0) st_release(&bstate[1], __float_as_uint(t) + 1u);  // t in [0, inf]: never wraps to 0
        }
        poll = true;
    }
    if (blockIdx.x == 0 && warp == 0) {  // the unaligned first point and the odd last point
        const int64_t last = head + 2 * npairs;
        float d = INFINITY;
        int64_t i = INT64_MAX;
        if (lane == 0 && head) d = sqdist(pts[0], pts[1], qx, qy), i = 0;
        if (lane == 1 && last < n) d = sqdist(pts[2 * last], pts[2 * last + 1], qx, qy), i = last;
        warp_offer<KT>(LD, LI, k, thr, d, i);
    }
    while (full) {
        const unsigned pb = (poll && lane == 0) ? ld_relaxed(&bstate[1]) : 0u;  // the bound, if published
        float dm = INFINITY;
#pragma unroll
        for (int u = 0; u < NU; ++u)
            dm = fminf(dm, fminf(sqdist(q[u].x, q[u].y, qx, qy), sqdist(q[u].z, q[u].w, qx, qy)));
        if (poll) {
            const unsigned b = __shfl_sync(0xffffffffu, pb, 0);
            if (b != 0u) {
                const float B = __uint_as_float(b - 1u);
                if (B < thr.d) thr = warp_apply_bound<KT>(LD, LI, k, B);
                poll = false;
            }
        }
        if (thr.d == INFINITY && k <= 32) {  // no bound yet: the k-th smallest lane minimum of this round
            const float B = warp_kth_smallest(dm, k);   // k distinct points reach it
            if (B < thr.d) thr = warp_apply_bound<KT>(LD, LI, k, B);
        }
        if (__any_sync(0xffffffffu, dm <= thr.d)) {
            // the points of this lane that beat the threshold now (it only
            // falls, so later winners are among them), then one pass over
            // the positions some lane has, in order
            unsigned bits = 0u;
#pragma unroll
            for (int j = 0; j < 2 * NU; ++j) {
                const float4 &v = q[j >> 1];
                const float dj = (j & 1) ? sqdist(v.z, v.w, qx, qy) : sqdist(v.x, v.y, qx, qy);
                bits |= (dj <= thr.d ? 1u : 0u) << j;
            }
            const unsigned any = __reduce_or_sync(0xffffffffu, bits);
            const int64_t ibase = head + 2 * (vb + lane);  // this lane's first point this round
#pragma unroll
            for (int j = 0; j < 2 * NU; ++j) {
                if (any & (1u << j)) {  // uniform across the warp
                    const float4 &v = q[j >> 1];
                    const float dj = (j & 1) ? sqdist(v.z, v.w, qx, qy) : sqdist(v.x, v.y, qx, qy);
                    const unsigned mask = __ballot_sync(0xffffffffu, ((bits >> j) & 1u) && dj <= thr.d);
                    if (mask) thr = warp_insert_slow<KT>(LD, LI, k, dj, ibase + 2 * (j >> 1) * NT + (j & 1), mask);
                }
            }
        }
        vb += vstep;
        full = vb + (NU - 1) * NT + 31 < npairs;
        if (full) {
            const float4 *p = v4 + vb + lane;
#pragma unroll
            for (int u = 0; u < NU; ++u) q[u] = ld_pts(p + u * NT);
        }
    }
    if (vb < npairs) {  // the last, partial round: points past the end never compete
        const int64_t ibase = head + 2 * (vb + lane);
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int64_t vv = vb + lane + u * NT;
            const bool ok = vv < npairs;
            const float4 v = ok ? ld_pts(v4 + vv) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float d0 = ok ? sqdist(v.x, v.y, qx, qy) : INFINITY;
            const float d1 = ok ? sqdist(v.z, v.w, qx, qy) : INFINITY;
            unsigned mask = __ballot_sync(0xffffffffu, ok && d0 <= thr.d);
            if (mask) thr = warp_insert_slow<KT>(LD, LI, k, d0, ibase + 2 * u * NT, mask);
            mask = __ballot_sync(0xffffffffu, ok && d1 <= thr.d);
            if (mask) thr = warp_insert_slow<KT>(LD, LI, k, d1, ibase + 2 * u * NT + 1, mask);
        }
    }
    cta_merge_warp_lists<KT, NT>(wld, wli, MD, MI);
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < KT; ++j) {
            PairSlot p;
            p.i = MI[j];
            p.d = MD[j];
            p.pad = 0;
            // the slots end where the sample's minima begin
            if (ACCR_DCHECK((int64_t)blockIdx.x * KT + j < (int64_t)((const char *)minima - (const char *)partials) /
                                                              (int64_t)sizeof(PairSlot),
                            DS_NEAREST_SLOT))
                partials[(int64_t)blockIdx.x * KT + j] = p;
        }
        __threadfence();
        am_last = atomicAdd(counter, 1u) == (unsigned)G - 1u;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    final_tournament<KT, NT>(partials, G, k, MD, MI);
    if (threadIdx.x == 0) {
        const int kk = ACCR_DCHECK(k >= 1 && k <= KT, DS_NEAREST_OUT) ? k : 0;  // the list holds KT entries
        for (int j = 0; j < kk; ++j) {
            const bool real = MI[j] != INT64_MAX;
            idx_out[j] = real ? MI[j] : -1;
            d_out[j] = real ? MD[j] : INFINITY;
        }
        *counter = 0u;
        if (sample_stride > 0) {  // every CTA has recorded its minimum and stopped polling
            bstate[0] = 0u;
            bstate[1] = 0u;
        }
    }
}

template <int KT>
static int nearest_launch(const float *pts, int64_t n, float qx, float qy, int k, int64_t *idx, float *d,
                          cudaStream_t s) {
    constexpr int NT = NK_THREADS;
    static int per_sm = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nearest_kernel<KT, NT>, NT, 0);
        if (per_sm < 1) per_sm = 1;
    });
    const DeviceInfo &di = device_info();
    const int64_t want = (n / 2 + NT * 16 - 1) / (NT * 16);  // one round of 16 vectors per thread
    const int64_t resident = std::min<int64_t>((int64_t)per_sm * di.sms, NK_MAX_GRID);
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), resident);
    // a sample of NK_SAMPLE points per CTA, spread over the array
    const bool use_bound = n >= NK_BOUND_MIN_N && grid >= 32 && n / grid >= NK_SAMPLE;
    // scratch: [partials: grid * KT slots][the CTAs' sample minima]
    const size_t part_bytes = sizeof(PairSlot) * (size_t)grid * KT;
    const size_t minima_off = (part_bytes + 255) & ~(size_t)255;
    Scratch *scr = scratch_for((accr_stream_t)s, minima_off + sizeof(float) * (size_t)grid);
    if (!scr) return ACCR_ENOMEM;
    PairSlot *partials = (PairSlot *)scr->buf;
    unsigned *counter = scr->counters + 1;
    unsigned *bstate = scr->counters + 5;  // words 5-6
    float *minima = (float *)((char *)scr->buf + minima_off);
    const int64_t stride = use_bound ? n / grid : 0;
    int rc = launch_guard("nearest_kernel");
    if (rc != ACCR_OK) return rc;
    // no CTA waits for another: a plain launch
    nearest_kernel<KT, NT><<<grid, NT, 0, s>>>(pts, n, qx, qy, k, idx, d, partials, counter, stride, minima, bstate);
    return launched("nearest_kernel");
}

// ============================================================================
// SRAD pattern: statistics of an array, then the standardised array
// ============================================================================

constexpr int SD_THREADS = 512;

struct __align__(16) StatPartial {
    float s1, c1, s2, c2;  // compensated sum of x and of x^2
};

struct StdShared {
    double mean, var;
    float mean_f, rstd_f;
};

__device__ __forceinline__ void stat_merge(float &s1, float &c1, float &s2, float &c2, float t1, float e1, float t2,
                                           float e2) {
    two_sum_merge(s1, c1, t1, e1);
    two_sum_merge(s2, c2, t2, e2);
}

// CTA merge of the four running values; thread 0 ends with the totals.
__device__ __forceinline__ void stat_cta(float &s1, float &c1, float &s2, float &c2, StatPartial *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const float t1 = __shfl_xor_sync(0xffffffffu, s1, m), e1 = __shfl_xor_sync(0xffffffffu, c1, m);
        const float t2 = __shfl_xor_sync(0xffffffffu, s2, m), e2 = __shfl_xor_sync(0xffffffffu, c2, m);
        if (threadIdx.x & m) {  // lane-order independent: every lane gets the same bits
            float a1 = t1, b1 = e1, a2 = t2, b2 = e2;
            stat_merge(a1, b1, a2, b2, s1, c1, s2, c2);
            s1 = a1, c1 = b1, s2 = a2, c2 = b2;
        } else {
            stat_merge(s1, c1, s2, c2, t1, e1, t2, e2);
        }
    }
    if (lane == 0) sh[warp] = StatPartial{s1, c1, s2, c2};
    __syncthreads();
    if (warp == 0) {
        StatPartial p = lane < SD_THREADS / 32 ? sh[lane] : StatPartial{-0.f, 0.f, -0.f, 0.f};
        s1 = p.s1, c1 = p.c1, s2 = p.s2, c2 = p.c2;
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            const float t1 = __shfl_xor_sync(0xffffffffu, s1, m), e1 = __shfl_xor_sync(0xffffffffu, c1, m);
            const float t2 = __shfl_xor_sync(0xffffffffu, s2, m), e2 = __shfl_xor_sync(0xffffffffu, c2, m);
            if (threadIdx.x & m) {
                float a1 = t1, b1 = e1, a2 = t2, b2 = e2;
                stat_merge(a1, b1, a2, b2, s1, c1, s2, c2);
                s1 = a1, c1 = b1, s2 = a2, c2 = b2;
            } else {
                stat_merge(s1, c1, s2, c2, t1, e1, t2, e2);
            }
        }
    }
    __syncthreads();
}

struct StdArgs {
    const float *x;
    float *y;
    int64_t n;
    double *stats;          // device [mean, var] for the caller
    StatPartial *partials;  // [grid]
    unsigned *counter;      // pass-1 arrivals (zero on entry and exit)
    unsigned *flag;         // generation published by the last CTA
    StdShared *shared;      // statistics for pass 2
    int *err;
    unsigned gen;
    int fused;              // 1: wait for the statistics and run pass 2 here
};

__device__ __forceinline__ void neumaier2(float &s, float &c, float x) { neumaier(s, c, x); }

// x^2 added exactly: p = fl(x*x) through the compensated sum, and the product's
// rounding error e = x*x - p (exact by fused multiply-add) into the compensation.
__device__ __forceinline__ void add_square(float &s, float &c, float x) {
    const float p = __fmul_rn(x, x);
    const float e = __fmaf_rn(x, x, -p);
    neumaier(s, c, p);
    c = __fadd_rn(c, e);
}

__device__ __forceinline__ void publish_stats(const StdArgs &p, const StatPartial *part, int G, StatPartial *sh) {
    // last CTA: merge all CTA partials in double, in a fixed order
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < G; i += SD_THREADS) {
        const uint4 raw = __ldcg(reinterpret_cast<const uint4 *>(part + i));
        a += (double)__uint_as_float(raw.x) + (double)__uint_as_float(raw.y);
        b += (double)__uint_as_float(raw.z) + (double)__uint_as_float(raw.w);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, m);
        b += __shfl_xor_sync(0xffffffffu, b, m);
    }
    __shared__ double sa[SD_THREADS / 32], sb[SD_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < SD_THREADS / 32; ++w) {
            ta += sa[w];
            tb += sb[w];
        }
        const double nn = (double)p.n;
        const double mean = p.n > 0 ? ta / nn : 0.0;
        const double var = p.n > 0 ? tb / nn - mean * mean : 0.0;
        p.shared->mean = mean;
        p.shared->var = var;
        p.shared->mean_f = (float)mean;
        p.shared->rstd_f = var > 0.0 ? (float)(1.0 / sqrt(var)) : 0.0f;
        p.stats[0] = mean;
        p.stats[1] = var;
        *p.counter = 0u;
        __threadfence();
        st_release(p.flag, p.gen);
    }
    (void)sh;
}

// SU vectors in flight per thread; a group's loads all come before its
// stores (each element is read and written by the same thread, so the order
// is right even when y aliases x).  Both the separate elementwise launch and
// the fused launch's second pass keep four.
template <int SU>
__device__ __forceinline__ void map_pass(const float *x, float *y, int64_t n, float mean_f, float rstd_f) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const bool al = (((uintptr_t)x | (uintptr_t)y) & 15) == 0;
    if (al) {
        const int64_t nv = n / 4;
        const float4 *x4 = (const float4 *)x;
        float4 *y4 = (float4 *)y;
        int64_t v = gtid;
        for (; v + (SU - 1) * nth < nv; v += SU * nth) {
            float4 a[SU];
#pragma unroll
            for (int u = 0; u < SU; ++u) a[u] = x4[v + u * nth];
#pragma unroll
            for (int u = 0; u < SU; ++u) {
                a[u].x = __fmul_rn(__fsub_rn(a[u].x, mean_f), rstd_f);
                a[u].y = __fmul_rn(__fsub_rn(a[u].y, mean_f), rstd_f);
                a[u].z = __fmul_rn(__fsub_rn(a[u].z, mean_f), rstd_f);
                a[u].w = __fmul_rn(__fsub_rn(a[u].w, mean_f), rstd_f);
                y4[v + u * nth] = a[u];
            }
        }
        for (; v < nv; v += nth) {
            float4 a = x4[v];
            a.x = __fmul_rn(__fsub_rn(a.x, mean_f), rstd_f);
            a.y = __fmul_rn(__fsub_rn(a.y, mean_f), rstd_f);
            a.z = __fmul_rn(__fsub_rn(a.z, mean_f), rstd_f);
            a.w = __fmul_rn(__fsub_rn(a.w, mean_f), rstd_f);
            y4[v] = a;
        }
        for (int64_t i = 4 * nv + gtid; i < n; i += nth) y[i] = __fmul_rn(__fsub_rn(x[i], mean_f), rstd_f);
    } else {
        for (int64_t i = gtid; i < n; i += nth) y[i] = __fmul_rn(__fsub_rn(x[i], mean_f), rstd_f);
    }
}

__global__ void __launch_bounds__(SD_THREADS) standardize_kernel(const __grid_constant__ StdArgs p) {
    __shared__ StatPartial sh[SD_THREADS / 32];
    __shared__ int am_last;
    float s1 = -0.f, c1 = 0.f, s2 = -0.f, c2 = 0.f;
    const int64_t gtid = (int64_t)blockIdx.x * SD_THREADS + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * SD_THREADS;
    const bool al = ((uintptr_t)p.x & 15) == 0;
    if (al) {
        const int64_t nv = p.n / 4;
        const float4 *x4 = (const float4 *)p.x;
        for (int64_t v = gtid; v < nv; v += nth) {
            const float4 a = __ldg(x4 + v);
            neumaier2(s1, c1, a.x);
            add_square(s2, c2, a.x);
            neumaier2(s1, c1, a.y);
            add_square(s2, c2, a.y);
            neumaier2(s1, c1, a.z);
            add_square(s2, c2, a.z);
            neumaier2(s1, c1, a.w);
            add_square(s2, c2, a.w);
        }
        for (int64_t i = 4 * nv + gtid; i < p.n; i += nth) {
            const float a = p.x[i];
            neumaier2(s1, c1, a);
            add_square(s2, c2, a);
        }
    } else {
        for (int64_t i = gtid; i < p.n; i += nth) {
            const float a = p.x[i];
            neumaier2(s1, c1, a);
            add_square(s2, c2, a);
        }
    }
    stat_cta(s1, c1, s2, c2, sh);
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        p.partials[blockIdx.x] = StatPartial{s1, c1, s2, c2};
        __threadfence();
        am_last = atomicAdd(p.counter, 1u) == (unsigned)G - 1u;
    }
    __syncthreads();
    if (am_last) {
        __threadfence();
        publish_stats(p, p.partials, G, sh);
    }
    if (!p.fused) return;
    // every CTA waits (bounded) for the statistics, then runs the elementwise pass
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        uint32_t i = 0;
        int ok = 1;
        while (ld_acquire(p.flag) != p.gen) {
            if (++i > kSpinLimit) {
                ok = 0;
                atomicExch(p.err, 6);
                break;
            }
            if (i > 256) __nanosleep(64);  // the statistics usually arrive within a few hundred polls
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    __threadfence();
    const float mean_f = *(volatile float *)&p.shared->mean_f;
    const float rstd_f = *(volatile float *)&p.shared->rstd_f;
    map_pass<4>(p.x, p.y, p.n, mean_f, rstd_f);
}

__global__ void map_kernel(const float *x, float *y, int64_t n, const StdShared *st, float mean_f, float rstd_f,
                           int from_device) {
    if (from_device) {
        mean_f = st->mean_f;
        rstd_f = st->rstd_f;
    }
    map_pass<4>(x, y, n, mean_f, rstd_f);
}

// ============================================================================
// BFS pattern: level-synchronous search on a grid with a convergence flag
// ============================================================================

constexpr int BF_THREADS = 256;
constexpr int BFP_THREADS = 1024;  // the persistent form: one CTA per SM

__global__ void bfs_init_kernel(int32_t *dist, int64_t total, int64_t src, const uint8_t *open) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x)
        dist[c] = (c == src && open[c]) ? 0 : -1;
}

// One level, pull form: an unvisited open cell with a neighbour at level L
// joins level L + 1.  Returns whether this thread changed any cell.
// One level of the pull formulation over the thread's cells, CU cells at a
// time with every load of a group issued before any is tested: the level is
// bound by L2 latency, not bandwidth, at the sizes of the BFS workloads.
__device__ __forceinline__ bool bfs_level(const uint8_t *__restrict__ open, int32_t *dist, int64_t rows,
                                          int64_t cols, int32_t L) {
    constexpr int CU = 4;
    const int64_t total = rows * cols;  // < 2^31 (checked on the host): 32-bit cell arithmetic
    const uint32_t ucols = (uint32_t)cols, urows = (uint32_t)rows;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    bool changed = false;
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c0 < total; c0 += CU * nth) {
        int32_t d[CU];
        bool need[CU];
#pragma unroll
        for (int j = 0; j < CU; ++j) {
            const int64_t c = c0 + j * nth;
            d[j] = c < total ? __ldcg(dist + c) : 0;
            need[j] = c < total && __ldg(open + c) != 0;
        }
        int32_t nb[CU][4];
#pragma unroll
        for (int j = 0; j < CU; ++j) {  // an unvisited open cell reads its four neighbours
            const uint32_t c = (uint32_t)(c0 + j * nth);
            const bool go = need[j] && d[j] == -1;
            const uint32_t r = c / ucols, q = c - r * ucols;
            nb[j][0] = go && r > 0 ? __ldcg(dist + c - ucols) : -2;
            nb[j][1] = go && r + 1 < urows ? __ldcg(dist + c + ucols) : -2;
            nb[j][2] = go && q > 0 ? __ldcg(dist + c - 1) : -2;
            nb[j][3] = go && q + 1 < ucols ? __ldcg(dist + c + 1) : -2;
        }
#pragma unroll
        for (int j = 0; j < CU; ++j) {
            if (nb[j][0] == L || nb[j][1] == L || nb[j][2] == L || nb[j][3] == L) {
                dist[c0 + j * nth] = L + 1;
                changed = true;
            }
        }
    }
    return changed;
}

// mode 0: `||` reduction of the flag (warp vote, CTA vote, last-CTA merge)
// mode 1: guarded write (the flag was cleared; threads only write 1)
__global__ void __launch_bounds__(BF_THREADS) bfs_level_kernel(const uint8_t *__restrict__ open, int32_t *dist,
                                                               int64_t rows, int64_t cols, int32_t L, int mode,
                                                               unsigned *more, unsigned *partial, unsigned *counter) {
    const bool changed = bfs_level(open, dist, rows, cols, L);
    if (mode == 1) {
        if (changed) *more = 1u;
        return;
    }
    const int any = __syncthreads_or(changed ? 1 : 0);
    __shared__ int am_last;
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = (unsigned)any;
        __threadfence();
        am_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    int v = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += BF_THREADS) v |= (int)__ldcg(partial + b);
    v = __syncthreads_or(v);
    if (threadIdx.x == 0) {
        *more = (unsigned)(v != 0);
        *counter = 0u;
    }
}

// All levels in one cooperative launch: per level, the || of the changed
// flags goes to a per-level slot, a bounded grid barrier separates levels.
// One CTA of BFP_THREADS per SM (fewer arrivals per grid barrier) and one
// barrier per level, which also carries the level's `||` flag: every CTA
// learns whether any cell changed from the barrier's release itself.
__global__ void __launch_bounds__(BFP_THREADS, 1) bfs_persistent_kernel(const uint8_t *__restrict__ open, int32_t *dist,
                                                                       int64_t rows, int64_t cols,
                                                                       int64_t max_levels, unsigned *bar,
                                                                       int64_t *levels_out, int *err) {
    unsigned gen = (*(volatile unsigned *)&bar[1]) >> 1;
    int64_t L = 0;
    for (; L < max_levels; ++L) {
        const bool changed = bfs_level(open, dist, rows, cols, (int32_t)L);
        const int any = __syncthreads_or(changed ? 1 : 0);
        const int r = grid_barrier_or(bar, gen, any != 0);
        if (r == 0) {
            if (threadIdx.x == 0) atomicExch(err, 7);
            return;
        }
        if (r == 1) break;  // no cell changed at this level
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *levels_out = L + 1;  // the level that found nothing new
}

}  // namespace accr

using namespace accr;

// ---- Nearest Neighbor ------------------------------------------------------------

extern "C" ACCR_API int accr_nearest_k(const float *pts, int64_t n, float qx, float qy, int32_t k,
                                       int64_t *idx_out, float *d2_out, uint32_t flags, accr_stream_t stream) {
    ACCR_TRACE("accr_nearest_k");
    clear_error();
    if (n < 0 || k < 1 || k > 16) return set_error(ACCR_EINVAL, "accr_nearest_k: need n >= 0 and 1 <= k <= 16");
    if (flags & ~ACCR_SYNC) return set_error(ACCR_EINVAL, "accr_nearest_k: unsupported flags 0x%x", flags);
    if ((n > 0 && !pts) || !idx_out || !d2_out) return set_error(ACCR_EINVAL, "accr_nearest_k: NULL pointer");
    if (((uintptr_t)pts & 7) || ((uintptr_t)idx_out & 7) || ((uintptr_t)d2_out & 3))
        return set_error(ACCR_EINVAL, "accr_nearest_k: misaligned pointer (points need 8 bytes)");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = k <= 8 ? nearest_launch<8>(pts, n, qx, qy, k, idx_out, d2_out, s)
                    : nearest_launch<16>(pts, n, qx, qy, k, idx_out, d2_out, s);
    if (rc != ACCR_OK) return rc;
    if (flags & ACCR_SYNC) return cuda_check(cudaStreamSynchronize(s), "accr_nearest_k: sync");
    return ACCR_OK;
}

// ---- SRAD pattern -------------------------------------------------------------------

struct StdState {
    std::mutex mu;
    unsigned gen = 0;
};
static StdState g_std;

extern "C" ACCR_API int accr_standardize(const float *x, int64_t n, float *y, double *stats, uint32_t flags,
                                         accr_stream_t stream) {
    ACCR_TRACE("accr_standardize");
    clear_error();
    if (n < 0 || (n > 0 && (!x || !y)) || !stats) return set_error(ACCR_EINVAL, "accr_standardize: bad arguments");
    if (((uintptr_t)x & 3) || ((uintptr_t)y & 3) || ((uintptr_t)stats & 7))
        return set_error(ACCR_EINVAL, "accr_standardize: misaligned pointer");
    if (flags & ~(ACCR_SYNC | ACCR_UNFUSED | ACCR_TWO_LEVEL_HOST))
        return set_error(ACCR_EINVAL, "accr_standardize: unsupported flags 0x%x", flags);
    cudaStream_t s = (cudaStream_t)stream;
    const DeviceInfo &di = device_info();
    static int per_sm = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, standardize_kernel, SD_THREADS, 0);
        if (per_sm < 1) per_sm = 1;
    });
    const int64_t want = (n / 4 + SD_THREADS * 4 - 1) / (SD_THREADS * 4);
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)per_sm * di.sms);
    // scratch: [counters][partials][shared stats][status]
    Scratch *scr = scratch_for(stream, sizeof(StatPartial) * (size_t)grid + 256);
    if (!scr) return ACCR_ENOMEM;
    StdArgs a;
    memset(&a, 0, sizeof a);
    a.x = x;
    a.y = y;
    a.n = n;
    a.stats = stats;
    a.partials = (StatPartial *)((char *)scr->buf + 256);
    a.counter = scr->counters + 2;
    a.flag = scr->counters + 3;
    a.shared = (StdShared *)scr->buf;
    a.err = (int *)(scr->counters + 4);
    {
        std::lock_guard<std::mutex> lk(g_std.mu);
        a.gen = ++g_std.gen;
        if (a.gen == 0) a.gen = ++g_std.gen;
    }
    int rc = cuda_check(cudaMemsetAsync(a.err, 0, sizeof(int), s), "accr_standardize: clear status");
    if (rc != ACCR_OK) return rc;
    if ((rc = launch_guard("standardize_kernel")) != ACCR_OK) return rc;
    if (flags & ACCR_TWO_LEVEL_HOST) {
        // the paper's form: CTA partials to the host, merged there, then the
        // elementwise region with the statistics as launch arguments
        a.fused = 0;
        standardize_kernel<<<grid, SD_THREADS, 0, s>>>(a);
        if ((rc = launched("standardize_kernel")) != ACCR_OK) return rc;
        StatPartial *h = (StatPartial *)host_staging_for(stream, sizeof(StatPartial) * (size_t)grid);
        if (!h) return ACCR_ENOMEM;
        rc = cuda_check(cudaMemcpyAsync(h, a.partials, sizeof(StatPartial) * (size_t)grid, cudaMemcpyDeviceToHost, s),
                        "accr_standardize: partials");
        if (rc == ACCR_OK) rc = cuda_check(cudaStreamSynchronize(s), "accr_standardize: sync");
        if (rc != ACCR_OK) return rc;
        double ta = 0.0, tb = 0.0;
        for (int i = 0; i < grid; ++i) {
            ta += (double)h[i].s1 + (double)h[i].c1;
            tb += (double)h[i].s2 + (double)h[i].c2;
        }
        const double mean = n > 0 ? ta / (double)n : 0.0, var = n > 0 ? tb / (double)n - mean * mean : 0.0;
        const float mean_f = (float)mean, rstd_f = var > 0.0 ? (float)(1.0 / sqrt(var)) : 0.0f;
        map_kernel<<<di.sms * 4, 512, 0, s>>>(x, y, n, nullptr, mean_f, rstd_f, 0);
        if ((rc = launched("map_kernel")) != ACCR_OK) return rc;
        const double st[2] = {mean, var};
        rc = cuda_check(cudaMemcpyAsync(stats, st, sizeof st, cudaMemcpyHostToDevice, s), "accr_standardize: stats");
        if (rc == ACCR_OK) rc = cuda_check(cudaStreamSynchronize(s), "accr_standardize: sync");
        return rc;
    }
    if (flags & ACCR_UNFUSED) {
        // two launches, the statistics stay on the device
        a.fused = 0;
        standardize_kernel<<<grid, SD_THREADS, 0, s>>>(a);
        if ((rc = launched("standardize_kernel")) != ACCR_OK) return rc;
        map_kernel<<<di.sms * 4, 512, 0, s>>>(x, y, n, a.shared, 0.f, 0.f, 1);
        if ((rc = launched("map_kernel")) != ACCR_OK) return rc;
    } else {
        // one cooperative launch: co-residency of every CTA is guaranteed, so
        // the wait for the statistics cannot starve the CTA that publishes them
        a.fused = 1;
        void *args[] = {&a};
        rc = cuda_check(cudaLaunchCooperativeKernel((const void *)standardize_kernel, grid, SD_THREADS, args, 0, s),
                        "accr_standardize: cooperative launch");
        if (rc != ACCR_OK) return rc;
        if ((rc = launched("standardize_kernel (fused)")) != ACCR_OK) return rc;
    }
    if (flags & ACCR_SYNC) {
        int h = 0;
        rc = cuda_check(cudaMemcpyAsync(&h, a.err, sizeof(int), cudaMemcpyDeviceToHost, s), "accr_standardize: status");
        if (rc == ACCR_OK) rc = cuda_check(cudaStreamSynchronize(s), "accr_standardize: sync");
        if (rc == ACCR_OK && h != 0) return set_error(ACCR_ETIMEDOUT, "accr_standardize: grid wait ran out");
    }
    return rc;
}

// ---- BFS pattern -------------------------------------------------------------------

extern "C" ACCR_API int accr_grid_bfs(const uint8_t *open, int64_t rows, int64_t cols, int64_t src, int32_t *dist,
                                      int32_t mode, int64_t *levels, accr_stream_t stream) {
    ACCR_TRACE("accr_grid_bfs");
    clear_error();
    if (rows < 0 || cols < 0 || (rows * cols > 0 && (!open || !dist)) || !levels)
        return set_error(ACCR_EINVAL, "accr_grid_bfs: bad arguments");
    if (rows * cols >= ((int64_t)1 << 31)) return set_error(ACCR_EINVAL, "accr_grid_bfs: grid too large");
    if (mode < ACCR_BFS_REDUCE || mode > ACCR_BFS_PERSISTENT) return set_error(ACCR_EINVAL, "accr_grid_bfs: bad mode");
    *levels = 0;
    const int64_t total = rows * cols;
    if (total == 0) return ACCR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const DeviceInfo &di = device_info();
    int rc;
    if ((rc = launch_guard("bfs_init_kernel")) != ACCR_OK) return rc;
    bfs_init_kernel<<<di.sms * 4, 256, 0, s>>>(dist, total, (src >= 0 && src < total) ? src : -1, open);
    if ((rc = launched("bfs_init_kernel")) != ACCR_OK) return rc;
    if (src < 0 || src >= total) return cuda_check(cudaStreamSynchronize(s), "accr_grid_bfs: sync");
    {  // a closed source cell reaches nothing: zero levels
        uint8_t o = 0;
        rc = cuda_check(cudaMemcpyAsync(&o, open + src, 1, cudaMemcpyDeviceToHost, s), "accr_grid_bfs: source");
        if (rc == ACCR_OK) rc = cuda_check(cudaStreamSynchronize(s), "accr_grid_bfs: sync");
        if (rc != ACCR_OK) return rc;
        if (!o) return ACCR_OK;
    }
    static int per_sm = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_level_kernel, BF_THREADS, 0);
        if (per_sm < 1) per_sm = 1;
    });
    const int64_t want = (total + BF_THREADS - 1) / BF_THREADS;
    const int grid = (int)std::min<int64_t>(want, (int64_t)per_sm * di.sms);
    Scratch *scr = scratch_for(stream, sizeof(unsigned) * (size_t)grid + 512);
    if (!scr) return ACCR_ENOMEM;
    unsigned *more = scr->counters + 8;
    unsigned *counter = scr->counters + 9;
    unsigned *bar = scr->counters + 12;      // arrivals, generation
    int *err = (int *)(scr->counters + 14);
    int64_t *lv = (int64_t *)((char *)scr->buf);
    unsigned *partial = (unsigned *)((char *)scr->buf + 64);
    unsigned *hmore = (unsigned *)host_staging_for(stream, 64);
    if (!hmore) return ACCR_ENOMEM;
    if (mode == ACCR_BFS_PERSISTENT) {
        rc = cuda_check(cudaMemsetAsync(err, 0, sizeof(int), s), "accr_grid_bfs: clear status");
        if (rc == ACCR_OK) rc = cuda_check(cudaMemsetAsync(bar, 0, sizeof(unsigned), s), "accr_grid_bfs: barrier");
        if (rc != ACCR_OK) return rc;
        int64_t maxl = total + 1;
        void *args[] = {(void *)&open, (void *)&dist, (void *)&rows, (void *)&cols, (void *)&maxl,
                        (void *)&bar, (void *)&lv, (void *)&err};
        if ((rc = launch_guard("bfs_persistent_kernel")) != ACCR_OK) return rc;
        const int pgrid = (int)std::min<int64_t>((total + BFP_THREADS - 1) / BFP_THREADS, (int64_t)di.sms);
        rc = cuda_check(cudaLaunchCooperativeKernel((const void *)bfs_persistent_kernel, pgrid, BFP_THREADS, args, 0, s),
                        "accr_grid_bfs: cooperative launch");
        if (rc != ACCR_OK) return rc;
        if ((rc = launched("bfs_persistent_kernel")) != ACCR_OK) return rc;
        int64_t hl[2] = {0, 0};
        rc = cuda_check(cudaMemcpyAsync(hl, lv, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "accr_grid_bfs: levels");
        int herr = 0;
        if (rc == ACCR_OK)
            rc = cuda_check(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s), "accr_grid_bfs: status");
        if (rc == ACCR_OK) rc = cuda_check(cudaStreamSynchronize(s), "accr_grid_bfs: sync");
        if (rc != ACCR_OK) return rc;
        if (herr) return set_error(ACCR_ETIMEDOUT, "accr_grid_bfs: grid barrier wait ran out");
        *levels = hl[0];
        return ACCR_OK;
    }
    // host-driven levels: one launch per level, the flag read back after each
    for (int64_t L = 0; L <= total; ++L) {
        if (mode == ACCR_BFS_GUARDED) {
            rc = cuda_check(cudaMemsetAsync(more, 0, sizeof(unsigned), s), "accr_grid_bfs: clear flag");
            if (rc != ACCR_OK) return rc;
        }
        if ((rc = launch_guard("bfs_level_kernel")) != ACCR_OK) return rc;
        bfs_level_kernel<<<grid, BF_THREADS, 0, s>>>(open, dist, rows, cols, (int32_t)L,
                                                     mode == ACCR_BFS_GUARDED ? 1 : 0, more, partial, counter);
        if ((rc = launched("bfs_level_kernel")) != ACCR_OK) return rc;
        rc = cuda_check(cudaMemcpyAsync(hmore, more, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "accr_grid_bfs: flag");
        if (rc == ACCR_OK) rc = cuda_check(cudaStreamSynchronize(s), "accr_grid_bfs: sync");
        if (rc != ACCR_OK) return rc;
        if (!*hmore) {
            *levels = L + 1;
            return ACCR_OK;
        }
    }
    *levels = total + 1;
    return ACCR_OK;
}
