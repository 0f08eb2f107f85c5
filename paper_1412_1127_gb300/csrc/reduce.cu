// reduce.cu -- one region: a `loop independent` loop over [0, n) with up to
// four reduction clauses, in one pass over the data (IPMACC Stage 3.4 items
// i-iii and the cross-block merge of Stage 3.7).
//
// Work sharing: gang -> CTA of a persistent grid sized to the SM count,
// worker -> warp, vector -> lane.  Each thread streams 16-byte vectors with
// non-allocating loads (RU vectors in flight per iteration, coalesced across
// the CTA), folding them into private accumulators.  Warps merge through
// shuffles, the CTA through shared memory, and each CTA writes one partial per
// clause.  The last CTA to finish (a counter in library scratch) merges the
// partials in a fixed order and writes the variables, so there is no second
// launch and no host round trip.  The paper's own form (block partials merged
// on the CPU, Sec. 4.2 on SRAD) is kept behind ACCR_TWO_LEVEL_HOST.
#include <string.h>

#include <atomic>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "fold.cuh"

namespace accr {

constexpr int RB = 512;          // threads per CTA
// 16-byte vectors per thread per iteration: picked by the autotuner
// ("vectors" in tuning.json), passed in by the build.
#ifndef ACCR_REDUCE_RU
#define ACCR_REDUCE_RU 4
#endif
constexpr int RU = ACCR_REDUCE_RU;
constexpr int kMaxGrid = 4096;   // bound on CTAs (and partials per clause)

struct ReduceArgs {
    const void *in;
    int64_t n;
    int nc;
    int two_level;               // 1: stop after writing the partials
    ClauseDev cl[ACCR_MAX_CLAUSES];
    Partial *partials;           // [nc][gridDim.x]
    unsigned *counter;           // zero on entry; zero again on exit
};

// 16-byte streaming load: read-only path, no L1 allocation, 256-byte L2 fetch.
__device__ __forceinline__ uint4 ld_stream(const uint4 *p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

__device__ __forceinline__ Partial ld_partial(const Partial *p) {
    uint4 v = __ldcg(reinterpret_cast<const uint4 *>(p));
    Partial q;
    q.a = ((uint64_t)v.y << 32) | v.x;
    q.c = __uint_as_float(v.z);
    q.pad = 0;
    return q;
}

// W0 / W1 >= 0 fix the working codes of clauses 0 / 1 at compile time (the
// operator switches fold away and the kernel's code shrinks to what the two
// operators need); -1 reads them from the arguments.
template <typename T, int NC, int W0 = -1, int W1 = -1>
__global__ void __launch_bounds__(RB, 2) reduce_kernel(const __grid_constant__ ReduceArgs p) {
    constexpr bool E64 = sizeof(T) == 8;
    constexpr int EPV = 16 / (int)sizeof(T);
    __shared__ Acc sh[NC][RB / 32];
    __shared__ int am_last;

    const T *in = (const T *)p.in;
    const int64_t n = p.n;
    const int64_t mis = (int64_t)(((16 - ((uintptr_t)in & 15)) & 15) / sizeof(T));
    const int64_t head = mis < n ? mis : n;          // elements before 16-B alignment
    const uint4 *vin = (const uint4 *)(in + head);
    const int64_t nvec = (n - head) / EPV;
    const int64_t tail0 = head + nvec * EPV;          // ragged tail start

    int w[NC];
    uint64_t ident[NC];
    Acc A[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        w[c] = (c == 0 && W0 >= 0) ? W0 : (c == 1 && W1 >= 0) ? W1 : p.cl[c].wcode;
        ident[c] = p.cl[c].ident;
        A[c].a = ident[c];
        A[c].c = 0.f;
    }

    const int64_t gtid = (int64_t)blockIdx.x * RB + threadIdx.x;
    if (gtid < head) {
        T x = in[gtid];
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_one<T>(w[c], A[c], x);
    }
    if (tail0 + gtid < n) {
        T x = in[tail0 + gtid];
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_one<T>(w[c], A[c], x);
    }

    int64_t v = (int64_t)blockIdx.x * (RB * RU) + threadIdx.x;
    const int64_t step = (int64_t)gridDim.x * (RB * RU);
    for (; v + (RU - 1) * RB < nvec; v += step) {
        uint4 b[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) b[u] = ld_stream(vin + v + u * RB);
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_vec<T, RU>(w[c], A[c], b);
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
        const int64_t vv = v + u * RB;
        if (vv < nvec) {
            uint4 b = ld_stream(vin + vv);
#pragma unroll
            for (int c = 0; c < NC; ++c) fold_vec<T, 1>(w[c], A[c], &b);
        }
    }

    cta_merge<NC, RB>(w, ident, E64, A, sh);
    const int G = gridDim.x;
    if (G == 1 && !p.two_level) {
        // one CTA: its merge is the region's (the same operations the last-CTA
        // merge below applies to a single partial: the final code's identity,
        // then the partial)
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                Acc F;
                F.a = final_ident(p.cl[c]);
                F.c = 0.f;
                merge(final_code(w[c]), E64, F, to_final(w[c], A[c]));
                store_var(p.cl[c], 0, finish(p.cl[c], E64, n == 0, F));
            }
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
            p.partials[c * G + blockIdx.x] = q;
        }
    }
    if (p.two_level) return;

    // single-pass cross-gang merge: the last CTA to arrive merges all partials.
    // The count is an acquire-release atomic at device scope: it publishes this
    // CTA's partials (release) and, for the last CTA, makes every other CTA's
    // partials visible to its thread 0 (acquire), and through the barrier to
    // the whole CTA -- no separate fences.
    if (threadIdx.x == 0) {
        unsigned t;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(t) : "l"(p.counter) : "memory");
        am_last = (t == (unsigned)G - 1u);
    }
    __syncthreads();
    if (!am_last) return;

    int fw[NC];
    uint64_t fid[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        fw[c] = final_code(w[c]);
        fid[c] = final_ident(p.cl[c]);
        A[c].a = fid[c];
        A[c].c = 0.f;
        for (int b = threadIdx.x; b < G; b += RB) {
            Partial q = ld_partial(&p.partials[c * G + b]);
            Acc Q;
            Q.a = q.a;
            Q.c = q.c;
            merge(fw[c], E64, A[c], to_final(w[c], Q));
        }
    }
    cta_merge<NC, RB>(fw, fid, E64, A, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) store_var(p.cl[c], 0, finish(p.cl[c], E64, n == 0, A[c]));
        *p.counter = 0u;
    }
}

// ---- host side -------------------------------------------------------------------

// Resident-grid size per device, computed once (a racing first computation
// stores the same value twice); read without a lock.
template <typename T, int NC>
static int occupancy_grid() {
    static std::atomic<int> cached[64];
    const DeviceInfo &d = device_info();
    std::atomic<int> &slot = cached[d.id & 63];
    int g = slot.load(std::memory_order_relaxed);
    if (!g) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reduce_kernel<T, NC>, RB, 0);
        if (per_sm < 1) per_sm = 1;
        g = per_sm * d.sms;
        if (g > kMaxGrid) g = kMaxGrid;
        slot.store(g, std::memory_order_relaxed);
    }
    return g;
}

template <typename T, int NC, int W0 = -1, int W1 = -1>
static int launch_t(ReduceArgs &a, int grid, cudaStream_t s) {
    int rc = launch_guard("reduce_kernel");
    if (rc != ACCR_OK) return rc;
    reduce_kernel<T, NC, W0, W1><<<grid, RB, 0, s>>>(a);
    return launched("reduce_kernel");
}

// A sum together with a max or a min -- the two-clause region of the paper's
// examples, reduction(+:s) reduction(max:m) -- runs a kernel with both codes
// fixed: the generic two-clause kernel carries every operator's code twice
// over, and on small regions its instruction fetch costs more than the data.
// The clause order is canonical (sum first) here: each clause descriptor
// carries its own output, and the kernel merges its own partials.  The grid
// stays the generic kernel's, so results do not depend on which one runs.
template <typename T, int W0, int W1>
static bool pair_t(ReduceArgs &a, int grid, cudaStream_t s, int &rc) {
    if (a.cl[0].wcode != W0 || a.cl[1].wcode != W1) return false;
    rc = launch_t<T, 2, W0, W1>(a, grid, s);
    return true;
}

template <typename T>
static bool launch_pair(ReduceArgs &a, int grid, cudaStream_t s, int &rc) {
    auto is_sum = [](int w) { return w == W_ADD32 || w == W_ADD64 || w == W_ADDF || w == W_ADDF_COMP || w == W_ADDF_WIDE; };
    if (!is_sum(a.cl[0].wcode) && is_sum(a.cl[1].wcode)) {
        const ClauseDev t = a.cl[0];
        a.cl[0] = a.cl[1];
        a.cl[1] = t;
    }
    if constexpr (std::is_same<T, int32_t>::value) {
        return pair_t<T, W_ADD32, W_MAXI>(a, grid, s, rc) || pair_t<T, W_ADD32, W_MINI>(a, grid, s, rc) ||
               pair_t<T, W_ADD64, W_MAXI>(a, grid, s, rc) || pair_t<T, W_ADD64, W_MINI>(a, grid, s, rc);
    } else if constexpr (std::is_same<T, int64_t>::value) {
        return pair_t<T, W_ADD64, W_MAXI>(a, grid, s, rc) || pair_t<T, W_ADD64, W_MINI>(a, grid, s, rc);
    } else if constexpr (std::is_same<T, float>::value) {
        return pair_t<T, W_ADDF, W_MAXF>(a, grid, s, rc) || pair_t<T, W_ADDF, W_MINF>(a, grid, s, rc) ||
               pair_t<T, W_ADDF_COMP, W_MAXF>(a, grid, s, rc) || pair_t<T, W_ADDF_COMP, W_MINF>(a, grid, s, rc) ||
               pair_t<T, W_ADDF_WIDE, W_MAXF>(a, grid, s, rc) || pair_t<T, W_ADDF_WIDE, W_MINF>(a, grid, s, rc);
    } else {
        return pair_t<T, W_ADDF, W_MAXF>(a, grid, s, rc) || pair_t<T, W_ADDF, W_MINF>(a, grid, s, rc);
    }
}

template <typename T>
static int launch_nc(ReduceArgs &a, int grid, cudaStream_t s) {
    int rc = ACCR_OK;
    // the two-level form merges the partials on the host in the caller's clause order
    if (a.nc == 2 && !a.two_level && launch_pair<T>(a, grid, s, rc)) return rc;
    switch (a.nc) {
    case 1: return launch_t<T, 1>(a, grid, s);
    case 2: return launch_t<T, 2>(a, grid, s);
    case 3: return launch_t<T, 3>(a, grid, s);
    default: return launch_t<T, 4>(a, grid, s);
    }
}

template <typename T>
static int grid_for(int nc, int64_t n) {
    int maxg;
    switch (nc) {
    case 1: maxg = occupancy_grid<T, 1>(); break;
    case 2: maxg = occupancy_grid<T, 2>(); break;
    case 3: maxg = occupancy_grid<T, 3>(); break;
    default: maxg = occupancy_grid<T, 4>(); break;
    }
    const int64_t nvec = n * (int64_t)sizeof(T) / 16;
    int64_t want = (nvec + (int64_t)RB * RU - 1) / ((int64_t)RB * RU);
    if (want < 1) want = 1;
    return (int)(want < maxg ? want : maxg);
}

// Grid used for (type, nclauses, n): depends only on these and the device, so
// floating-point results are reproducible run to run.
int reduce_grid(int in_type, int nc, int64_t n) {
    switch (in_type) {
    case ACCR_I32: return grid_for<int32_t>(nc, n);
    case ACCR_I64: return grid_for<int64_t>(nc, n);
    case ACCR_F32: return grid_for<float>(nc, n);
    default: return grid_for<double>(nc, n);
    }
}

// Issues the kernel for a region whose clauses are already lowered.
int reduce_launch(const void *in, int64_t n, int in_type, const ClauseDev *cl, int nc, int two_level,
                  Partial *partials, unsigned *counter, int grid, cudaStream_t s) {
    ReduceArgs a;
    memset(&a, 0, sizeof a);
    a.in = in;
    a.n = n;
    a.nc = nc;
    a.two_level = two_level;
    for (int c = 0; c < nc; ++c) a.cl[c] = cl[c];
    a.partials = partials;
    a.counter = counter;
    switch (in_type) {
    case ACCR_I32: return launch_nc<int32_t>(a, grid, s);
    case ACCR_I64: return launch_nc<int64_t>(a, grid, s);
    case ACCR_F32: return launch_nc<float>(a, grid, s);
    default: return launch_nc<double>(a, grid, s);
    }
}

// The paper's second level on the CPU: merge the block partials in block
// order and meet the variable's prior value (Sec. 4.2, SRAD).
static void host_merge(const ClauseDev *cl, int nc, bool e64, bool n_zero, const Partial *part,
                       int grid) {
    for (int c = 0; c < nc; ++c) {
        const int fw = final_code(cl[c].wcode);
        Acc F;
        F.a = final_ident(cl[c]);
        F.c = 0.f;
        for (int b = 0; b < grid; ++b) {
            Acc Q;
            Q.a = part[c * grid + b].a;
            Q.c = part[c * grid + b].c;
            merge(fw, e64, F, to_final(cl[c].wcode, Q));
        }
        const uint64_t bits = finish(cl[c], e64, n_zero, F);
        if (cl[c].acc_type == ACCR_I32 || cl[c].acc_type == ACCR_F32) {
            uint32_t v = (uint32_t)bits;
            memcpy(cl[c].out, &v, 4);
        } else {
            memcpy(cl[c].out, &bits, 8);
        }
    }
}

}  // namespace accr

using namespace accr;

extern "C" ACCR_API int accr_reduce(const void *in, int64_t n, int32_t in_type, const accr_clause *clauses,
                           int32_t nclauses, uint32_t flags, accr_stream_t stream) {
    ACCR_TRACE("accr_reduce");
    clear_error();
    if (flags & ~(ACCR_COMPENSATED | ACCR_SYNC | ACCR_TWO_LEVEL_HOST))
        return set_error(ACCR_EINVAL, "accr_reduce: unknown flags 0x%x", flags);
    if (n < 0) return set_error(ACCR_EINVAL, "accr_reduce: n = %lld < 0", (long long)n);
    ClauseDev cl[ACCR_MAX_CLAUSES];
    int rc = lower_clauses(in_type, clauses, nclauses, flags, cl);
    if (rc != ACCR_OK) return rc;
    if (n > 0 && !in) return set_error(ACCR_EINVAL, "accr_reduce: in is NULL");
    if (((uintptr_t)in % (uintptr_t)type_bytes(in_type)) != 0)
        return set_error(ACCR_EINVAL, "accr_reduce: in is not aligned to its element size");
    const int grid = reduce_grid(in_type, nclauses, n);
    const size_t pbytes = (size_t)nclauses * (size_t)grid * sizeof(Partial);
    log_msg(2, "accr_reduce: n=%lld type=%d clauses=%d grid=%d%s", (long long)n, in_type, nclauses, grid,
            (flags & ACCR_TWO_LEVEL_HOST) ? " (two-level host merge)" : "");
    Scratch *scr = scratch_for(stream, pbytes);
    if (!scr) return ACCR_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    const bool two = (flags & ACCR_TWO_LEVEL_HOST) != 0;
    rc = reduce_launch(in, n, in_type, cl, nclauses, two ? 1 : 0, (Partial *)scr->buf, scr->counters, grid, s);
    if (rc != ACCR_OK) return rc;
    if (two) {
        // block partials to the host, merged there (the paper's two levels)
        void *h = host_staging_for(stream, pbytes);
        if (!h) return ACCR_ENOMEM;
        rc = cuda_check(cudaMemcpyAsync(h, scr->buf, pbytes, cudaMemcpyDeviceToHost, s), "accr_reduce: D2H partials");
        if (rc != ACCR_OK) return rc;
        rc = cuda_check(cudaStreamSynchronize(s), "accr_reduce: sync");
        if (rc != ACCR_OK) return rc;
        host_merge(cl, nclauses, type_bytes(in_type) == 8, n == 0, (const Partial *)h, grid);
        return ACCR_OK;
    }
    if (flags & ACCR_SYNC) return cuda_check(cudaStreamSynchronize(s), "accr_reduce: sync");
    return ACCR_OK;
}
