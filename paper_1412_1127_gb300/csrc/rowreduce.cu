// rowreduce.cu -- the nest `for i (gang) { for j (vector) var_i (op)= A[i][j] }`:
// one reduction variable per row of a row-major matrix (the two-level loop
// shape of Listing 1a with an inner reduction; IPMACC Sec. 1.3, Stage 3.4).
//
// Mapping: gang -> CTA, worker -> warp, vector -> lane.  A warp folds one
// stretch of a row at a time: lanes stream it in 16-byte vectors (RU2 in
// flight per lane) and merge through shuffles.  Stretches whose start is not
// 16-byte aligned (ld not a multiple of the vector) fold their head and tail
// element by element.  Two forms, chosen by the row's length alone, so a
// row's result never depends on how many rows the matrix has:
//
//   * rows shorter than SPLIT_ROW_BYTES: the stretch is the whole row and
//     lane 0 writes the row's variable; no cross-warp merge at all.
//   * longer rows: the stretch is one of the row's SPLIT_CHUNK_BYTES chunks
//     (a few long rows then spread over every SM instead of a few warps).
//     The launch has one 1024-thread CTA per SM (256-thread CTAs, as many as
//     fit, where the fold needs more registers), and CTA b
//     takes the contiguous run [total b / G, total (b + 1) / G) of the
//     rows x cpr chunks, so every SM streams the same number of chunks to
//     within one; its 32 warps take the run's chunks in turn, so the warps
//     left with a last chunk are many and keep the SM's loads in flight.
//     Lane 0 stores each chunk's partial in the chunk's own slot; the CTA
//     then counts its chunks into each row it touched, and the CTA whose
//     count completes a row merges the row's partials in chunk order (thread
//     t takes chunks t, t + 1024 (or 256), ..., loads in flight, then the CTA's
//     shuffle and shared-memory tree) and writes the variable.  The partial
//     slots and the merge order depend on the row length and the clauses
//     only, not on which warp folded which chunk.
#include <string.h>

#include <atomic>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "debug.cuh"
#include "fold.cuh"

namespace accr {


constexpr int WB = 256;  // threads per CTA of the warp-per-row form (8 rows in flight)
// Threads per CTA of the split form: 1024 (one CTA per SM) where the fold
// fits 64 registers (4-byte elements, one or two clauses), else 256 (as many
// CTAs per SM as the registers allow).
template <typename T, int NC, bool SPLIT>
constexpr int row_threads() {
    return !SPLIT ? WB : (sizeof(T) == 4 && NC <= 2) ? 1024 : 256;
}
// 16-byte vectors per lane per iteration: picked by the autotuner ("vectors"
// in tuning.json), passed in by the build.
#ifndef ACCR_ROW_RU
#define ACCR_ROW_RU 8
#endif
constexpr int RU2 = ACCR_ROW_RU;
constexpr int64_t SPLIT_ROW_BYTES = 256 * 1024;
constexpr int64_t SPLIT_CHUNK_BYTES = 32 * 1024;

struct RowArgs {
    const void *A;
    int64_t rows, cols, ld;
    int nc;
    ClauseDev cl[ACCR_MAX_CLAUSES];
    int64_t chunk;        // split form: elements per chunk
    int64_t cpr;          // split form: chunks per row
    Partial *partials;    // split form: [rows][nc][cpr]
    unsigned *counters;   // split form: [rows], zero on entry, zero again on exit (zeroed_words_for)
};

__device__ __forceinline__ Partial ld_row_partial(const Partial *p) {
    uint4 v = __ldcg(reinterpret_cast<const uint4 *>(p));
    Partial q;
    q.a = ((uint64_t)v.y << 32) | v.x;
    q.c = __uint_as_float(v.z);
    q.pad = 0;
    return q;
}

__device__ __forceinline__ uint4 ld_row(const uint4 *p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

// One stretch of a row (elements [lo, lo + len) of row r), folded by one
// warp and merged across its lanes.
template <typename T, int NC>
__device__ __forceinline__ void fold_stretch(const RowArgs &p, const int (&w)[NC], int64_t r, int64_t lo, int64_t len,
                                             int lane, Acc (&A)[NC]) {
    constexpr bool E64 = sizeof(T) == 8;
    constexpr int EPV = 16 / (int)sizeof(T);
    const T *row = (const T *)p.A + r * p.ld + lo;
    const int64_t mis = (int64_t)(((16 - ((uintptr_t)row & 15)) & 15) / sizeof(T));
    const int64_t head = mis < len ? mis : len;
    const uint4 *vr = (const uint4 *)(row + head);
    const int64_t nvec = (len - head) / EPV;
    const int64_t tail0 = head + nvec * EPV;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        A[c].a = p.cl[c].ident;
        A[c].c = 0.f;
    }
    if (lane < head) {
        T x = row[lane];
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_one<T>(w[c], A[c], x);
    }
    if (tail0 + lane < len) {
        T x = row[tail0 + lane];
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_one<T>(w[c], A[c], x);
    }
    int64_t v = lane;
    for (; v + (RU2 - 1) * 32 < nvec; v += 32 * RU2) {
        uint4 b[RU2];
#pragma unroll
        for (int u = 0; u < RU2; ++u) b[u] = ld_row(vr + v + u * 32);
#pragma unroll
        for (int c = 0; c < NC; ++c) fold_vec<T, RU2>(w[c], A[c], b);
    }
#pragma unroll
    for (int u = 0; u < RU2; ++u) {
        const int64_t vv = v + u * 32;
        if (vv < nvec) {
            uint4 b = ld_row(vr + vv);
#pragma unroll
            for (int c = 0; c < NC; ++c) fold_vec<T, 1>(w[c], A[c], &b);
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) warp_merge(w[c], E64, A[c]);
}

// W0 / W1 >= 0 fix the working codes of clauses 0 / 1 at compile time (the
// fold's operator switch then disappears from the row loop); -1 reads them
// from the arguments.  SPLIT selects the chunked form for long rows.
template <typename T, int NC, int W0 = -1, int W1 = -1, bool SPLIT = false>
__global__ void __launch_bounds__(row_threads<T, NC, SPLIT>()) rowreduce_kernel(const __grid_constant__ RowArgs p) {
    constexpr bool E64 = sizeof(T) == 8;
    constexpr int NTH = row_threads<T, NC, SPLIT>(), NW = NTH / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * NW + warp;
    const int64_t cols = p.cols;
    int w[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] = (c == 0 && W0 >= 0) ? W0 : (c == 1 && W1 >= 0) ? W1 : p.cl[c].wcode;
    Acc A[NC];

    if (!SPLIT) {
        const int64_t warps = (int64_t)gridDim.x * NW;
        for (int64_t r = gw; r < p.rows; r += warps) {
            fold_stretch<T, NC>(p, w, r, 0, cols, lane, A);
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (ACCR_DCHECK(r < p.rows, DS_ROW_VAR))
                        store_var(p.cl[c], r, finish(p.cl[c], E64, cols == 0, to_final(w[c], A[c])));
            }
        }
        return;
    }
    // this CTA's run of the rows x cpr chunks, its warps taking them in turn
    __shared__ Acc sh[NC][NW];
    const int64_t total = p.rows * p.cpr;
    const int64_t c0 = total * (int64_t)blockIdx.x / gridDim.x, c1 = total * ((int64_t)blockIdx.x + 1) / gridDim.x;
    for (int64_t k = c0 + warp; k < c1; k += NW) {
        const int64_t r = k / p.cpr, j = k - r * p.cpr, lo = j * p.chunk;
        const int64_t len = (cols - lo) < p.chunk ? (cols - lo) : p.chunk;
        if (!ACCR_DCHECK(r < p.rows && lo + len <= cols, DS_ROW_CHUNK)) continue;
        fold_stretch<T, NC>(p, w, r, lo, len, lane, A);
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                Partial q;
                q.a = A[c].a;
                q.c = A[c].c;
                q.pad = 0;
                if (ACCR_DCHECK((r * NC + c) * p.cpr + j < p.rows * NC * p.cpr, DS_ROW_PARTIAL))
                    p.partials[(r * NC + c) * p.cpr + j] = q;
            }
        }
    }
    // the CTA counts its chunks into each row it touched, thread t into row
    // r0 + t (an acquire-release add: it releases the CTA's partials, which
    // the barrier before it ordered, and the add that completes a row
    // acquires every other CTA's); the CTA then merges each row it completed
    // in chunk order (thread t takes chunks t, t + NTH, ..., loads in flight,
    // then the CTA tree)
    __shared__ int64_t s_rows[NTH];
    __shared__ int s_nd;
    __syncthreads();
    if (c0 >= c1) return;  // uniform across the CTA
    const int64_t r0 = c0 / p.cpr, r1 = (c1 - 1) / p.cpr;
    for (int64_t rb = r0; rb <= r1; rb += NTH) {
        if (threadIdx.x == 0) s_nd = 0;
        __syncthreads();
        const int64_t r = rb + threadIdx.x;
        if (r <= r1 && ACCR_DCHECK(r < p.rows, DS_ROW_COUNTER)) {
            const int64_t a = (r * p.cpr > c0 ? r * p.cpr : c0), b = ((r + 1) * p.cpr < c1 ? (r + 1) * p.cpr : c1);
            unsigned old;
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                         : "=r"(old)
                         : "l"(&p.counters[r]), "r"((unsigned)(b - a))
                         : "memory");
            if (old + (unsigned)(b - a) == (unsigned)p.cpr) s_rows[atomicAdd(&s_nd, 1)] = r;
        }
        __syncthreads();
        const int nd = s_nd;
        for (int iq = 0; iq < nd; ++iq) {
            const int64_t rr = s_rows[iq];
            int fw[NC];
            uint64_t fid[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                fw[c] = final_code(w[c]);
                fid[c] = final_ident(p.cl[c]);
                A[c].a = fid[c];
                A[c].c = 0.f;
            }
            constexpr int U = NC == 1 ? 4 : NC == 2 ? 2 : 1;  // loads in flight per clause and thread
            for (int64_t b0 = threadIdx.x; b0 < p.cpr; b0 += (int64_t)NTH * U) {
                Partial q[NC][U];
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (b0 + u * NTH < p.cpr)
                            q[c][u] = ld_row_partial(&p.partials[(rr * NC + c) * p.cpr] + b0 + u * NTH);
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (b0 + u * NTH < p.cpr) {
                            Acc Q;
                            Q.a = q[c][u].a;
                            Q.c = q[c][u].c;
                            merge(fw[c], E64, A[c], to_final(w[c], Q));
                        }
                    }
            }
            cta_merge<NC, NTH>(fw, fid, E64, A, sh);
            if (threadIdx.x == 0) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (ACCR_DCHECK(rr < p.rows, DS_ROW_VAR))
                        store_var(p.cl[c], rr, finish(p.cl[c], E64, cols == 0, A[c]));
                p.counters[rr] = 0u;
            }
            __syncthreads();
        }
    }
}

template <typename T, int NC, int W0, int W1, bool SPLIT>
static int max_row_grid() {
    static std::atomic<int> cached[64];
    const DeviceInfo &d = device_info();
    std::atomic<int> &slot = cached[d.id & 63];
    int g = slot.load(std::memory_order_relaxed);
    if (!g) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rowreduce_kernel<T, NC, W0, W1, SPLIT>,
                                                      row_threads<T, NC, SPLIT>(), 0);
        if (per_sm < 1) per_sm = 1;
        g = per_sm * d.sms;
        slot.store(g, std::memory_order_relaxed);
    }
    return g;
}

// CTAs for `segs` stretches: rows (one warp per row, at most the resident
// grid, the rest in later rounds), or chunks of long rows (the resident grid,
// at most one CTA per chunk, each CTA taking a contiguous run).
template <typename T, int NC, int W0, int W1, bool SPLIT>
static int row_grid(int64_t segs) {
    const int64_t maxg = max_row_grid<T, NC, W0, W1, SPLIT>();
    const int64_t g = SPLIT ? segs : (segs + WB / 32 - 1) / (WB / 32);
    return (int)(g < 1 ? 1 : g < maxg ? g : maxg);
}

template <typename T, int NC, int W0 = -1, int W1 = -1>
static int row_launch_t(RowArgs &a, cudaStream_t s) {
    int rc = launch_guard("rowreduce_kernel");
    if (rc != ACCR_OK) return rc;
    if (a.cpr > 0) {
        rowreduce_kernel<T, NC, W0, W1, true>
            <<<row_grid<T, NC, W0, W1, true>(a.rows * a.cpr), row_threads<T, NC, true>(), 0, s>>>(a);
    } else {
        rowreduce_kernel<T, NC, W0, W1, false><<<row_grid<T, NC, W0, W1, false>(a.rows), WB, 0, s>>>(a);
    }
    return launched("rowreduce_kernel");
}

// A sum together with a max or a min (the two-clause form of a region that
// reports a total and an extreme) gets a kernel with both codes fixed: the
// generic two-clause fold needs 64 registers a thread, the fixed one 32-40,
// which leaves room for more rows in flight per SM.
template <typename T, int W0, int W1>
static bool pair_launch(RowArgs &a, cudaStream_t s, int &rc) {
    if (a.cl[0].wcode != W0 || a.cl[1].wcode != W1) return false;
    rc = row_launch_t<T, 2, W0, W1>(a, s);
    return true;
}

template <typename T>
static bool row_launch_pair(RowArgs &a, cudaStream_t s, int &rc) {
    auto is_sum = [](int w) { return w == W_ADD32 || w == W_ADD64 || w == W_ADDF || w == W_ADDF_COMP; };
    if (!is_sum(a.cl[0].wcode) && is_sum(a.cl[1].wcode)) {  // each clause carries its own output
        const ClauseDev t = a.cl[0];
        a.cl[0] = a.cl[1];
        a.cl[1] = t;
    }
    if constexpr (std::is_same<T, float>::value) {
        return pair_launch<T, W_ADDF, W_MAXF>(a, s, rc) || pair_launch<T, W_ADDF, W_MINF>(a, s, rc) ||
               pair_launch<T, W_ADDF_COMP, W_MAXF>(a, s, rc) || pair_launch<T, W_ADDF_COMP, W_MINF>(a, s, rc);
    } else if constexpr (std::is_same<T, double>::value) {
        return pair_launch<T, W_ADDF, W_MAXF>(a, s, rc) || pair_launch<T, W_ADDF, W_MINF>(a, s, rc);
    } else if constexpr (std::is_same<T, int32_t>::value) {
        return pair_launch<T, W_ADD32, W_MAXI>(a, s, rc) || pair_launch<T, W_ADD32, W_MINI>(a, s, rc) ||
               pair_launch<T, W_ADD64, W_MAXI>(a, s, rc) || pair_launch<T, W_ADD64, W_MINI>(a, s, rc);
    } else {
        return pair_launch<T, W_ADD64, W_MAXI>(a, s, rc) || pair_launch<T, W_ADD64, W_MINI>(a, s, rc);
    }
}

template <typename T>
static int row_launch(RowArgs &a, cudaStream_t s) {
    int rc = ACCR_OK;
    if (a.nc == 2 && row_launch_pair<T>(a, s, rc)) return rc;
    switch (a.nc) {
    case 1: return row_launch_t<T, 1>(a, s);
    case 2: return row_launch_t<T, 2>(a, s);
    case 3: return row_launch_t<T, 3>(a, s);
    default: return row_launch_t<T, 4>(a, s);
    }
}

}  // namespace accr

using namespace accr;

extern "C" ACCR_API int accr_rowreduce(const void *A, int64_t rows, int64_t cols, int64_t ld, int32_t in_type,
                              const accr_clause *clauses, int32_t nclauses, uint32_t flags,
                              accr_stream_t stream) {
    ACCR_TRACE("accr_rowreduce");
    clear_error();
    if (flags & ~(ACCR_COMPENSATED | ACCR_SYNC))
        return set_error(ACCR_EINVAL, "accr_rowreduce: unsupported flags 0x%x", flags);
    if (rows < 0 || cols < 0) return set_error(ACCR_EINVAL, "accr_rowreduce: negative size");
    if (ld < cols) return set_error(ACCR_EINVAL, "accr_rowreduce: ld = %lld < cols = %lld", (long long)ld, (long long)cols);
    ClauseDev cl[ACCR_MAX_CLAUSES];
    int rc = lower_clauses(in_type, clauses, nclauses, flags, cl);
    if (rc != ACCR_OK) return rc;
    if (rows == 0) return ACCR_OK;
    if (cols > 0 && !A) return set_error(ACCR_EINVAL, "accr_rowreduce: A is NULL");
    if (((uintptr_t)A % (uintptr_t)type_bytes(in_type)) != 0)
        return set_error(ACCR_EINVAL, "accr_rowreduce: A is not aligned to its element size");
    cudaStream_t s = (cudaStream_t)stream;
    RowArgs a;
    memset(&a, 0, sizeof a);
    const int64_t eb = type_bytes(in_type), row_bytes = cols * eb;
    log_msg(2, "accr_rowreduce: %lld x %lld (ld %lld) type=%d clauses=%d form=%s", (long long)rows, (long long)cols,
            (long long)ld, in_type, nclauses, row_bytes >= SPLIT_ROW_BYTES ? "split rows" : "warp per row");
    if (row_bytes >= SPLIT_ROW_BYTES) {
        // chunked form: partials [rows][nclauses][cpr] and one counter per row
        a.chunk = SPLIT_CHUNK_BYTES / eb;
        a.cpr = (cols + a.chunk - 1) / a.chunk;
        const size_t pbytes = (size_t)rows * (size_t)nclauses * (size_t)a.cpr * sizeof(Partial);
        Scratch *scr = scratch_for(stream, pbytes);
        if (!scr) return ACCR_ENOMEM;
        a.partials = (Partial *)scr->buf;
        a.counters = zeroed_words_for(stream, (size_t)rows);  // every row completes, so each returns to zero
        if (!a.counters) return ACCR_ENOMEM;
    }
    a.A = A;
    a.rows = rows;
    a.cols = cols;
    a.ld = ld;
    a.nc = nclauses;
    for (int c = 0; c < nclauses; ++c) a.cl[c] = cl[c];
    switch (in_type) {
    case ACCR_I32: rc = row_launch<int32_t>(a, s); break;
    case ACCR_I64: rc = row_launch<int64_t>(a, s); break;
    case ACCR_F32: rc = row_launch<float>(a, s); break;
    default: rc = row_launch<double>(a, s); break;
    }
    if (rc != ACCR_OK) return rc;
    if (flags & ACCR_SYNC) return cuda_check(cudaStreamSynchronize(s), "accr_rowreduce: sync");
    return ACCR_OK;
}
