// rowreduce.cu -- the nest `for i (gang) { for j (vector) var_i (op)= A[i][j] }`:
// one reduction variable per row of a row-major matrix (the two-level loop
// shape of Listing 1a with an inner reduction; IPMACC Sec. 1.3, Stage 3.4).
//
// Mapping: gang -> CTA, worker -> warp, vector -> lane.  Two forms, chosen by
// the row's length alone (so a row's result never depends on how many rows
// the matrix has):
//
//   * rows shorter than SPLIT_ROW_BYTES: one warp owns a row, so no
//     cross-warp or cross-gang merge is needed: lanes stream the row in
//     16-byte vectors (RU2 in flight per lane), merge through shuffles, and
//     lane 0 writes the row's variable.  Rows whose start is not 16-byte
//     aligned (ld not a multiple of the vector) fold their head and tail
//     element by element.
//   * longer rows: each row is a region of one batched launch (batch.cu),
//     cut into CTA tiles of split_tile_bytes(row bytes) (at least 256 tiles a
//     row up to 2 MiB tiles); a tile's partial goes to scratch and the row's
//     last tile merges the partials in tile order.  A few long rows then
//     spread over every SM instead of over a few warps.
#include <string.h>

#include <mutex>
#include <type_traits>

#include "batch.cuh"
#include "common.cuh"
#include "fold.cuh"

namespace accr {

constexpr int64_t SPLIT_ROW_BYTES = 256 * 1024;

// Tile of the split-row form: row bytes / 256 rounded down to a power of two,
// within [64 KiB, 2 MiB].
static int64_t split_tile_bytes(int64_t row_bytes) {
    int64_t t = 64 * 1024;
    while (t * 2 <= row_bytes / 256 && t < 2 * 1024 * 1024) t *= 2;
    return t;
}

constexpr int WB = 256;  // threads per CTA (8 warps = 8 rows in flight)
constexpr int RU2 = 8;   // 16-byte vectors per lane per iteration

struct RowArgs {
    const void *A;
    int64_t rows, cols, ld;
    int nc;
    ClauseDev cl[ACCR_MAX_CLAUSES];
};

__device__ __forceinline__ uint4 ld_row(const uint4 *p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

// W0 / W1 >= 0 fix the working codes of clauses 0 / 1 at compile time (the
// fold's operator switch then disappears from the row loop); -1 reads them
// from the arguments.
template <typename T, int NC, int W0 = -1, int W1 = -1>
__global__ void __launch_bounds__(WB) rowreduce_kernel(const __grid_constant__ RowArgs p) {
    constexpr bool E64 = sizeof(T) == 8;
    constexpr int EPV = 16 / (int)sizeof(T);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (WB / 32);
    const int64_t cols = p.cols;
    int w[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] = (c == 0 && W0 >= 0) ? W0 : (c == 1 && W1 >= 0) ? W1 : p.cl[c].wcode;

    for (int64_t r = (int64_t)blockIdx.x * (WB / 32) + (threadIdx.x >> 5); r < p.rows; r += warps) {
        const T *row = (const T *)p.A + r * p.ld;
        const int64_t mis = (int64_t)(((16 - ((uintptr_t)row & 15)) & 15) / sizeof(T));
        const int64_t head = mis < cols ? mis : cols;
        const uint4 *vr = (const uint4 *)(row + head);
        const int64_t nvec = (cols - head) / EPV;
        const int64_t tail0 = head + nvec * EPV;
        Acc A[NC];
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
        if (tail0 + lane < cols) {
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
        for (int c = 0; c < NC; ++c) {
            warp_merge(w[c], E64, A[c]);
            if (lane == 0) store_var(p.cl[c], r, finish(p.cl[c], E64, cols == 0, to_final(w[c], A[c])));
        }
    }
}

template <typename T, int NC, int W0 = -1, int W1 = -1>
static int row_grid(int64_t rows) {
    static std::mutex mu;
    static int cached[64] = {0};
    const DeviceInfo &d = device_info();
    int maxg;
    {
        std::lock_guard<std::mutex> lk(mu);
        int &slot = cached[d.id & 63];
        if (!slot) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rowreduce_kernel<T, NC, W0, W1>, WB, 0);
            if (per_sm < 1) per_sm = 1;
            slot = per_sm * d.sms;
        }
        maxg = slot;
    }
    int64_t want = (rows + WB / 32 - 1) / (WB / 32);
    if (want < 1) want = 1;
    return (int)(want < maxg ? want : maxg);
}

template <typename T, int NC, int W0 = -1, int W1 = -1>
static int row_launch_t(RowArgs &a, cudaStream_t s) {
    int rc = launch_guard("rowreduce_kernel");
    if (rc != ACCR_OK) return rc;
    rowreduce_kernel<T, NC, W0, W1><<<row_grid<T, NC, W0, W1>(a.rows), WB, 0, s>>>(a);
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
    const int64_t row_bytes = cols * (int64_t)type_bytes(in_type);
    if (row_bytes >= SPLIT_ROW_BYTES) {
        rc = batch_launch_rows(A, rows, cols, ld, in_type, cl, nclauses, split_tile_bytes(row_bytes), stream);
        if (rc != ACCR_OK) return rc;
        if (flags & ACCR_SYNC) return cuda_check(cudaStreamSynchronize(s), "accr_rowreduce: sync");
        return ACCR_OK;
    }
    RowArgs a;
    memset(&a, 0, sizeof a);
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
