// matmul_tc.cu -- the Listing-1a nest on the 5th-generation tensor cores in
// BF16x3 split precision.
//
// The nest c[i][j] = sum_l a[i][l] * b[l][j] is a dense contraction, so it is
// the one place in this library that uses tcgen05.  Each float operand is
// split as x = hi + lo with hi = bf16(x) and lo = bf16(x - hi) (round to
// nearest), and
//
//     c ~= a_hi b_hi + a_hi b_lo + a_lo b_hi
//
// is accumulated in FP32 in tensor memory (the dropped a_lo b_lo term and the
// split residuals are of order 2^-16 of |a||b|).
//
// Kernel shape: one CTA computes a 128 x 256 block of c with
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = 256, K = 16).  A TMA
// producer thread streams 64-wide k slices of the four split operands into a
// two-stage shared-memory ring (128-byte swizzle, the layout the MMA
// descriptors expect); an MMA thread waits on each stage's mbarrier, issues
// the three products for the four 16-wide k steps, and frees the stage with
// tcgen05.commit; after the last slice the four warps read the accumulator
// out of tensor memory (tcgen05.ld 32x32b) and store c.
//
// Every wait is bounded: if one runs out, the CTA records an error code in
// global memory, lets its own copies in flight land, releases its tensor
// memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <string.h>

#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace accr {

constexpr int TBM = 128, TBN = 256, TBK = 64;
constexpr int TSTAGES = 2;
constexpr int A_TILE_BYTES = TBM * TBK * 2;                       // 16 KiB
constexpr int B_TILE_BYTES = TBN * TBK * 2;                       // 32 KiB
constexpr int STAGE_BYTES = 2 * A_TILE_BYTES + 2 * B_TILE_BYTES;  // 96 KiB
constexpr int TMEM_COLS = 256;
constexpr uint32_t kMaxTries = 1u << 24;

// Instruction descriptor (kind::f16): FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                           ((uint32_t)(TBM >> 4) << 24);

struct TcBars {
    uint64_t full[TSTAGES];
    uint64_t empty[TSTAGES];
    uint64_t done;
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kMaxTries; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // version
    d |= (uint64_t)2 << 61;            // SWIZZLE_128B
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        ::"r"(tmem), "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(128, 1)
    bf16x3_gemm_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                       const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
                       float *__restrict__ C, int M, int N, int Kp, int *err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcBars *bars = (TcBars *)(smem + TSTAGES * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const int nkb = Kp / TBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TSTAGES; ++s) {
            mbar_init(smem_u32(&bars->full[s]), 1);
            mbar_init(smem_u32(&bars->empty[s]), 1);
        }
        mbar_init(smem_u32(&bars->done), 1);
        bars->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = bars->tmem;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer ----
        int issued[TSTAGES];
        for (int s = 0; s < TSTAGES; ++s) issued[s] = -1;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % TSTAGES, use = kb / TSTAGES;
            if (use > 0 && !mbar_wait(smem_u32(&bars->empty[s]), (uint32_t)((use - 1) & 1))) {
                atomicExch(err, 1);
                bars->abort = 1;
                break;
            }
            if (*(volatile int *)&bars->abort) break;
            uint8_t *st = smem + s * STAGE_BYTES;
            const uint32_t fb = smem_u32(&bars->full[s]);
            mbar_expect_tx(fb, STAGE_BYTES);
            tma_load_2d(smem_u32(st), &tAh, kb * TBK, m0, fb);
            tma_load_2d(smem_u32(st + A_TILE_BYTES), &tAl, kb * TBK, m0, fb);
            tma_load_2d(smem_u32(st + 2 * A_TILE_BYTES), &tBh, kb * TBK, n0, fb);
            tma_load_2d(smem_u32(st + 2 * A_TILE_BYTES + B_TILE_BYTES), &tBl, kb * TBK, n0, fb);
            issued[s] = use;
        }
        // let every copy this thread issued land before the CTA can exit
        for (int s = 0; s < TSTAGES; ++s)
            if (issued[s] >= 0 && !mbar_wait(smem_u32(&bars->full[s]), (uint32_t)(issued[s] & 1))) atomicExch(err, 2);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % TSTAGES, use = kb / TSTAGES;
            if (!mbar_wait(smem_u32(&bars->full[s]), (uint32_t)(use & 1))) {
                atomicExch(err, 3);
                bars->abort = 1;
                break;
            }
            if (*(volatile int *)&bars->abort) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t ah = st, al = st + A_TILE_BYTES;
            const uint32_t bh = st + 2 * A_TILE_BYTES, bl = bh + B_TILE_BYTES;
#pragma unroll
            for (int kk = 0; kk < TBK / 16; ++kk) {
                const uint32_t off = kk * 32;  // 16 bf16 along K inside the 128-byte swizzle atom
                mma_bf16(tmem, smem_desc(ah + off), smem_desc(bh + off), (kb > 0 || kk > 0) ? 1u : 0u);
                mma_bf16(tmem, smem_desc(ah + off), smem_desc(bl + off), 1u);
                mma_bf16(tmem, smem_desc(al + off), smem_desc(bh + off), 1u);
            }
            mma_commit(smem_u32(&bars->empty[s]));
        }
        mma_commit(smem_u32(&bars->done));  // fires when every MMA issued above is complete
    }
    __syncwarp();

    // ---- epilogue: accumulator rows 32*warp .. +31 to c ----
    bool ready = mbar_wait(smem_u32(&bars->done), 0);
    if (!ready) atomicExch(err, 4);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool store = ready && !*(volatile int *)&bars->abort;
    const int row = m0 + warp * 32 + lane;
    const bool vec = (N % 4 == 0) && (((uintptr_t)C & 15) == 0);
#pragma unroll 1
    for (int ch = 0; ch < TBN / 32; ++ch) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32), r);
        if (!store || row >= M) continue;
        const int col = n0 + ch * 32;
        float *dst = C + (size_t)row * (size_t)N + col;
        if (vec && col + 32 <= N) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                *reinterpret_cast<float4 *>(dst + j) =
                    make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                __uint_as_float(r[j + 3]));
        } else {
            for (int j = 0; j < 32; ++j)
                if (col + j < N) dst[j] = __uint_as_float(r[j]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Self-test of the bounded wait: nothing ever arrives on this barrier.
__global__ void wait_selftest_kernel(uint32_t tries, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = false;
        for (uint32_t i = 0; i < tries && !ok; ++i) {
            uint32_t r;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(r)
                : "r"(smem_u32(&bar)), "r"(0u)
                : "memory");
            ok = r != 0;
        }
        if (!ok) atomicExch(err, 5);
    }
}

// hi = bf16(x), lo = bf16(x - hi); a row-major M x K -> [M][Kp] (zero padded)
__global__ void split_rows_kernel(const float *__restrict__ a, int64_t M, int64_t K, int64_t Kp,
                                  __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo) {
    const int64_t total = M * Kp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / Kp, k = i - r * Kp;
        const float x = k < K ? a[r * K + k] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[i] = h;
        lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// b row-major K x N -> transposed split [N][Kp] (zero padded), 32 x 32 tiles
__global__ void split_cols_kernel(const float *__restrict__ b, int64_t K, int64_t N, int64_t Kp,
                                  __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo) {
    __shared__ float tile[32][33];
    const int64_t k0 = (int64_t)blockIdx.y * 32, n0 = (int64_t)blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t k = k0 + r, n = n0 + threadIdx.x;
        tile[r][threadIdx.x] = (k < K && n < N) ? b[k * N + n] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t n = n0 + r, k = k0 + threadIdx.x;
        if (n < N && k < Kp) {
            const float x = tile[threadIdx.x][r];
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            hi[n * Kp + k] = h;
            lo[n * Kp + k] = __float2bfloat16_rn(x - __bfloat162float(h));
        }
    }
}

// ---- host side --------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// 2-D bf16 map over [rows][Kp], box {64, box_rows}, 128-byte swizzle.
static int make_map(CUtensorMap *m, const void *base, int64_t rows, int64_t Kp, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return set_error(ACCR_ECUDA, "accr_matmul_nest: cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(ACCR_ECUDA, "accr_matmul_nest: tensor map encode failed (%d)", (int)r);
    return ACCR_OK;
}

struct SplitBufs {
    void *buf = nullptr;
    size_t bytes = 0;
};
static std::mutex g_split_mu;
static std::map<std::pair<int, uintptr_t>, SplitBufs> g_split;

int matmul_bf16x3(const float *a, const float *b, float *c, int64_t len, cudaStream_t s, bool sync) {
    if (len == 0) return ACCR_OK;
    if (len > (1 << 20)) return set_error(ACCR_EINVAL, "accr_matmul_nest: len too large for the tensor-core path");
    const int64_t M = len, N = len, K = len;
    const int64_t Kp = (K + TBK - 1) / TBK * TBK;
    const size_t abytes = (size_t)M * Kp * 2, bbytes = (size_t)N * Kp * 2;
    const size_t need = 2 * abytes + 2 * bbytes + 256;
    SplitBufs *sb;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(g_split_mu);
        sb = &g_split[std::make_pair(dev, (uintptr_t)s)];
        if (sb->bytes < need && fault_take(ACCR_FAULT_ALLOC))
            return set_error(ACCR_ENOMEM, "accr_matmul_nest: injected allocation failure");
        if (sb->bytes < need) {
            if (sb->buf) {
                cudaStreamSynchronize(s);
                cudaFree(sb->buf);
                sb->buf = nullptr;
                sb->bytes = 0;
            }
            if (cudaMalloc(&sb->buf, need) != cudaSuccess) {
                cudaGetLastError();
                return set_error(ACCR_ENOMEM, "accr_matmul_nest: split buffers (%zu bytes)", need);
            }
            sb->bytes = need;
        }
    }
    char *base = (char *)sb->buf;
    int *err = (int *)base;
    __nv_bfloat16 *ah = (__nv_bfloat16 *)(base + 256), *al = (__nv_bfloat16 *)(base + 256 + abytes);
    __nv_bfloat16 *bh = (__nv_bfloat16 *)(base + 256 + 2 * abytes), *bl = (__nv_bfloat16 *)(base + 256 + 2 * abytes + bbytes);
    int rc = launch_guard("bf16x3_gemm_kernel");
    if (rc != ACCR_OK) return rc;
    rc = cuda_check(cudaMemsetAsync(err, 0, sizeof(int), s), "accr_matmul_nest: clear flag");
    if (rc != ACCR_OK) return rc;
    const DeviceInfo &di = device_info();
    split_rows_kernel<<<di.sms * 8, 256, 0, s>>>(a, M, K, Kp, ah, al);
    if ((rc = launched("split_rows_kernel")) != ACCR_OK) return rc;
    dim3 tg((unsigned)((N + 31) / 32), (unsigned)((Kp + 31) / 32));
    split_cols_kernel<<<tg, dim3(32, 8), 0, s>>>(b, K, N, Kp, bh, bl);
    if ((rc = launched("split_cols_kernel")) != ACCR_OK) return rc;
    CUtensorMap mah, mal, mbh, mbl;
    if ((rc = make_map(&mah, ah, M, Kp, TBM)) != ACCR_OK) return rc;
    if ((rc = make_map(&mal, al, M, Kp, TBM)) != ACCR_OK) return rc;
    if ((rc = make_map(&mbh, bh, N, Kp, TBN)) != ACCR_OK) return rc;
    if ((rc = make_map(&mbl, bl, N, Kp, TBN)) != ACCR_OK) return rc;
    const int smem = TSTAGES * STAGE_BYTES + (int)sizeof(TcBars) + 1024;
    static std::once_flag attr_once;
    std::call_once(attr_once, [smem] {
        cudaFuncSetAttribute(bf16x3_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    dim3 grid((unsigned)((N + TBN - 1) / TBN), (unsigned)((M + TBM - 1) / TBM));
    bf16x3_gemm_kernel<<<grid, 128, smem, s>>>(mah, mal, mbh, mbl, c, (int)M, (int)N, (int)Kp, err);
    if ((rc = launched("bf16x3_gemm_kernel")) != ACCR_OK) return rc;
    if (sync) {
        int h = 0;
        rc = cuda_check(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s), "accr_matmul_nest: flag");
        if (rc == ACCR_OK) rc = cuda_check(cudaStreamSynchronize(s), "accr_matmul_nest: sync");
        if (rc == ACCR_OK && h != 0)
            return set_error(ACCR_ETIMEDOUT, "accr_matmul_nest: a pipeline wait ran out (code %d)", h);
    }
    return rc;
}

int selftest_wait_timeout(uint32_t tries, cudaStream_t s) {
    Scratch *scr = scratch_for((accr_stream_t)s, 64);
    if (!scr) return ACCR_ENOMEM;
    int *err = (int *)scr->buf;
    int rc = cuda_check(cudaMemsetAsync(err, 0, sizeof(int), s), "selftest: clear");
    if (rc != ACCR_OK) return rc;
    if ((rc = launch_guard("wait_selftest_kernel")) != ACCR_OK) return rc;
    wait_selftest_kernel<<<1, 32, 0, s>>>(tries, err);
    if ((rc = launched("wait_selftest_kernel")) != ACCR_OK) return rc;
    int h = 0;
    rc = cuda_check(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s), "selftest: flag");
    if (rc == ACCR_OK) rc = cuda_check(cudaStreamSynchronize(s), "selftest: sync");
    if (rc != ACCR_OK) return rc;
    if (h == 5) return set_error(ACCR_ETIMEDOUT, "selftest: the bounded wait ran out after %u polls", tries);
    return ACCR_OK;
}

}  // namespace accr

extern "C" ACCR_API int accr_selftest_wait_timeout(uint32_t tries, accr_stream_t stream) {
    accr::clear_error();
    return accr::selftest_wait_timeout(tries, (cudaStream_t)stream);
}
