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
// Kernel shape: one CTA computes a 128 x 224 block of c with
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = 224, K = 16).  The split
// operands are stored packed: every 32-wide k block of a row holds its 32 hi
// values followed by its 32 lo values, one 128-byte row.  A TMA producer
// thread streams one such k block of a and of b per stage into a four-stage
// shared-memory ring (128-byte swizzle, the layout the MMA descriptors
// expect: two TMA copies and 128-byte rows per stage); an MMA thread waits on
// each stage's mbarrier, issues the three products for the two 16-wide k
// steps (hi and lo sit 64 bytes apart inside the swizzled row), and frees the
// stage with tcgen05.commit; after the last slice the four warps read the
// accumulator out of tensor memory (tcgen05.ld 32x32b) and store c.
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
#include "debug.cuh"

namespace accr {

// CTA tile 128 x 224: at LEN 4096 the 19 x 32 = 608 tiles are exactly four
// waves on 152 SMs (128 x 256 tiles would be 3.4 waves); 32-wide k slices,
// hi and lo packed in one 128-byte swizzled row, give a four-stage ring in
// 176 KiB of shared memory.
constexpr int TBM = 128, TBN = 224, TBK = 32;
constexpr int TSTAGES = 4;
constexpr int SWZ = 128;                             // swizzle span (bytes) = one packed k-block row
constexpr int PK = 2 * TBK;                          // packed row length (bf16): 32 hi then 32 lo
constexpr int A_TILE_BYTES = TBM * PK * 2;           // 16 KiB
constexpr int B_TILE_BYTES = TBN * PK * 2;           // 28 KiB
constexpr int STAGE_BYTES = A_TILE_BYTES + B_TILE_BYTES;  // 44 KiB, a multiple of the 1 KiB swizzle pattern
constexpr int TMEM_COLS = 512;                                    // two accumulators, at columns 0 and 256
constexpr int GEMM_THREADS = 192;  // warp 0 TMA producer, warp 1 MMA issuer, warps 2-5 epilogue
constexpr uint32_t kMaxTries = 1u << 24;

// Instruction descriptor (kind::f16): FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                           ((uint32_t)(TBM >> 4) << 24);

struct TcBars {
    uint64_t full[TSTAGES];   // stage s loaded (TMA transaction count)
    uint64_t empty[TSTAGES];  // stage s consumed (MMA commit)
    uint64_t tfull[2];        // accumulator b complete (MMA commit)
    uint64_t tempty[2];       // accumulator b drained (one arrival per epilogue warp)
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
// groups 8 x 128 = 1024 bytes apart (SBO), descriptor version 1.  A start
// address inside a row (the k step and the hi/lo half, < 128 bytes) leaves
// the pattern phase, address bits 7-9, at zero.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((8 * SWZ) >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;                  // version
    d |= (uint64_t)2 << 61;                  // SWIZZLE_128B
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent: one CTA per SM walks the tiles tile = blockIdx.x, +gridDim.x, ...
// The k-slice ring runs on across tiles; the accumulator alternates between
// two tensor-memory buffers so the epilogue of one tile overlaps the main
// loop of the next.
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    bf16x3_gemm_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
                       float *__restrict__ C, int M, int N, int Kp, int tiles_n, int ntiles, int *err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcBars *bars = (TcBars *)(smem + TSTAGES * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = Kp / TBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TSTAGES; ++s) {
            mbar_init(smem_u32(&bars->full[s]), 1);
            mbar_init(smem_u32(&bars->empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bars->tfull[b]), 1);
            mbar_init(smem_u32(&bars->tempty[b]), 4);
        }
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
    volatile int *abort = &bars->abort;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer ----
        int issued[TSTAGES];
        for (int s = 0; s < TSTAGES; ++s) issued[s] = -1;
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x) {
            const int m0 = (tile / tiles_n) * TBM, n0 = (tile % tiles_n) * TBN;
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = it % TSTAGES, use = it / TSTAGES;
                if (use > 0 && !mbar_wait(smem_u32(&bars->empty[s]), (uint32_t)((use - 1) & 1))) {
                    atomicExch(err, 1);
                    *abort = 1;
                    break;
                }
                if (*abort) break;
                uint8_t *st = smem + s * STAGE_BYTES;
                const uint32_t fb = smem_u32(&bars->full[s]);
                mbar_expect_tx(fb, STAGE_BYTES);
                tma_load_2d(smem_u32(st), &tA, kb * PK, m0, fb);
                tma_load_2d(smem_u32(st + A_TILE_BYTES), &tB, kb * PK, n0, fb);
                issued[s] = use;
            }
        }
        // let every copy this thread issued land before the CTA can exit
        for (int s = 0; s < TSTAGES; ++s)
            if (issued[s] >= 0 && !mbar_wait(smem_u32(&bars->full[s]), (uint32_t)(issued[s] & 1))) atomicExch(err, 2);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        int it = 0, j = 0;
        for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x, ++j) {
            const int b = j & 1, u = j >> 1;
            if (u > 0 && !mbar_wait(smem_u32(&bars->tempty[b]), (uint32_t)((u - 1) & 1))) {
                atomicExch(err, 5);
                *abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)(b * 256);
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = it % TSTAGES, use = it / TSTAGES;
                if (!mbar_wait(smem_u32(&bars->full[s]), (uint32_t)(use & 1))) {
                    atomicExch(err, 3);
                    *abort = 1;
                    ok = false;
                    break;
                }
                if (*abort) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = smem_u32(smem + s * STAGE_BYTES);
                const uint32_t ah = st, al = st + 64;  // hi and lo halves of the packed row
                const uint32_t bh = st + A_TILE_BYTES, bl = bh + 64;
#pragma unroll
                for (int kk = 0; kk < TBK / 16; ++kk) {
                    const uint32_t off = kk * 32;  // 16 bf16 along K inside each half
                    mma_bf16(acc, smem_desc(ah + off), smem_desc(bh + off), (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_bf16(acc, smem_desc(ah + off), smem_desc(bl + off), 1u);
                    mma_bf16(acc, smem_desc(al + off), smem_desc(bh + off), 1u);
                }
                mma_commit(smem_u32(&bars->empty[s]));
            }
            mma_commit(smem_u32(&bars->tfull[b]));  // fires when this tile's MMAs are complete
            if (!ok) break;
        }
    } else if (warp >= 2) {
        // ---- epilogue: accumulator lanes 32*q .. +31 (q = warp % 4) to c ----
        const int q = warp & 3;
        const bool vec = (N % 4 == 0) && (((uintptr_t)C & 15) == 0);
        int j = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
            const int b = j & 1, u = j >> 1;
            const bool ready = mbar_wait(smem_u32(&bars->tfull[b]), (uint32_t)(u & 1));
            if (!ready) {
                if (lane == 0) atomicExch(err, 4);
                *abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (tile / tiles_n) * TBM, n0 = (tile % tiles_n) * TBN;
            // a tile with no element inside c means the host's tile count is wrong
            const bool store = !*abort && ACCR_DCHECK(m0 < M && n0 < N, DS_GEMM_STORE);
            const int row = m0 + q * 32 + lane;
#pragma unroll 1
            for (int ch = 0; ch < TBN / 32; ++ch) {
                uint32_t r[32];
                tmem_ld32(tmem + (uint32_t)(b * 256) + ((uint32_t)(q * 32) << 16) + (uint32_t)(ch * 32), r);
                if (!store || row >= M) continue;
                const int col = n0 + ch * 32;
                float *dst = C + (size_t)row * (size_t)N + col;
                if (vec && col + 32 <= N) {
#pragma unroll
                    for (int e = 0; e < 32; e += 4)
                        *reinterpret_cast<float4 *>(dst + e) =
                            make_float4(__uint_as_float(r[e]), __uint_as_float(r[e + 1]), __uint_as_float(r[e + 2]),
                                        __uint_as_float(r[e + 3]));
                } else {
                    for (int e = 0; e < 32; ++e)
                        if (col + e < N) dst[e] = __uint_as_float(r[e]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[b]));  // buffer b may be overwritten
            if (*abort) break;
        }
    }
    __syncwarp();
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

__device__ __forceinline__ void split2(float x, __nv_bfloat16 &h, __nv_bfloat16 &l) {
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(__fsub_rn(x, __bfloat162float(h)));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 (&v)[8]) {
    return make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}

// Offset of element k of a packed row: k block k / 32 holds 32 hi values and
// then 32 lo values, so hi of k sits at 64 (k / 32) + k % 32 and lo 32 later.
__device__ __forceinline__ int64_t packed_hi(int64_t k) { return (k >> 5) * PK + (k & 31); }

constexpr int SPLIT_THREADS = 256;
constexpr int SPLIT_A_ITEMS = 4;  // 8-element groups of a per thread

// One launch splits both operands (hi = bf16(x), lo = bf16(x - hi)) into the
// packed, zero-padded layout the GEMM streams: blocks [0, nblk_a) take a
// (row-major len x len, rows kept), the rest take 64 x 64 tiles of b
// (row-major, transposed through shared memory so that a row of the packed
// b is a column of b).
__global__ void __launch_bounds__(SPLIT_THREADS) split_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                                              int64_t len, int64_t Kp, __nv_bfloat16 *__restrict__ ap,
                                                              __nv_bfloat16 *__restrict__ bp, int nblk_a, int tiles_n,
                                                              int vec) {
    __shared__ float tile[64][65];
    const int64_t row_stride = 2 * Kp;
    if ((int)blockIdx.x < nblk_a) {
        const int64_t k8 = Kp / 8, total = len * k8;
        const int64_t t0 = (int64_t)blockIdx.x * (SPLIT_THREADS * SPLIT_A_ITEMS) + threadIdx.x;
        float x[SPLIT_A_ITEMS][8];
#pragma unroll
        for (int j = 0; j < SPLIT_A_ITEMS; ++j) {  // every load first, then the stores
            const int64_t t = t0 + (int64_t)j * SPLIT_THREADS;
            const int64_t r = t / k8, k0 = (t - r * k8) * 8;
            if (t < total && vec && k0 + 8 <= len) {
                const float4 u = __ldg(reinterpret_cast<const float4 *>(a + r * len + k0));
                const float4 w = __ldg(reinterpret_cast<const float4 *>(a + r * len + k0 + 4));
                x[j][0] = u.x, x[j][1] = u.y, x[j][2] = u.z, x[j][3] = u.w;
                x[j][4] = w.x, x[j][5] = w.y, x[j][6] = w.z, x[j][7] = w.w;
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) x[j][e] = (t < total && k0 + e < len) ? a[r * len + k0 + e] : 0.f;
            }
        }
#pragma unroll
        for (int j = 0; j < SPLIT_A_ITEMS; ++j) {
            const int64_t t = t0 + (int64_t)j * SPLIT_THREADS;
            if (t >= total) break;
            const int64_t r = t / k8, k0 = (t - r * k8) * 8;
            __nv_bfloat16 h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) split2(x[j][e], h[e], l[e]);
            __nv_bfloat16 *dst = ap + r * row_stride + packed_hi(k0);
            *reinterpret_cast<uint4 *>(dst) = pack8(h);
            *reinterpret_cast<uint4 *>(dst + TBK) = pack8(l);
        }
        return;
    }
    const int bt = (int)blockIdx.x - nblk_a;
    const int64_t k0 = (int64_t)(bt / tiles_n) * 64, n0 = (int64_t)(bt % tiles_n) * 64;
    {  // 64 k x 64 n: 16 float4 per k row, four rows per thread, loads first
        const int c4 = (threadIdx.x & 15) * 4, r0 = threadIdx.x >> 4;
        float4 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t k = k0 + r0 + 16 * i, n = n0 + c4;
            if (vec && k < len && n + 4 <= len) {
                v[i] = __ldg(reinterpret_cast<const float4 *>(b + k * len + n));
            } else {
                v[i].x = (k < len && n + 0 < len) ? b[k * len + n + 0] : 0.f;
                v[i].y = (k < len && n + 1 < len) ? b[k * len + n + 1] : 0.f;
                v[i].z = (k < len && n + 2 < len) ? b[k * len + n + 2] : 0.f;
                v[i].w = (k < len && n + 3 < len) ? b[k * len + n + 3] : 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float *t = &tile[r0 + 16 * i][c4];
            t[0] = v[i].x, t[1] = v[i].y, t[2] = v[i].z, t[3] = v[i].w;
        }
    }
    __syncthreads();
    // 64 n x 8 groups of 8 k = 512 groups, two per thread; the eight groups of
    // one n are eight neighbouring threads (256 contiguous output bytes)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int g = threadIdx.x + j * SPLIT_THREADS;
        const int nn = g >> 3, kg = (g & 7) * 8;
        const int64_t n = n0 + nn, k = k0 + kg;
        if (n >= len || k >= Kp) continue;
        __nv_bfloat16 h[8], l[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) split2(tile[kg + e][nn], h[e], l[e]);
        __nv_bfloat16 *dst = bp + n * row_stride + packed_hi(k);
        *reinterpret_cast<uint4 *>(dst) = pack8(h);
        *reinterpret_cast<uint4 *>(dst + TBK) = pack8(l);
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

// 2-D bf16 map over the packed [rows][2 Kp], box {64, box_rows} (one
// 128-byte k block per row), 128-byte swizzle.
static int make_map(CUtensorMap *m, const void *base, int64_t rows, int64_t Kp, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return set_error(ACCR_ECUDA, "accr_matmul_nest: cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)(2 * Kp), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(2 * Kp) * 2};
    cuuint32_t box[2] = {(cuuint32_t)PK, (cuuint32_t)box_rows};
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
    const float *a = nullptr, *b = nullptr;  // operands of the last split on this stream
    int64_t len = -1;
};
static std::mutex g_split_mu;
static std::map<std::pair<int, uintptr_t>, SplitBufs> g_split;

int matmul_bf16x3(const float *a, const float *b, float *c, int64_t len, cudaStream_t s, bool sync, bool reuse) {
    if (len == 0) return ACCR_OK;
    if (len > (1 << 20)) return set_error(ACCR_EINVAL, "accr_matmul_nest: len too large for the tensor-core path");
    const int64_t M = len, N = len, K = len;
    const int64_t Kp = (K + TBK - 1) / TBK * TBK;
    const size_t abytes = (size_t)M * Kp * 4, bbytes = (size_t)N * Kp * 4;  // packed hi + lo
    const size_t need = abytes + bbytes + 256;
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
            sb->a = sb->b = nullptr;
            sb->len = -1;
            if (cudaMalloc(&sb->buf, need) != cudaSuccess) {
                cudaGetLastError();
                return set_error(ACCR_ENOMEM, "accr_matmul_nest: split buffers (%zu bytes)", need);
            }
            sb->bytes = need;
        }
    }
    char *base = (char *)sb->buf;
    int *err = (int *)base;
    __nv_bfloat16 *ap = (__nv_bfloat16 *)(base + 256), *bp = (__nv_bfloat16 *)(base + 256 + abytes);
    int rc = launch_guard("bf16x3_gemm_kernel");
    if (rc != ACCR_OK) return rc;
    rc = cuda_check(cudaMemsetAsync(err, 0, sizeof(int), s), "accr_matmul_nest: clear flag");
    if (rc != ACCR_OK) return rc;
    const DeviceInfo &di = device_info();
    if (!(reuse && sb->a == a && sb->b == b && sb->len == len)) {
        const int64_t items_a = M * (Kp / 8), per_blk = SPLIT_THREADS * SPLIT_A_ITEMS;
        const int64_t nblk_a = (items_a + per_blk - 1) / per_blk;
        const int64_t tn = (N + 63) / 64, nblk_b = tn * ((Kp + 63) / 64);
        if (nblk_a + nblk_b > INT32_MAX) return set_error(ACCR_EINVAL, "accr_matmul_nest: len too large for the split");
        const int vec = (K % 4 == 0) && (((uintptr_t)a & 15) == 0) && (((uintptr_t)b & 15) == 0);
        split_kernel<<<(unsigned)(nblk_a + nblk_b), SPLIT_THREADS, 0, s>>>(a, b, len, Kp, ap, bp, (int)nblk_a,
                                                                          (int)tn, vec);
        if ((rc = launched("split_kernel")) != ACCR_OK) return rc;
        sb->a = a;
        sb->b = b;
        sb->len = len;
    }
    CUtensorMap ma, mb;
    if ((rc = make_map(&ma, ap, M, Kp, TBM)) != ACCR_OK) return rc;
    if ((rc = make_map(&mb, bp, N, Kp, TBN)) != ACCR_OK) return rc;
    const int smem = TSTAGES * STAGE_BYTES + (int)sizeof(TcBars) + 1024;
    {  // the shared-memory opt-in is a per-device function attribute
        static std::mutex attr_mu;
        static bool attr_set[64] = {false};
        std::lock_guard<std::mutex> lk(attr_mu);
        if (!attr_set[di.id & 63]) {
            rc = cuda_check(cudaFuncSetAttribute(bf16x3_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                            "accr_matmul_nest: shared memory opt-in");
            if (rc != ACCR_OK) return rc;
            attr_set[di.id & 63] = true;
        }
    }
    const int tiles_n = (int)((N + TBN - 1) / TBN), ntiles = tiles_n * (int)((M + TBM - 1) / TBM);
    const int grid = ntiles < di.sms ? ntiles : di.sms;  // persistent: one CTA per SM
    bf16x3_gemm_kernel<<<grid, GEMM_THREADS, smem, s>>>(ma, mb, c, (int)M, (int)N, (int)Kp, tiles_n,
                                                        ntiles, err);
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
    ACCR_TRACE("accr_selftest_wait_timeout");
    accr::clear_error();
    return accr::selftest_wait_timeout(tries, (cudaStream_t)stream);
}
