// matmul_simt.cu -- the Listing-1a nest on FP32 CUDA cores.
//
//   for i (gang, independent) for j (vector, independent)
//     { float sum = 0; for l (serial) sum += a[i*LEN+l] * b[l*LEN+j]; c[i*LEN+j] = sum; }
//
// The paper's own CUDA version (Listing 1b) gives every thread one output and
// reads a and b straight from global memory; Sec. 4.2 (Matrix Mul) notes that
// the tiled CUDA SDK version, which stages tiles in shared memory and shares
// them among a block's threads, is much faster.  This kernel is the tiled
// form: a CTA computes a 128 x 128 block of c, stages 16-wide k slices of a
// (transposed) and b in double-buffered shared memory, and every thread keeps
// an 8 x 8 register block (two 4 x 4 quadrants 64 apart, so the 16-byte
// shared-memory reads of a warp hit distinct banks or broadcast), with its
// operand fragments double-buffered in registers.
//
// Every output still sums its l terms in order 0..LEN-1.  Mode SERIAL rounds
// each product and then each sum (no fused multiply-add), which is exactly
// the serial float program, bit for bit; mode FMA fuses them (faster, and
// closer to the exact product).
#include <string.h>

#include "common.cuh"

namespace accr {

constexpr int MT = 128;   // CTA tile (rows and columns of c)
constexpr int KT = 16;    // k slice per stage
constexpr int NTH = 256;  // threads per CTA

template <bool SERIAL>
__device__ __forceinline__ float mac(float acc, float x, float y) {
    if constexpr (SERIAL) return __fadd_rn(acc, __fmul_rn(x, y));
    else return __fmaf_rn(x, y, acc);
}

template <bool SERIAL, bool VEC>
__global__ void __launch_bounds__(NTH, 2) matmul_simt_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                                             float *__restrict__ c, int64_t len) {
    __shared__ __align__(16) float As[2][KT][MT];  // a slice, transposed: As[k][row]
    __shared__ __align__(16) float Bs[2][KT][MT];  // b slice: Bs[k][col]
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.y * MT, col0 = (int64_t)blockIdx.x * MT;

    // loaders: a 128x16 slice = 512 float4 (two per thread: rows tid>>2 and 64 + tid>>2,
    //          k (tid&3)*4); b 16x128 slice = 512 float4 (k tid>>5 and 8 + tid>>5, col (tid&31)*4)
    const int a_r = tid >> 2, a_k = (tid & 3) * 4;
    const int b_k = tid >> 5, b_c = (tid & 31) * 4;

    auto load_a = [&](int64_t k0, int half, float4 &v) {
        const int64_t r = row0 + a_r + half * 64, k = k0 + a_k;
        if (VEC && r < len && k + 3 < len) {
            v = __ldg(reinterpret_cast<const float4 *>(a + r * len + k));
        } else {
            v.x = (r < len && k + 0 < len) ? a[r * len + k + 0] : 0.f;
            v.y = (r < len && k + 1 < len) ? a[r * len + k + 1] : 0.f;
            v.z = (r < len && k + 2 < len) ? a[r * len + k + 2] : 0.f;
            v.w = (r < len && k + 3 < len) ? a[r * len + k + 3] : 0.f;
        }
    };
    auto load_b = [&](int64_t k0, int half, float4 &v) {
        const int64_t k = k0 + b_k + half * 8, cc = col0 + b_c;
        if (VEC && k < len && cc + 3 < len) {
            v = __ldg(reinterpret_cast<const float4 *>(b + k * len + cc));
        } else {
            v.x = (k < len && cc + 0 < len) ? b[k * len + cc + 0] : 0.f;
            v.y = (k < len && cc + 1 < len) ? b[k * len + cc + 1] : 0.f;
            v.z = (k < len && cc + 2 < len) ? b[k * len + cc + 2] : 0.f;
            v.w = (k < len && cc + 3 < len) ? b[k * len + cc + 3] : 0.f;
        }
    };
    auto store_tiles = [&](int buf, const float4 (&va)[2], const float4 (&vb)[2]) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            As[buf][a_k + 0][a_r + h * 64] = va[h].x;
            As[buf][a_k + 1][a_r + h * 64] = va[h].y;
            As[buf][a_k + 2][a_r + h * 64] = va[h].z;
            As[buf][a_k + 3][a_r + h * 64] = va[h].w;
            *reinterpret_cast<float4 *>(&Bs[buf][b_k + h * 8][b_c]) = vb[h];
        }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float4 va[2], vb[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        load_a(0, h, va[h]);
        load_b(0, h, vb[h]);
    }
    store_tiles(0, va, vb);
    __syncthreads();
    const int64_t nk = (len + KT - 1) / KT;
    for (int64_t kt = 0; kt < nk; ++kt) {
        const int cur = (int)(kt & 1);
        const bool more = kt + 1 < nk;
        if (more) {  // fetch the next slice while this one is used
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                load_a((kt + 1) * KT, h, va[h]);
                load_b((kt + 1) * KT, h, vb[h]);
            }
        }
        // operand fragments double-buffered in registers: k+1 is read from
        // shared memory while the 64 products of k issue
        float4 fa[2][2], fb[2][2];
        fa[0][0] = *reinterpret_cast<const float4 *>(&As[cur][0][ty * 4]);
        fa[0][1] = *reinterpret_cast<const float4 *>(&As[cur][0][64 + ty * 4]);
        fb[0][0] = *reinterpret_cast<const float4 *>(&Bs[cur][0][tx * 4]);
        fb[0][1] = *reinterpret_cast<const float4 *>(&Bs[cur][0][64 + tx * 4]);
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int p = k & 1;
            if (k + 1 < KT) {
                fa[p ^ 1][0] = *reinterpret_cast<const float4 *>(&As[cur][k + 1][ty * 4]);
                fa[p ^ 1][1] = *reinterpret_cast<const float4 *>(&As[cur][k + 1][64 + ty * 4]);
                fb[p ^ 1][0] = *reinterpret_cast<const float4 *>(&Bs[cur][k + 1][tx * 4]);
                fb[p ^ 1][1] = *reinterpret_cast<const float4 *>(&Bs[cur][k + 1][64 + tx * 4]);
            }
            const float ar[8] = {fa[p][0].x, fa[p][0].y, fa[p][0].z, fa[p][0].w,
                                 fa[p][1].x, fa[p][1].y, fa[p][1].z, fa[p][1].w};
            const float br[8] = {fb[p][0].x, fb[p][0].y, fb[p][0].z, fb[p][0].w,
                                 fb[p][1].x, fb[p][1].y, fb[p][1].z, fb[p][1].w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = mac<SERIAL>(acc[i][j], ar[i], br[j]);
        }
        if (more) store_tiles(cur ^ 1, va, vb);
        __syncthreads();
    }
    // write the 8 x 8 register block
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (r >= len) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t cc = col0 + h * 64 + tx * 4;
            float4 v = make_float4(acc[i][h * 4 + 0], acc[i][h * 4 + 1], acc[i][h * 4 + 2], acc[i][h * 4 + 3]);
            if (VEC && cc + 3 < len) {
                *reinterpret_cast<float4 *>(c + r * len + cc) = v;
            } else {
                if (cc + 0 < len) c[r * len + cc + 0] = v.x;
                if (cc + 1 < len) c[r * len + cc + 1] = v.y;
                if (cc + 2 < len) c[r * len + cc + 2] = v.z;
                if (cc + 3 < len) c[r * len + cc + 3] = v.w;
            }
        }
    }
}


// Packed pairs of floats (sm_100 family f32x2): each half is an ordinary
// round-to-nearest fused multiply-add.  Used only by the packed FP32 probe:
// measured on GB300, a packed instruction moves no more float work per clock
// than two scalar ones (the FMA pipe is the limit either way).
typedef unsigned long long f2;

__device__ __forceinline__ float lo_of(f2 v) { return __uint_as_float((unsigned)(v & 0xffffffffull)); }
__device__ __forceinline__ float hi_of(f2 v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f2 pack2(float lo, float hi) {
    return ((f2)__float_as_uint(hi) << 32) | (f2)__float_as_uint(lo);
}

// FP32 peak probe: 16 independent FMA chains per thread (latency hidden by
// the chains and by 8 warps per SM sub-partition at 4 CTAs per SM); b and c
// keep every chain bounded (x -> 0.999 x + 0.001 tends to 1).
constexpr int PROBE_THREADS = 256;

__global__ void __launch_bounds__(PROBE_THREADS) fma_probe_kernel(int64_t rounds, float *sink, float b, float c) {
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int64_t r = 0; r < rounds; ++r) {
#pragma unroll
        for (int i = 0; i < 16; ++i) a[i] = __fmaf_rn(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += a[i];
    sink[(int64_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = s * (1.f / 16.f);
}

// The same probe issuing packed pairs: 16 independent f32x2 chains per thread,
// 32 fused multiply-adds per round.  If the packed form moves more float work
// per clock than scalar instructions, this is the FP32 peak.
__global__ void __launch_bounds__(PROBE_THREADS) fma2_probe_kernel(int64_t rounds, float *sink, float b, float c) {
    f2 a[16];
    const f2 bb = pack2(b, b), cc = pack2(c, c);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float lo = (float)(threadIdx.x + i) * 1e-3f, hi = (float)(threadIdx.x + i + 16) * 1e-3f;
        a[i] = pack2(lo, hi);
    }
    for (int64_t r = 0; r < rounds; ++r) {
#pragma unroll
        for (int i = 0; i < 16; ++i) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += lo_of(a[i]) + hi_of(a[i]);
    sink[(int64_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = s * (1.f / 32.f);
}

int matmul_simt(const float *a, const float *b, float *c, int64_t len, bool serial, cudaStream_t s) {
    if (len == 0) return ACCR_OK;
    const int64_t tiles = (len + MT - 1) / MT;
    if (tiles > 65535) return set_error(ACCR_EINVAL, "accr_matmul_nest: len too large for the SIMT grid");
    dim3 grid((unsigned)tiles, (unsigned)tiles);
    // 16-byte vector access needs 16-byte aligned rows
    int rc = launch_guard("matmul_simt_kernel");
    if (rc != ACCR_OK) return rc;
    const bool vec = (len % 4 == 0) && ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0) && ((uintptr_t)c % 16 == 0);
    if (serial) {
        if (vec) matmul_simt_kernel<true, true><<<grid, NTH, 0, s>>>(a, b, c, len);
        else matmul_simt_kernel<true, false><<<grid, NTH, 0, s>>>(a, b, c, len);
    } else {
        if (vec) matmul_simt_kernel<false, true><<<grid, NTH, 0, s>>>(a, b, c, len);
        else matmul_simt_kernel<false, false><<<grid, NTH, 0, s>>>(a, b, c, len);
    }
    return launched("matmul_simt_kernel");
}

}  // namespace accr

extern "C" ACCR_API int accr_probe_fma(int32_t ctas, int64_t rounds, float *sink, accr_stream_t stream) {
    ACCR_TRACE("accr_probe_fma");
    accr::clear_error();
    if (ctas < 1 || rounds < 1 || !sink) return accr::set_error(ACCR_EINVAL, "accr_probe_fma: bad arguments");
    int rc = accr::launch_guard("fma_probe_kernel");
    if (rc != ACCR_OK) return rc;
    accr::fma_probe_kernel<<<ctas, accr::PROBE_THREADS, 0, (cudaStream_t)stream>>>(rounds, sink, 0.999f, 0.001f);
    return accr::launched("fma_probe_kernel");
}

extern "C" ACCR_API int accr_probe_fma_packed(int32_t ctas, int64_t rounds, float *sink, accr_stream_t stream) {
    ACCR_TRACE("accr_probe_fma_packed");
    accr::clear_error();
    if (ctas < 1 || rounds < 1 || !sink) return accr::set_error(ACCR_EINVAL, "accr_probe_fma_packed: bad arguments");
    int rc = accr::launch_guard("fma2_probe_kernel");
    if (rc != ACCR_OK) return rc;
    accr::fma2_probe_kernel<<<ctas, accr::PROBE_THREADS, 0, (cudaStream_t)stream>>>(rounds, sink, 0.999f, 0.001f);
    return accr::launched("fma2_probe_kernel");
}
