// fold.cuh -- device side of the reduction clause (IPMACC Stage 3.4 item iii,
// Stage 3.7): what one thread folds per element, how two partial results
// merge, and how the merged result meets the variable's prior value.
//
// A clause (op, element type, variable type) is lowered on the host to a
// "working code": the per-element operation in the narrowest exact width.
// Integer max/min/&/|/^/&&/|| work in the element's width and are widened at
// the end (sign extension commutes with them); + and * work in the variable's
// width.  Floating-point max/min work on order-preserving integer keys, which
// order -0 below +0 and are exact.  Float + may be compensated (Neumaier per
// thread, TwoSum when merging, double for the cross-gang merge).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "accr.h"

namespace accr {

enum WCode : int {
    W_ADD32 = 0,  // integer + modulo 2^32
    W_ADD64,      // integer + modulo 2^64 (int32 elements sign-extended)
    W_MUL32,      // integer * modulo 2^32
    W_MUL64,      // integer * modulo 2^64
    W_MAXI,       // signed max in the element's width
    W_MINI,       // signed min in the element's width
    W_AND,        // bitwise, element width
    W_OR,
    W_XOR,
    W_LAND,       // 0/1 flag: all elements nonzero
    W_LOR,        // 0/1 flag: some element nonzero
    W_ADDF,       // float + in the element's type
    W_ADDF_COMP,  // float + compensated: (s, c) pairs
    W_ADDF_WIDE,  // float elements summed in double
    W_MULF,       // float * in the element's type
    W_MULF_WIDE,  // float elements multiplied in double
    W_MAXF,       // max over order-preserving keys, element width
    W_MINF,       // min over order-preserving keys, element width
    W_COUNT
};

// Per-clause description passed to kernels by value.
struct ClauseDev {
    int wcode;       // WCode
    int op;          // accr_op
    int acc_type;    // accr_type of the variable
    int pad;
    uint64_t init;   // variable's prior value (bits in acc_type); identity if none
    uint64_t ident;  // identity of the working code (bits of the working slot)
    void *out;       // device pointer of the variable (array for row/segment forms)
};

// A private accumulator: a 64-bit slot (integer bits, float bits, double bits
// or a key) plus the compensation term of compensated float sums.
struct Acc {
    uint64_t a;
    float c;
};

// Partial results in global memory: 16 bytes each.
struct __align__(16) Partial {
    uint64_t a;
    float c;
    uint32_t pad;
};

// ---- bit helpers -------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t f2u(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
__host__ __device__ __forceinline__ uint64_t d2u(double d) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t u;
    memcpy(&u, &d, 8);
    return u;
#endif
}
__host__ __device__ __forceinline__ double u2d(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, 8);
    return d;
#endif
}

// Round-to-nearest arithmetic usable on both sides (the host path merges the
// block partials of the two-level form).  No multiply-add contraction.
__host__ __device__ __forceinline__ float hd_fadd(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    volatile float r = a + b;
    return r;
#endif
}
__host__ __device__ __forceinline__ float hd_fsub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    volatile float r = a - b;
    return r;
#endif
}
__host__ __device__ __forceinline__ float hd_fmul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    volatile float r = a * b;
    return r;
#endif
}
__host__ __device__ __forceinline__ double hd_dadd(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    volatile double r = a + b;
    return r;
#endif
}
__host__ __device__ __forceinline__ double hd_dmul(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    volatile double r = a * b;
    return r;
#endif
}

// Order-preserving keys: signed integer compare of keys equals the numeric
// order of the floats, with -0 < +0 (NaN excluded).  The map is an involution.
__host__ __device__ __forceinline__ int32_t fkey32(uint32_t b) {
    const int32_t s = (int32_t)b;
    return s ^ (int32_t)((uint32_t)(s >> 31) >> 1);  // negative: flip all but the sign bit
}
__host__ __device__ __forceinline__ int64_t fkey64(uint64_t b) {
    const int64_t s = (int64_t)b;
    return s ^ (int64_t)((uint64_t)(s >> 63) >> 1);
}

template <typename T>
__device__ __forceinline__ T from_bits32(uint32_t u) {
    if constexpr (std::is_same<T, float>::value) return __uint_as_float(u);
    else return (T)(int32_t)u;
}
template <typename T>
__device__ __forceinline__ T from_bits64(uint64_t u) {
    if constexpr (std::is_same<T, double>::value) return __longlong_as_double((long long)u);
    else return (T)(int64_t)u;
}

// Element k of a 16-byte vector (k a compile-time constant after unrolling).
__device__ __forceinline__ uint32_t word32(const uint4 &v, int k) {
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}
__device__ __forceinline__ uint64_t word64(const uint4 &v, int k) {
    return k == 0 ? (((uint64_t)v.y << 32) | v.x) : (((uint64_t)v.w << 32) | v.z);
}

template <typename T, int NV, typename F>
__device__ __forceinline__ void for_each_elem(const uint4 *v, F &&f) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int k = 0; k < 4; ++k) f(from_bits32<T>(word32(v[i], k)));
        } else {
#pragma unroll
            for (int k = 0; k < 2; ++k) f(from_bits64<T>(word64(v[i], k)));
        }
    }
}

// Neumaier step: (s, c) += x.
__device__ __forceinline__ void neumaier(float &s, float &c, float x) {
    float t = __fadd_rn(s, x);
    float big = fabsf(s) >= fabsf(x) ? s : x;
    float small = fabsf(s) >= fabsf(x) ? x : s;
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(big, t), small));
    s = t;
}

// TwoSum merge of two compensated pairs.
__host__ __device__ __forceinline__ void two_sum_merge(float &s, float &c, float s2, float c2) {
    float t = hd_fadd(s, s2);
    float bp = hd_fsub(t, s);
    float e = hd_fadd(hd_fsub(s, hd_fsub(t, bp)), hd_fsub(s2, bp));
    s = t;
    c = hd_fadd(hd_fadd(c, c2), e);
}

// Sum of the 2*NV doubles of a chunk.  GB300's FP64 pipe retires about two
// adds per SM per clock, too few for a double sum at HBM rate, so chunks of
// 8 or more values are summed in integer block floating point: each
// significand (with its implicit bit) is aligned to the chunk's largest
// exponent with 6 guard bits, the aligned magnitudes are added in an int64
// with their signs, and the total is converted and scaled by an exact power
// of two -- three FP64-pipe operations per chunk instead of one per value.
// Bits shifted out are truncated: at most 2^-6 of the largest value's ulp per
// element (under 0.25 ulp for a chunk of 16).  Chunks whose largest exponent
// is within 60 of the subnormal range, and short chunks, are added as
// doubles.  Finite inputs only.
template <int NV>
__device__ __forceinline__ double chunk_sum_f64(const uint4 *v) {
    constexpr int E = 2 * NV;
    uint64_t b[E];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        b[2 * i] = word64(v[i], 0);
        b[2 * i + 1] = word64(v[i], 1);
    }
    if constexpr (E < 8) {
        double t = u2d(b[0]);
#pragma unroll
        for (int j = 1; j < E; ++j) t = __dadd_rn(t, u2d(b[j]));
        return t;
    } else {
        int ex[E];
        int emax = 1;
#pragma unroll
        for (int j = 0; j < E; ++j) {
            ex[j] = (int)((b[j] >> 52) & 0x7ffu);
            emax = ex[j] > emax ? ex[j] : emax;
        }
        if (emax < 61) {  // tiny values: the scale below would leave the normal range
            double t = u2d(b[0]);
#pragma unroll
            for (int j = 1; j < E; ++j) t = __dadd_rn(t, u2d(b[j]));
            return t;
        }
        int64_t S = 0;
#pragma unroll
        for (int j = 0; j < E; ++j) {
            uint64_t m = b[j] & 0x000FFFFFFFFFFFFFull;
            int e = ex[j];
            if (e) m |= 0x0010000000000000ull;
            else e = 1;
            const int sh = emax - e;
            const int64_t mag = sh < 64 ? (int64_t)((m << 6) >> sh) : 0;
            S += (b[j] >> 63) ? -mag : mag;
        }
        // S counts units of 2^(emax - 1075 - 6); that power of two is normal here
        const double scale = u2d((uint64_t)(emax - 1081 + 1023) << 52);
        return __dmul_rn(__ll2double_rn((long long)S), scale);
    }
}

// ---- per-element folding -------------------------------------------------------
// Fold NV 16-byte vectors of T into A under working code w (warp-uniform).
template <typename T, int NV>
__device__ __forceinline__ void fold_vec(int w, Acc &A, const uint4 *v) {
    if constexpr (std::is_integral<T>::value) {
        using UT = typename std::make_unsigned<T>::type;
        switch (w) {
        case W_ADD32: {
            uint32_t a = (uint32_t)A.a;
            for_each_elem<T, NV>(v, [&](T x) { a += (uint32_t)x; });
            A.a = a;
        } break;
        case W_ADD64: {
            uint64_t a = A.a;
            for_each_elem<T, NV>(v, [&](T x) { a += (uint64_t)(int64_t)x; });
            A.a = a;
        } break;
        case W_MUL32: {
            uint32_t a = (uint32_t)A.a;
            for_each_elem<T, NV>(v, [&](T x) { a *= (uint32_t)x; });
            A.a = a;
        } break;
        case W_MUL64: {
            uint64_t a = A.a;
            for_each_elem<T, NV>(v, [&](T x) { a *= (uint64_t)(int64_t)x; });
            A.a = a;
        } break;
        case W_MAXI: {
            T a = (T)(UT)A.a;
            for_each_elem<T, NV>(v, [&](T x) { a = x > a ? x : a; });
            A.a = (uint64_t)(UT)a;
        } break;
        case W_MINI: {
            T a = (T)(UT)A.a;
            for_each_elem<T, NV>(v, [&](T x) { a = x < a ? x : a; });
            A.a = (uint64_t)(UT)a;
        } break;
        case W_AND: {
            UT a = (UT)A.a;
            for_each_elem<T, NV>(v, [&](T x) { a &= (UT)x; });
            A.a = a;
        } break;
        case W_OR: {
            UT a = (UT)A.a;
            for_each_elem<T, NV>(v, [&](T x) { a |= (UT)x; });
            A.a = a;
        } break;
        case W_XOR: {
            UT a = (UT)A.a;
            for_each_elem<T, NV>(v, [&](T x) { a ^= (UT)x; });
            A.a = a;
        } break;
        case W_LAND: {
            uint32_t f = (uint32_t)A.a;
            for_each_elem<T, NV>(v, [&](T x) { f &= (uint32_t)(x != 0); });
            A.a = f;
        } break;
        case W_LOR: {
            uint32_t f = (uint32_t)A.a;
            for_each_elem<T, NV>(v, [&](T x) { f |= (uint32_t)(x != 0); });
            A.a = f;
        } break;
        default: break;
        }
    } else {
        constexpr bool F32 = std::is_same<T, float>::value;
        switch (w) {
        case W_ADDF: {
            if constexpr (F32) {
                // one partial sum per vector slot: dependency chains of NV
                // adds instead of 4 NV, merged pairwise at the end
                float p0 = u2f((uint32_t)A.a), p1 = -0.f, p2 = -0.f, p3 = -0.f;
#pragma unroll
                for (int i = 0; i < NV; ++i) {
                    p0 = p0 + __uint_as_float(v[i].x);
                    p1 = p1 + __uint_as_float(v[i].y);
                    p2 = p2 + __uint_as_float(v[i].z);
                    p3 = p3 + __uint_as_float(v[i].w);
                }
                A.a = f2u((p0 + p1) + (p2 + p3));
            } else {
                A.a = d2u(__dadd_rn(u2d(A.a), chunk_sum_f64<NV>(v)));
            }
        } break;
        case W_ADDF_COMP: {
            if constexpr (F32) {
                float s = u2f((uint32_t)A.a), c = A.c;
                for_each_elem<T, NV>(v, [&](T x) { neumaier(s, c, x); });
                A.a = f2u(s);
                A.c = c;
            }
        } break;
        case W_ADDF_WIDE: {
            double a = u2d(A.a);
            for_each_elem<T, NV>(v, [&](T x) { a = __dadd_rn(a, (double)x); });
            A.a = d2u(a);
        } break;
        case W_MULF: {
            T a = F32 ? (T)u2f((uint32_t)A.a) : (T)u2d(A.a);
            for_each_elem<T, NV>(v, [&](T x) { a = a * x; });
            if constexpr (F32) A.a = f2u((float)a); else A.a = d2u((double)a);
        } break;
        case W_MULF_WIDE: {
            double a = u2d(A.a);
            for_each_elem<T, NV>(v, [&](T x) { a = __dmul_rn(a, (double)x); });
            A.a = d2u(a);
        } break;
        case W_MAXF: {
            if constexpr (F32) {  // four independent key chains, as for the sum
                int32_t a0 = (int32_t)(uint32_t)A.a, a1 = a0, a2 = a0, a3 = a0;
#pragma unroll
                for (int i = 0; i < NV; ++i) {
                    a0 = max(a0, fkey32(v[i].x));
                    a1 = max(a1, fkey32(v[i].y));
                    a2 = max(a2, fkey32(v[i].z));
                    a3 = max(a3, fkey32(v[i].w));
                }
                A.a = (uint32_t)max(max(a0, a1), max(a2, a3));
            } else {
                int64_t a = (int64_t)A.a;
                for_each_elem<T, NV>(v, [&](T x) {
                    int64_t k = fkey64((uint64_t)__double_as_longlong(x));
                    a = k > a ? k : a;
                });
                A.a = (uint64_t)a;
            }
        } break;
        case W_MINF: {
            if constexpr (F32) {
                int32_t a0 = (int32_t)(uint32_t)A.a, a1 = a0, a2 = a0, a3 = a0;
#pragma unroll
                for (int i = 0; i < NV; ++i) {
                    a0 = min(a0, fkey32(v[i].x));
                    a1 = min(a1, fkey32(v[i].y));
                    a2 = min(a2, fkey32(v[i].z));
                    a3 = min(a3, fkey32(v[i].w));
                }
                A.a = (uint32_t)min(min(a0, a1), min(a2, a3));
            } else {
                int64_t a = (int64_t)A.a;
                for_each_elem<T, NV>(v, [&](T x) {
                    int64_t k = fkey64((uint64_t)__double_as_longlong(x));
                    a = k < a ? k : a;
                });
                A.a = (uint64_t)a;
            }
        } break;
        default: break;
        }
    }
}

// Fold one scalar element (unaligned heads and ragged tails).
template <typename T>
__device__ __forceinline__ void fold_one(int w, Acc &A, T x) {
    if constexpr (std::is_integral<T>::value) {
        using UT = typename std::make_unsigned<T>::type;
        switch (w) {
        case W_ADD32: A.a = (uint32_t)((uint32_t)A.a + (uint32_t)x); break;
        case W_ADD64: A.a = A.a + (uint64_t)(int64_t)x; break;
        case W_MUL32: A.a = (uint32_t)((uint32_t)A.a * (uint32_t)x); break;
        case W_MUL64: A.a = A.a * (uint64_t)(int64_t)x; break;
        case W_MAXI: { T a = (T)(UT)A.a; A.a = (uint64_t)(UT)(x > a ? x : a); } break;
        case W_MINI: { T a = (T)(UT)A.a; A.a = (uint64_t)(UT)(x < a ? x : a); } break;
        case W_AND: A.a = (UT)((UT)A.a & (UT)x); break;
        case W_OR: A.a = (UT)((UT)A.a | (UT)x); break;
        case W_XOR: A.a = (UT)((UT)A.a ^ (UT)x); break;
        case W_LAND: A.a = (uint32_t)A.a & (uint32_t)(x != 0); break;
        case W_LOR: A.a = (uint32_t)A.a | (uint32_t)(x != 0); break;
        default: break;
        }
    } else {
        constexpr bool F32 = std::is_same<T, float>::value;
        switch (w) {
        case W_ADDF:
            if constexpr (F32) A.a = f2u(__fadd_rn(u2f((uint32_t)A.a), (float)x));
            else A.a = d2u(__dadd_rn(u2d(A.a), (double)x));
            break;
        case W_ADDF_COMP:
            if constexpr (F32) {
                float s = u2f((uint32_t)A.a), c = A.c;
                neumaier(s, c, (float)x);
                A.a = f2u(s);
                A.c = c;
            }
            break;
        case W_ADDF_WIDE: A.a = d2u(__dadd_rn(u2d(A.a), (double)x)); break;
        case W_MULF:
            if constexpr (F32) A.a = f2u(__fmul_rn(u2f((uint32_t)A.a), (float)x));
            else A.a = d2u(__dmul_rn(u2d(A.a), (double)x));
            break;
        case W_MULF_WIDE: A.a = d2u(__dmul_rn(u2d(A.a), (double)x)); break;
        case W_MAXF:
            if constexpr (F32) {
                int32_t a = (int32_t)(uint32_t)A.a, k = fkey32(__float_as_uint((float)x));
                A.a = (uint32_t)(k > a ? k : a);
            } else {
                int64_t a = (int64_t)A.a, k = fkey64((uint64_t)__double_as_longlong((double)x));
                A.a = (uint64_t)(k > a ? k : a);
            }
            break;
        case W_MINF:
            if constexpr (F32) {
                int32_t a = (int32_t)(uint32_t)A.a, k = fkey32(__float_as_uint((float)x));
                A.a = (uint32_t)(k < a ? k : a);
            } else {
                int64_t a = (int64_t)A.a, k = fkey64((uint64_t)__double_as_longlong((double)x));
                A.a = (uint64_t)(k < a ? k : a);
            }
            break;
        default: break;
        }
    }
}

// ---- merging two partial results ------------------------------------------------
// `elem64`: the element (and so the working slot) is 64 bits wide.
__host__ __device__ __forceinline__ void merge(int w, bool elem64, Acc &A, const Acc &B) {
    switch (w) {
    case W_ADD32: A.a = (uint32_t)((uint32_t)A.a + (uint32_t)B.a); break;
    case W_ADD64: A.a = A.a + B.a; break;
    case W_MUL32: A.a = (uint32_t)((uint32_t)A.a * (uint32_t)B.a); break;
    case W_MUL64: A.a = A.a * B.a; break;
    case W_MAXI:
        if (elem64) A.a = (int64_t)B.a > (int64_t)A.a ? B.a : A.a;
        else A.a = (int32_t)(uint32_t)B.a > (int32_t)(uint32_t)A.a ? B.a : A.a;
        break;
    case W_MINI:
        if (elem64) A.a = (int64_t)B.a < (int64_t)A.a ? B.a : A.a;
        else A.a = (int32_t)(uint32_t)B.a < (int32_t)(uint32_t)A.a ? B.a : A.a;
        break;
    case W_AND: A.a &= B.a; break;
    case W_OR: A.a |= B.a; break;
    case W_XOR: A.a ^= B.a; break;
    case W_LAND: A.a &= B.a; break;
    case W_LOR: A.a |= B.a; break;
    case W_ADDF:
        if (elem64) A.a = d2u(hd_dadd(u2d(A.a), u2d(B.a)));
        else A.a = f2u(hd_fadd(u2f((uint32_t)A.a), u2f((uint32_t)B.a)));
        break;
    case W_ADDF_COMP: {
        float s = u2f((uint32_t)A.a), c = A.c;
        two_sum_merge(s, c, u2f((uint32_t)B.a), B.c);
        A.a = f2u(s);
        A.c = c;
    } break;
    case W_ADDF_WIDE: A.a = d2u(hd_dadd(u2d(A.a), u2d(B.a))); break;
    case W_MULF:
        if (elem64) A.a = d2u(hd_dmul(u2d(A.a), u2d(B.a)));
        else A.a = f2u(hd_fmul(u2f((uint32_t)A.a), u2f((uint32_t)B.a)));
        break;
    case W_MULF_WIDE: A.a = d2u(hd_dmul(u2d(A.a), u2d(B.a))); break;
    case W_MAXF:
        if (elem64) A.a = (int64_t)B.a > (int64_t)A.a ? B.a : A.a;
        else A.a = (int32_t)(uint32_t)B.a > (int32_t)(uint32_t)A.a ? B.a : A.a;
        break;
    case W_MINF:
        if (elem64) A.a = (int64_t)B.a < (int64_t)A.a ? B.a : A.a;
        else A.a = (int32_t)(uint32_t)B.a < (int32_t)(uint32_t)A.a ? B.a : A.a;
        break;
    default: break;
    }
}

__device__ __forceinline__ Acc shfl_xor_acc(const Acc &A, int m) {
    Acc B;
    B.a = __shfl_xor_sync(0xffffffffu, (unsigned long long)A.a, m);
    B.c = __shfl_xor_sync(0xffffffffu, A.c, m);
    return B;
}

// Butterfly merge across the 32 lanes of a warp (every lane ends with the total).
__device__ __forceinline__ void warp_merge(int w, bool elem64, Acc &A) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        Acc B = shfl_xor_acc(A, m);
        // combine in a lane-independent order so all lanes hold identical bits
        Acc lo = (threadIdx.x & m) ? B : A;
        Acc hi = (threadIdx.x & m) ? A : B;
        merge(w, elem64, lo, hi);
        A = lo;
    }
}

// Merge one accumulator per clause across a CTA of NT threads (all threads
// call it); thread 0 ends with the totals.  `sh` is NC x NT/32 shared slots.
template <int NC, int NT>
__device__ __forceinline__ void cta_merge(const int (&w)[NC], const uint64_t (&ident)[NC], bool e64,
                                          Acc (&A)[NC], Acc (*sh)[NT / 32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        warp_merge(w[c], e64, A[c]);
        if (lane == 0) sh[c][warp] = A[c];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            Acc B;
            if (lane < NT / 32) B = sh[c][lane];
            else { B.a = ident[c]; B.c = 0.f; }
            warp_merge(w[c], e64, B);
            A[c] = B;
        }
    }
    __syncthreads();
}

// The cross-gang merge of compensated sums runs in double: each (s, c) pair
// becomes s + c in double and the doubles are added.
__host__ __device__ __forceinline__ int final_code(int w) { return w == W_ADDF_COMP ? W_ADDF_WIDE : w; }
__host__ __device__ __forceinline__ uint64_t final_ident(const ClauseDev &cl) {
    return cl.wcode == W_ADDF_COMP ? d2u(-0.0) : cl.ident;
}
__host__ __device__ __forceinline__ Acc to_final(int w, const Acc &A) {
    if (w != W_ADDF_COMP) return A;
    Acc B;
    B.a = d2u(hd_dadd((double)u2f((uint32_t)A.a), (double)A.c));
    B.c = 0.f;
    return B;
}

// The merged working value `tot` (in final_code(w)) meets the variable's prior
// value: var = init (op) tot, computed in the variable's type.  n == 0 leaves
// the variable as it was.  Returns the variable's bits.
__host__ __device__ __forceinline__ uint64_t finish(const ClauseDev &cl, bool elem64, bool n_zero,
                                          const Acc &tot) {
    if (n_zero) return cl.init;
    const int w = cl.wcode;
    const bool acc64 = cl.acc_type == ACCR_I64 || cl.acc_type == ACCR_F64;
    if (cl.acc_type == ACCR_I32 || cl.acc_type == ACCR_I64) {
        // the total in the variable's width (int32 working values sign-extend)
        uint64_t t = tot.a;
        if (!elem64 && acc64 && w != W_ADD64 && w != W_MUL64) t = (uint64_t)(int64_t)(int32_t)(uint32_t)t;
        uint64_t i = cl.init, r = 0;
        switch (cl.op) {
        case ACCR_ADD: r = i + t; break;
        case ACCR_MUL: r = i * t; break;
        case ACCR_MAX:
            r = acc64 ? ((int64_t)t > (int64_t)i ? t : i)
                      : ((int32_t)(uint32_t)t > (int32_t)(uint32_t)i ? t : i);
            break;
        case ACCR_MIN:
            r = acc64 ? ((int64_t)t < (int64_t)i ? t : i)
                      : ((int32_t)(uint32_t)t < (int32_t)(uint32_t)i ? t : i);
            break;
        case ACCR_BAND: r = i & t; break;
        case ACCR_BOR: r = i | t; break;
        case ACCR_BXOR: r = i ^ t; break;
        case ACCR_LAND: r = (acc64 ? i != 0 : (uint32_t)i != 0) && t != 0; break;
        case ACCR_LOR: r = (acc64 ? i != 0 : (uint32_t)i != 0) || t != 0; break;
        }
        return acc64 ? r : (uint64_t)(uint32_t)r;
    }
    // floating point
    if (cl.acc_type == ACCR_F32) {
        float i = u2f((uint32_t)cl.init), v;
        switch (w) {
        case W_ADDF: v = hd_fadd(i, u2f((uint32_t)tot.a)); break;
        case W_ADDF_COMP: v = (float)hd_dadd((double)i, u2d(tot.a)); break;
        case W_MULF: v = hd_fmul(i, u2f((uint32_t)tot.a)); break;
        case W_MAXF: {
            int32_t k = (int32_t)(uint32_t)tot.a, ki = fkey32(f2u(i));
            v = u2f((uint32_t)fkey32((uint32_t)(k > ki ? k : ki)));
        } break;
        case W_MINF: {
            int32_t k = (int32_t)(uint32_t)tot.a, ki = fkey32(f2u(i));
            v = u2f((uint32_t)fkey32((uint32_t)(k < ki ? k : ki)));
        } break;
        default: v = i; break;
        }
        return f2u(v);
    }
    double i = u2d(cl.init), v;
    switch (w) {
    case W_ADDF:
    case W_ADDF_WIDE: v = hd_dadd(i, u2d(tot.a)); break;
    case W_MULF:
    case W_MULF_WIDE: v = hd_dmul(i, u2d(tot.a)); break;
    case W_MAXF:
    case W_MINF: {
        // the key is in the element's width; bring the element to double first
        double x = elem64 ? u2d((uint64_t)fkey64(tot.a))
                          : (double)u2f((uint32_t)fkey32((uint32_t)tot.a));
        int64_t k = fkey64(d2u(x)), ki = fkey64(d2u(i));
        int64_t r = (w == W_MAXF) ? (k > ki ? k : ki) : (k < ki ? k : ki);
        v = u2d((uint64_t)fkey64((uint64_t)r));
    } break;
    default: v = i; break;
    }
    return d2u(v);
}

// Stores a variable's bits (4 or 8 bytes by type) at element `idx` of out.
__device__ __forceinline__ void store_var(const ClauseDev &cl, int64_t idx, uint64_t bits) {
    if (cl.acc_type == ACCR_I32 || cl.acc_type == ACCR_F32)
        ((uint32_t *)cl.out)[idx] = (uint32_t)bits;
    else
        ((uint64_t *)cl.out)[idx] = bits;
}

}  // namespace accr
