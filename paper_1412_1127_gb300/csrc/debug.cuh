// debug.cuh -- bounds checks of ACCR_DEBUG builds.
//
// A debug build (`build(debug=True)`: libaccr_debug.so, -DACCR_DEBUG) checks
// the index of every global store of the row, batched-region, k-nearest and
// tensor-core kernels (and the chunk bounds of the split rows) against the
// bound the host computed.  A failed check does not trap: it counts the
// violation in a status word of its translation unit, records the first
// failing site, and skips the access.  accr_debug_report() reads and clears
// the words.  In release builds ACCR_DCHECK is `true` and nothing is emitted.
#pragma once

#include "common.cuh"

namespace accr {

// Sites (the first failing one is reported).
enum DebugSite : unsigned {
    DS_ROW_VAR = 1,        // row nest: variable index < rows
    DS_ROW_PARTIAL = 2,    // split rows: partial slot < rows x clauses x chunks
    DS_ROW_COUNTER = 3,    // split rows: row counter < rows
    DS_ROW_CHUNK = 4,      // split rows: chunk end <= cols
    DS_BATCH_TILE = 5,     // batch: tile of a region < the region's tiles
    DS_BATCH_SLOT = 6,     // batch: partial slot < all tiles' slots
    DS_BATCH_REGION = 7,   // batch: region index < descriptors
    DS_NEAREST_SLOT = 8,   // k-nearest: partial slot < CTAs x list length
    DS_NEAREST_OUT = 9,    // k-nearest: output index < k
    DS_GEMM_STORE = 10,    // BF16x3 epilogue: row < M and columns < N
};

// Host side (runtime.cu): each translation unit with checks registers a
// reader of its status word.
typedef int (*DebugReader)(unsigned long long *count, unsigned long long *first_site, bool clear);
void debug_register(DebugReader reader);

}  // namespace accr

#ifdef ACCR_DEBUG
namespace {
// [0] violations, [1] first failing site (0: none) -- one pair per translation unit
__device__ unsigned long long accr_dbg_word[2];

__device__ __noinline__ bool accr_dcheck_fail(unsigned site) {
    atomicAdd(&accr_dbg_word[0], 1ull);
    atomicCAS(&accr_dbg_word[1], 0ull, (unsigned long long)site);
    return false;
}

int accr_dbg_read(unsigned long long *count, unsigned long long *site, bool clear) {
    unsigned long long w[2] = {0, 0};
    if (cudaMemcpyFromSymbol(w, accr_dbg_word, sizeof w) != cudaSuccess) return ACCR_ECUDA;
    *count = w[0];
    *site = w[1];
    if (clear) {
        const unsigned long long z[2] = {0, 0};
        if (cudaMemcpyToSymbol(accr_dbg_word, z, sizeof z) != cudaSuccess) return ACCR_ECUDA;
    }
    return ACCR_OK;
}

struct AccrDbgRegistrar {
    AccrDbgRegistrar() { accr::debug_register(accr_dbg_read); }
};
AccrDbgRegistrar accr_dbg_registrar;
}  // namespace
#define ACCR_DCHECK(cond, site) ((cond) ? true : accr_dcheck_fail(site))
#else
#define ACCR_DCHECK(cond, site) true
#endif
