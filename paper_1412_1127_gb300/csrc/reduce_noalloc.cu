// reduce_noalloc.cu -- accr_reduce for callers that cannot call cudaMalloc.
//
// Some callers cannot let a library allocate device memory: processes that
// hand all device memory to their own pool or arena up front, and
// latency-sensitive loops that cannot afford the device-wide synchronisation
// cudaMalloc and cudaFree can cause.  accr_reduce takes its scratch (the block
// partials and the last-block-done counter) from a per-stream cache it
// allocates on first use; this entry point instead uses one fixed array
// compiled into the library, so it allocates nothing.
//
// The array is a file-scope __device__ variable of ACCR_NOALLOC_SCRATCH_BYTES
// bytes.  Every GPU that loads the library holds it until the process exits.
// In host code its name only stands in for the device variable, so the
// device address is looked up once per device with cudaGetSymbolAddress (on
// the first call made with that device current) and cached for the life of
// the process, so calls after cudaDeviceReset on that device are not valid.
//
// All calls share the array: calls that overlap on the GPU (on different
// streams, or from different threads) race on it and give wrong results.  The
// counter is cleared on the caller's stream before every launch, so a call
// never depends on what an earlier call left behind.
#include <mutex>

#include "common.cuh"
#include "fold.cuh"

namespace accr {

// Defined in reduce.cu.
int reduce_grid(int in_type, int nc, int64_t n);
int reduce_launch(const void *in, int64_t n, int in_type, const ClauseDev *cl, int nc, int two_level,
                  Partial *partials, unsigned *counter, int grid, cudaStream_t s);

constexpr size_t kNoallocCounterBytes = 256;

// [0, 256): the last-block-done counter; [256, 256 + ACCR_NOALLOC_SCRATCH_BYTES): partials.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocCounterBytes + ACCR_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];

// Device address of the array on the current device (looked up once per device).
static int noalloc_scratch(void **addr) {
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "accr_reduce_noalloc: cudaGetDevice");
    if (rc != ACCR_OK) return rc;
    if (dev < 0 || dev >= 64) return set_error(ACCR_EINVAL, "accr_reduce_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "accr_reduce_noalloc: cudaGetSymbolAddress");
        if (rc != ACCR_OK) return rc;
        g_noalloc_addr[dev] = p;
    }
    *addr = g_noalloc_addr[dev];
    return ACCR_OK;
}

}  // namespace accr

using namespace accr;

extern "C" ACCR_API int accr_reduce_noalloc(const void *in, int64_t n, int32_t in_type,
                                            const accr_clause *clauses, int32_t nclauses, uint32_t flags,
                                            accr_stream_t stream) {
    ACCR_TRACE("accr_reduce_noalloc");
    clear_error();
    if (flags & ~(ACCR_COMPENSATED | ACCR_SYNC))
        return set_error(ACCR_EINVAL, "accr_reduce_noalloc: unsupported flags 0x%x (only ACCR_COMPENSATED, "
                         "ACCR_SYNC; the two-level host form needs a pinned buffer)", flags);
    if (n < 0) return set_error(ACCR_EINVAL, "accr_reduce_noalloc: n = %lld < 0", (long long)n);
    ClauseDev cl[ACCR_MAX_CLAUSES];
    int rc = lower_clauses(in_type, clauses, nclauses, flags, cl);
    if (rc != ACCR_OK) return rc;
    if (n > 0 && !in) return set_error(ACCR_EINVAL, "accr_reduce_noalloc: in is NULL");
    if (((uintptr_t)in % (uintptr_t)type_bytes(in_type)) != 0)
        return set_error(ACCR_EINVAL, "accr_reduce_noalloc: in is not aligned to its element size");
    // same grid as accr_reduce, so both give the same bits
    const int grid = reduce_grid(in_type, nclauses, n);
    const size_t need = (size_t)nclauses * (size_t)grid * sizeof(Partial);
    if (need > (size_t)ACCR_NOALLOC_SCRATCH_BYTES)
        return set_error(ACCR_EINVAL, "accr_reduce_noalloc: %d clauses over %d blocks need %zu bytes of "
                         "scratch, more than the fixed %d", nclauses, grid, need, ACCR_NOALLOC_SCRATCH_BYTES);
    void *base = nullptr;
    rc = noalloc_scratch(&base);
    if (rc != ACCR_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *counter = (unsigned *)base;
    Partial *partials = (Partial *)((unsigned char *)base + kNoallocCounterBytes);
    rc = cuda_check(cudaMemsetAsync(counter, 0, sizeof(unsigned), s), "accr_reduce_noalloc: clear counter");
    if (rc != ACCR_OK) return rc;
    rc = reduce_launch(in, n, in_type, cl, nclauses, 0, partials, counter, grid, s);
    if (rc != ACCR_OK) return rc;
    if (flags & ACCR_SYNC) return cuda_check(cudaStreamSynchronize(s), "accr_reduce_noalloc: sync");
    return ACCR_OK;
}
