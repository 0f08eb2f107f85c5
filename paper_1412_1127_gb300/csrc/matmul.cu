// matmul.cu -- C-ABI entry of the Listing-1a nest (IPMACC Sec. 1.3).
#include "common.cuh"

namespace accr {
int matmul_simt(const float *a, const float *b, float *c, int64_t len, bool serial, cudaStream_t s);
int matmul_bf16x3(const float *a, const float *b, float *c, int64_t len, cudaStream_t s, bool sync, bool reuse);
}  // namespace accr

using namespace accr;

extern "C" ACCR_API int accr_matmul_nest(const float *a, const float *b, float *c, int64_t len, int32_t mode,
                                         uint32_t flags, accr_stream_t stream) {
    ACCR_TRACE("accr_matmul_nest");
    clear_error();
    if (len < 0) return set_error(ACCR_EINVAL, "accr_matmul_nest: len < 0");
    if (flags & ~(ACCR_SYNC | ACCR_MM_REUSE_SPLIT))
        return set_error(ACCR_EINVAL, "accr_matmul_nest: unsupported flags 0x%x", flags);
    if (len > 0 && (!a || !b || !c)) return set_error(ACCR_EINVAL, "accr_matmul_nest: NULL matrix");
    if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 3)
        return set_error(ACCR_EINVAL, "accr_matmul_nest: matrices must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    log_msg(2, "accr_matmul_nest: len=%lld mode=%d%s", (long long)len, mode,
            (flags & ACCR_MM_REUSE_SPLIT) ? " (split reused if the operands are unchanged)" : "");
    int rc;
    switch (mode) {
    case ACCR_MM_SIMT: rc = matmul_simt(a, b, c, len, false, s); break;
    case ACCR_MM_SIMT_SERIAL: rc = matmul_simt(a, b, c, len, true, s); break;
    case ACCR_MM_BF16X3:
        return matmul_bf16x3(a, b, c, len, s, (flags & ACCR_SYNC) != 0, (flags & ACCR_MM_REUSE_SPLIT) != 0);
    default: return set_error(ACCR_EINVAL, "accr_matmul_nest: unknown mode %d", mode);
    }
    if (rc != ACCR_OK) return rc;
    if (flags & ACCR_SYNC) return cuda_check(cudaStreamSynchronize(s), "accr_matmul_nest: sync");
    return ACCR_OK;
}
