// common.cuh -- host-side plumbing shared by the kernels of the accr library:
// error state, launch counting, device properties and per-stream scratch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "accr.h"

namespace accr {

// ---- errors ---------------------------------------------------------------
// Records `code` and a printf-style message for accr_last_error(); returns code.
int set_error(int code, const char *fmt, ...);
// Maps a CUDA error to ACCR_ECUDA with the CUDA message; ACCR_OK if e == success.
int cuda_check(cudaError_t e, const char *where);
// Checks the launch just issued (cudaGetLastError) and counts it.
int launched(const char *what, int kernels = 1);
void clear_error();

// ---- tracing and logging ----------------------------------------------------
// Every entry point opens an NVTX range named after itself for the length of
// the call (shown by Nsight Systems and `ncu --nvtx`; with no tool attached a
// range costs one predictable branch).
struct TraceRange {
    explicit TraceRange(const char *name);
    ~TraceRange();
};
#define ACCR_TRACE(name) ::accr::TraceRange accr_trace_range_(name)
// Log level from the environment variable ACCR_LOG, read once: 0 (default)
// silent; 1 every error as it is recorded; 2 also each call's shape and the
// path it takes (grid, split form, plan size).  Lines go to stderr.
int log_level();
void log_msg(int level, const char *fmt, ...);

// ---- host-side fault injection (tests) --------------------------------------
// True if an injected fault of `kind` (ACCR_FAULT_*) fires now (and uses it up).
bool fault_take(int kind);
// Returns ACCR_ECUDA (message set) if an injected launch fault fires.
int launch_guard(const char *what);

// ---- device ---------------------------------------------------------------
struct DeviceInfo {
    int id;
    int sms;
    int l2_bytes;
    int max_smem_optin;
};
// Properties of the current device (cached per device).
const DeviceInfo &device_info();

// ---- scratch --------------------------------------------------------------
// Library-owned device memory for one (device, stream) pair, created on first
// use and kept until exit.  `counters` are zero before the first kernel and
// every kernel that takes one returns it to zero.
struct Scratch {
    unsigned *counters;  // ACCR_NUM_COUNTERS words
    void *buf;           // `bytes` bytes, 256-byte aligned
    size_t bytes;
};
constexpr int kNumCounters = 64;
// Returns scratch of at least `bytes` for `stream` on the current device.
// Growing it synchronises `stream` first.  Returns nullptr (and sets the error)
// on failure.
Scratch *scratch_for(accr_stream_t stream, size_t bytes);

// Pinned host staging of at least `bytes` for `stream` (for D2H of partials).
void *host_staging_for(accr_stream_t stream, size_t bytes);

// At least `n` device words for `stream` on the current device that are zero
// whenever no kernel is using them: cleared on the stream when created or
// grown, and every kernel that takes them returns each word it touched to
// zero before it exits.  Returns nullptr (and sets the error) on failure.
unsigned *zeroed_words_for(accr_stream_t stream, size_t n);

// ---- types ----------------------------------------------------------------
inline int type_bytes(int t) { return (t == ACCR_I32 || t == ACCR_F32) ? 4 : 8; }
inline bool type_is_int(int t) { return t == ACCR_I32 || t == ACCR_I64; }
inline bool type_valid(int t) { return t >= ACCR_I32 && t <= ACCR_F64; }

}  // namespace accr

namespace accr {
struct ClauseDev;
// Checks the clauses of one region against its element type and lowers each
// to its device form (working code, identity, prior value).  Returns ACCR_OK,
// ACCR_EINVAL or ACCR_ETYPE (with the message set).
int lower_clauses(int in_type, const accr_clause *c, int nc, unsigned flags, ClauseDev *dev);
}  // namespace accr
