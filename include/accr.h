/*
 * accr.h -- C ABI of the GB300 runtime for the device side of an OpenACC
 * accelerator region (IPMACC, arXiv 1412.1127).
 *
 * A call is one region (Sec. 1.3: the `kernels` directive marks a region for
 * the accelerator): arrays already copied in (the `copy(a[start:n])` data
 * clause of Listing 1a, here device pointers the caller owns), the loop
 * bounds, and for each `reduction(op:var)` clause the operator and the type
 * of the variable (Stage 3.4: "performing variable reductions"; Stage 3.7:
 * the reduction merge across thread blocks).  A `loop independent` loop is
 * work-shared gang -> CTA (grid), worker -> warp, vector -> lane (Sec. 1.2
 * names the four levels; this mapping is the reading used here).
 *
 * Conventions for every entry point
 *  - Pointers named "device" must point to memory of the current CUDA device;
 *    pointers named "host" to ordinary host memory.  The library never frees
 *    caller memory.  Scratch space (block partials, counters, split buffers)
 *    is owned by the library, cached per device and stream, and lives until
 *    the process exits.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *    asynchronous on `stream` unless ACCR_SYNC is set or stated otherwise.
 *  - Return value: ACCR_OK (0) or a negative ACCR_E* code.  The message of the
 *    last error on the calling thread is returned by accr_last_error().  No
 *    entry point aborts the process.
 *  - Element arrays must be aligned to their element size.  Any further
 *    alignment is handled inside (unaligned heads and ragged tails included).
 *  - Indices and lengths are 64-bit.
 *  - Tracing and logging: every compute and serving entry point opens an NVTX
 *    range named after itself for the length of the call (visible in Nsight
 *    Systems and `ncu --nvtx`).  The environment variable ACCR_LOG, read once
 *    per process, sets a log level on stderr: 0 or unset, silent; 1, every
 *    error as it is recorded; 2, also each call's shape and the path it takes
 *    (grid, row form, plan size, served batch).
 */
#ifndef ACCR_H
#define ACCR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ACCR_API __attribute__((visibility("default")))
#else
#define ACCR_API
#endif

/* A CUDA stream handle (the same type as cudaStream_t). */
typedef struct CUstream_st *accr_stream_t;

/* Element and reduction-variable types. */
typedef enum {
    ACCR_I32 = 0, /* int32_t */
    ACCR_I64 = 1, /* int64_t */
    ACCR_F32 = 2, /* float   */
    ACCR_F64 = 3  /* double  */
} accr_type;

/* Reduction operators of the reduction clause.  Identities: + 0, * 1,
 * max lowest (INT_MIN / -inf), min highest (INT_MAX / +inf), & ~0, | 0, ^ 0,
 * && 1, || 0.  Integer + and * wrap modulo 2^32 / 2^64.  && and || give 0 or 1
 * (C semantics).  Bitwise and logical operators are defined on integers only.
 * Floating-point max/min order +0 above -0; NaN inputs are outside the
 * contract (results unspecified). */
typedef enum {
    ACCR_ADD = 0,
    ACCR_MUL = 1,
    ACCR_MAX = 2,
    ACCR_MIN = 3,
    ACCR_BAND = 4,
    ACCR_BOR = 5,
    ACCR_BXOR = 6,
    ACCR_LAND = 7,
    ACCR_LOR = 8
} accr_op;

/* Status codes. */
#define ACCR_OK 0
#define ACCR_EINVAL (-1)    /* bad pointer, size, alignment or flag */
#define ACCR_ETYPE (-2)     /* operator undefined for the type, or narrowing */
#define ACCR_ENOMEM (-3)    /* scratch allocation failed */
#define ACCR_ECUDA (-4)     /* a CUDA call failed (message has the CUDA error) */
#define ACCR_EAGAIN (-5)    /* result not ready yet (accr_poll) */
#define ACCR_EBUDGET (-6)   /* region larger than the server's memory budget */
#define ACCR_ETIMEDOUT (-7) /* a bounded wait ran out */

/* Flags. */
#define ACCR_COMPENSATED 0x1u   /* float + into a float variable: compensated
                                   (Neumaier) sums per thread, pairwise TwoSum
                                   combine, double-precision cross-gang merge */
#define ACCR_SYNC 0x2u          /* return only after the result is written */
#define ACCR_TWO_LEVEL_HOST 0x4u /* the paper's two-level form (SRAD in Sec. 4.2):
                                   block partials on the GPU, copied to the
                                   host and merged there; `out` is then a HOST
                                   pointer and the call is synchronous */

#define ACCR_PLAIN 0x8u          /* accr_batch_reduce: one launch per region */
#define ACCR_UNFUSED 0x10u       /* accr_standardize: two launches */

#define ACCR_MAX_CLAUSES 4

/* One reduction(op:var) clause.  The accumulator type is the variable's type:
 * integer elements need an integer variable at least as wide (int32 elements
 * into an int64 variable are sign-extended); floating-point elements need a
 * floating-point variable at least as wide. */
typedef struct {
    int32_t op;       /* accr_op */
    int32_t acc_type; /* accr_type of the variable */
    const void *init; /* HOST pointer to the variable's value before the
                         region (read during the call), or NULL = identity */
    void *out;        /* DEVICE pointer receiving the variable's value after
                         the region, or pinned (page-locked) host memory, which
                         the last CTA then writes directly; ordinary host
                         memory under ACCR_TWO_LEVEL_HOST */
} accr_clause;

/*
 * accr_reduce -- one region: a `loop independent` loop over i in [0, n) with
 * 1..ACCR_MAX_CLAUSES reduction clauses evaluated in the same single pass
 * (e.g. `reduction(+:s) reduction(max:m)`).
 *
 * Semantics (Stage 3.4 iii, Stage 3.7): for each clause,
 *   var = init (op) x[0] (op) x[1] ... (op) x[n-1]
 * where init is the variable's prior value.  Integer, bitwise, logical and
 * min/max results are exact (any association gives the same bits).  Float +
 * and * are evaluated in a fixed tree order (deterministic for a given device
 * and n); n == 0 leaves the variable equal to init.
 *
 *   in        DEVICE, n elements of in_type
 *   n         number of iterations (>= 0)
 *   clauses   HOST array of nclauses clauses (1..ACCR_MAX_CLAUSES)
 *   flags     ACCR_COMPENSATED | ACCR_SYNC | ACCR_TWO_LEVEL_HOST
 *
 * Device side: one persistent launch; each CTA folds its share into private
 * accumulators, combines them through warp shuffles and shared memory, writes
 * one partial per clause, and the last CTA to finish merges all partials in
 * CTA order (a counter in library scratch, reset by that CTA).  Calls on
 * different streams use different scratch and may overlap.
 */
ACCR_API int accr_reduce(const void *in, int64_t n, int32_t in_type,
                const accr_clause *clauses, int32_t nclauses, uint32_t flags,
                accr_stream_t stream);

/*
 * accr_rowreduce -- the nest `for i (gang) { for j (vector) var_i (op)= A[i][j] }`
 * over a row-major matrix: out[i] = init (op) A[i*ld + 0] ... (op) A[i*ld + cols-1]
 * for every row i < rows (the nest shape of Listing 1a with an inner
 * reduction).  Each clause's `out` is a DEVICE array of `rows` variables; its
 * `init` (if any) is the prior value of every row's variable.
 *
 *   A         DEVICE, rows x ld elements of in_type (ld >= cols)
 *   flags     ACCR_COMPENSATED | ACCR_SYNC
 */
ACCR_API int accr_rowreduce(const void *A, int64_t rows, int64_t cols, int64_t ld,
                   int32_t in_type, const accr_clause *clauses,
                   int32_t nclauses, uint32_t flags, accr_stream_t stream);

/* ---- the Listing-1a nest ------------------------------------------------------ */

#define ACCR_MM_SIMT 0        /* FP32 on CUDA cores, fused multiply-add */
#define ACCR_MM_SIMT_SERIAL 1 /* FP32 on CUDA cores, each product rounded then
                                 added, l in order: the serial program's bits */
#define ACCR_MM_BF16X3 2      /* tensor cores (tcgen05), BF16x3 split precision */
#define ACCR_MM_REUSE_SPLIT 0x20u /* flag: reuse the previous call's bf16 split */

/*
 * accr_matmul_nest -- Listing 1a (Sec. 1.3):
 *   for i, j (independent):  c[i*len + j] = sum over l = 0..len-1 (in order)
 *                                             of a[i*len + l] * b[l*len + j]
 * with float inputs and a float accumulator.
 *
 *   a, b, c   DEVICE, len x len row-major float (4-byte aligned; 16-byte
 *             aligned rows take the vector path)
 *   mode      ACCR_MM_SIMT: tiled FP32 fused multiply-add (per output the l
 *                 terms are still added in order); error at most about
 *                 len * 2^-24 * sum_l |a_il b_lj|.
 *             ACCR_MM_SIMT_SERIAL: the same tiling with the product rounded
 *                 before the add: bit-identical to the serial float program.
 *             ACCR_MM_BF16X3: each operand split into bf16 hi + lo, c =
 *                 a_hi b_hi + a_hi b_lo + a_lo b_hi accumulated in FP32 in
 *                 tensor memory (tcgen05.mma, TMA-fed); error of order 2^-16
 *                 of sum_l |a_il b_lj| (the dropped lo*lo term and the split
 *                 residuals).  Uses library scratch of 8 * len * ceil64(len)
 *                 bytes per stream for the split operands.
 *   flags     ACCR_SYNC (with ACCR_MM_BF16X3 also reports ACCR_ETIMEDOUT if
 *             a pipeline wait inside the kernel ran out) | ACCR_MM_REUSE_SPLIT
 *             (ACCR_MM_BF16X3: a and b are unchanged since the previous call
 *             on this stream with the same a, b and len, so their bf16 split
 *             is reused instead of recomputed; the caller guarantees it)
 */
ACCR_API int accr_matmul_nest(const float *a, const float *b, float *c,
                              int64_t len, int32_t mode, uint32_t flags,
                              accr_stream_t stream);

/* One region of a batch: the loop over in[0, n) with its own clauses.  Each
 * clause's `out` is the DEVICE address of this region's variable. */
typedef struct {
    const void *in;    /* DEVICE, n elements of in_type */
    int64_t n;         /* >= 0 */
    int32_t in_type;   /* accr_type */
    int32_t nclauses;  /* 1..ACCR_MAX_CLAUSES */
    uint32_t flags;    /* ACCR_COMPENSATED or 0 */
    int32_t reserved;  /* 0 */
    accr_clause clauses[ACCR_MAX_CLAUSES];
} accr_region;

/* A prepared batch (see accr_batch_create). */
typedef struct accr_batch accr_batch;

/*
 * accr_batch_reduce -- many independent regions, each with the semantics of
 * accr_reduce, in ONE persistent launch.  This removes the per-region launch
 * cost that the paper's time breakdown charges to every kernel call
 * (Methodology: cudaLaunch, cudaSetupArgument, cudaConfigureCall).
 *
 * Work split: a region of at most ACCR_SMALL_BYTES (by default) is folded
 * whole by one warp; a longer region is cut into tiles of ACCR_TILE_BYTES (by
 * default) that CTAs fold independently; the last tile of a region to finish
 * merges the region's tile partials in tile order and writes its variables.
 * The split depends only on each region's own type and length (under the
 * tiling in force), so a region gives the same bits alone and inside any
 * batch.  A batch of at most 16 regions passes its plan in the kernel's
 * arguments; a larger one uploads it with one copy.  A region with three or
 * four clauses is run as two halves (clauses 0-1, 2-3) that each read its
 * elements.
 *
 *   regions   HOST array of nregions descriptors (read during the call; the
 *             `init` values are read then too)
 *   flags     ACCR_SYNC | ACCR_PLAIN (ACCR_PLAIN: the unbatched form, one
 *             accr_reduce launch per region in order, as the comparison point)
 */
ACCR_API int accr_batch_reduce(const accr_region *regions, int64_t nregions,
                               uint32_t flags, accr_stream_t stream);

/*
 * accr_segmented_reduce -- regions that share one element array, element type
 * and clause list: segment s is values[offsets[s] .. offsets[s+1]).  Each
 * clause's `out` is a DEVICE array of nseg variables; `init` (if any) is the
 * prior value of every segment's variable.  Same device path as
 * accr_batch_reduce.
 *
 *   values    DEVICE array of in_type
 *   offsets   HOST array of nseg+1 non-decreasing element offsets (loop bounds
 *             are host values, as in Listing 1a)
 *   flags     ACCR_COMPENSATED | ACCR_SYNC
 */
ACCR_API int accr_segmented_reduce(const void *values, const int64_t *offsets,
                                   int64_t nseg, int32_t in_type,
                                   const accr_clause *clauses, int32_t nclauses,
                                   uint32_t flags, accr_stream_t stream);

/*
 * accr_batch_create / accr_batch_launch / accr_batch_destroy -- a batch that
 * is run many times.  Create plans the tiles, uploads the plan to device
 * memory owned by the batch, and captures the persistent launch in a CUDA
 * graph; launch replays that graph on `stream` (one graph launch, no host
 * planning, no upload); destroy waits for the batch's work and frees it.
 * The descriptors (pointers, lengths, clauses, init values) are fixed at
 * create time.  Launches of one batch must not overlap on the GPU (they share
 * the batch's tile partials).
 */
ACCR_API int accr_batch_create(const accr_region *regions, int64_t nregions,
                               uint32_t flags, accr_batch **batch);
ACCR_API int accr_batch_launch(accr_batch *batch, accr_stream_t stream);
ACCR_API int accr_batch_destroy(accr_batch *batch);

/* Tiling of batched regions, process-wide: regions of at most small_bytes are
 * folded by one warp, longer ones in tiles of tile_bytes (both multiples of
 * 16, tile_bytes >= 4096).  Changing it changes the evaluation order of float
 * sums (every later call uses the new split).  Returns the previous values
 * through the pointers when they are not NULL; 0 keeps a value. */
ACCR_API int accr_batch_tiling(int64_t small_bytes, int64_t tile_bytes,
                               int64_t *old_small, int64_t *old_tile);
#define ACCR_SMALL_BYTES 65536
#define ACCR_TILE_BYTES 2097152
/* The served loop cuts long regions into tiles of this size, whatever the
 * process-wide tiling: a region is spread over more CTAs, which shortens its
 * latency (measured on GB300 at 50 k regions/s: about half the p50 and p99 of
 * 2 MiB tiles) at a small cost in batch throughput. */
#define ACCR_SERVED_TILE_BYTES 524288

/* ---- patterns of the paper's applications (Sec. 4.2) -------------------------- */

/*
 * accr_nearest_k -- Nearest Neighbor: the k (1..16) points nearest to
 * (qx, qy).  d_i = (x_i - qx)^2 + (y_i - qy)^2 in float, every operation
 * rounded (no fused multiply-add); the k smallest by (d, i), ties by index,
 * in increasing order -- a reduction whose operator keeps a sorted list.
 * One launch.  Each warp starts from a distance bound that k of its own
 * first points reach; for n >= 2^22 the launch also takes the k-th smallest
 * of per-CTA minima over a sample spread across the array and publishes it
 * while the scan runs (no CTA waits for it).  Only points within the
 * current bound are tested one by one; results do not depend on the bounds.
 *
 *   pts       DEVICE, n points as float pairs (x0, y0, x1, y1, ...), 8-byte aligned
 *   idx_out   DEVICE int64[k]; d2_out DEVICE float[k] (-1 / +inf past n)
 *   flags     ACCR_SYNC
 */
ACCR_API int accr_nearest_k(const float *pts, int64_t n, float qx, float qy,
                            int32_t k, int64_t *idx_out, float *d2_out,
                            uint32_t flags, accr_stream_t stream);

/*
 * accr_standardize -- SRAD's reduction region feeding its data-parallel
 * region: mean = sum x / n and var = sum x^2 / n - mean^2 (compensated float
 * sums, merged in double), then y_i = (x_i - (float)mean) * (float)(1/sqrt(var))
 * (y may alias x).  stats receives {mean, var} (DEVICE double[2]).
 *
 * Default: one cooperative launch -- the last CTA of the reduction publishes
 * the statistics and every CTA waits for them (bounded) before the
 * elementwise pass.  ACCR_UNFUSED: two launches, statistics kept on the
 * device.  ACCR_TWO_LEVEL_HOST: the paper's form (partials merged on the
 * host, then the elementwise launch; synchronous).
 *   flags     ACCR_SYNC | ACCR_UNFUSED | ACCR_TWO_LEVEL_HOST
 */
ACCR_API int accr_standardize(const float *x, int64_t n, float *y,
                              double *stats, uint32_t flags,
                              accr_stream_t stream);

#define ACCR_BFS_REDUCE 0     /* levels driven by the host; || reduction of the flag */
#define ACCR_BFS_GUARDED 1    /* levels driven by the host; flag cleared, threads write only 1 */
#define ACCR_BFS_PERSISTENT 2 /* all levels in one cooperative launch, grid barriers */

/*
 * accr_grid_bfs -- BFS's convergence loop: level-synchronous search on a
 * rows x cols grid of cells (open[c] != 0 is passable, 4-neighbour moves) from
 * cell `src`: dist[c] = number of moves, -1 if unreachable.  The loop stops
 * when a level changes no cell; *levels (HOST) = largest distance + 1 (0 if
 * the source is closed).  Synchronous.
 *
 *   open      DEVICE uint8[rows*cols]; dist DEVICE int32[rows*cols]
 *   mode      ACCR_BFS_REDUCE | ACCR_BFS_GUARDED | ACCR_BFS_PERSISTENT
 */
ACCR_API int accr_grid_bfs(const uint8_t *open, int64_t rows, int64_t cols,
                           int64_t src, int32_t *dist, int32_t mode,
                           int64_t *levels, accr_stream_t stream);

/* ---- served request loop ---------------------------------------------------- */

/* A request loop that takes regions as they arrive and runs them in
 * continuous batches (see accr_server_create). */
typedef struct accr_server accr_server;

/* Result of one served region. */
typedef struct {
    int32_t status;                     /* ACCR_OK or the error of its batch */
    int32_t nclauses;
    uint64_t value[ACCR_MAX_CLAUSES];   /* each variable's bits (4-byte types
                                           in the low half) */
    int64_t submit_ns;                  /* steady-clock times: accepted, */
    int64_t launch_ns;                  /* its batch launched, */
    int64_t done_ns;                    /* result visible to the host */
} accr_result;

/*
 * accr_server_create -- start a request loop on the current device.
 *
 * Regions submitted with accr_submit wait in a FIFO queue.  A region is
 * admitted when the bytes of all admitted-but-unfinished regions plus its
 * own stay within `hbm_budget_bytes` (the arrays stay resident on the device;
 * the budget bounds how much of them is in flight).  A scheduler thread
 * forms a batch of up to `max_batch` admitted regions whenever one of
 * `nstreams` stream slots is free and launches it with the batched-region
 * kernel (accr_batch_reduce); batches on different slots overlap on the GPU,
 * and regions that arrive while batches run form the next batch.  Each
 * region's variables come back to the host with its batch.  A region's
 * result does not depend on which batch it ran in.
 */
ACCR_API int accr_server_create(uint64_t hbm_budget_bytes, int32_t nstreams,
                                int32_t max_batch, accr_server **server);

/* Queue one region (`clauses[c].out` is ignored: results come back through
 * accr_poll).  Returns ACCR_EBUDGET if the region alone exceeds the budget.
 * The descriptor is copied, and so is each clause's prior value (`init`): the
 * caller may reuse or free the descriptor and the prior values as soon as
 * this returns.  The region's elements must stay valid until its result has
 * been polled. */
ACCR_API int accr_submit(accr_server *server, const accr_region *region,
                         uint64_t *ticket);

/* Result of `ticket`: timeout_us == 0 returns ACCR_EAGAIN at once if it is
 * not ready; timeout_us > 0 waits at most that long (then ACCR_ETIMEDOUT);
 * timeout_us < 0 waits until it is ready.  A result is returned once. */
ACCR_API int accr_poll(accr_server *server, uint64_t ticket, accr_result *out,
                       int64_t timeout_us);

/* Drain the queue, stop the scheduler and free the server. */
ACCR_API int accr_server_destroy(accr_server *server);

/*
 * accr_server_replay -- an open-loop client for measurement: submits
 * regions[i] at arrival_s[i] seconds after the call starts (in order, waiting
 * on the steady clock), then collects every result into results[i].  With
 * ACCR_PLAIN in `flags` the server is bypassed: each region runs as one
 * synchronous accr_reduce on `stream` at (or after) its arrival time -- the
 * sequential plain-launch comparison.  `server` may be NULL with ACCR_PLAIN.
 */
ACCR_API int accr_server_replay(accr_server *server, const accr_region *regions,
                                const double *arrival_s, int64_t n,
                                uint32_t flags, accr_stream_t stream,
                                accr_result *results);

/*
 * accr_reduce_noalloc -- accr_reduce without any device allocation.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- processes that hand all device memory to their own pool
 * or arena up front, and latency-sensitive loops that cannot afford the
 * device-wide synchronisation cudaMalloc and cudaFree can cause.
 *
 * Same arguments and results as accr_reduce (same grid, so the same bits),
 * except that the block partials and the counter live in one fixed array of
 * ACCR_NOALLOC_SCRATCH_BYTES (+256) bytes compiled into the library, which
 * every GPU that loads the library holds until the process exits.  A region
 * whose nclauses x blocks x 16 bytes exceeds that size is rejected with
 * ACCR_EINVAL (on a 152-SM GB300 the largest need is about 40 KB).
 *
 *   flags     ACCR_COMPENSATED | ACCR_SYNC (ACCR_TWO_LEVEL_HOST needs a pinned
 *             host buffer and is rejected with ACCR_EINVAL)
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset (or anything else that destroys the device's
 * primary context) calls on that device are not valid.  Every call clears the counter on `stream` before
 * its launch.  All calls share the one array: calls that overlap on the GPU
 * (different streams or threads) race on it and give wrong results, so
 * serialise them.  Allocates nothing: no cudaMalloc, cudaFree or allocating
 * library routine is called.
 */
#define ACCR_NOALLOC_SCRATCH_BYTES 65536
ACCR_API int accr_reduce_noalloc(const void *in, int64_t n, int32_t in_type,
                                 const accr_clause *clauses, int32_t nclauses,
                                 uint32_t flags, accr_stream_t stream);

/* ---- failure detection support ------------------------------------------------ */

#define ACCR_FAULT_ALLOC 1  /* device / pinned allocations report ACCR_ENOMEM */
#define ACCR_FAULT_LAUNCH 2 /* kernel launches are skipped and report ACCR_ECUDA */
#define ACCR_FAULT_ADMIT 3  /* accr_submit reports ACCR_EBUDGET */

/* Host-side fault injection for tests: the next `count` operations of `kind`
 * (in any thread) fail as described above, without touching the GPU; count 0
 * clears the kind.  Faults are made on the host only. */
ACCR_API int accr_fault_inject(int32_t kind, int64_t count);

/* Self-test of the bounded waits used inside the tensor-core pipeline: one CTA
 * waits on an mbarrier that nothing ever arrives on, gives up after `tries`
 * polls, records the expiry in a status word and exits.  Returns
 * ACCR_ETIMEDOUT (the expected outcome) after the kernel has finished; the
 * context stays usable. */
ACCR_API int accr_selftest_wait_timeout(uint32_t tries, accr_stream_t stream);

/* ---- measurement support -------------------------------------------------------- */

/* FP32 peak probe, the denominator of the SIMT matrix nest's roofline (no
 * counterpart in the paper): `ctas` CTAs of 256 threads each run `rounds`
 * rounds of 16 independent fused multiply-adds per thread, i.e.
 * 2 * 16 * 256 * ctas * rounds flop, then write one float per thread to
 * `sink` (device memory, caller-owned, at least 256 * ctas floats; every value
 * ends near 1.0) so that no work can be dropped.  Asynchronous on `stream`;
 * time it with events on that stream.  ACCR_EINVAL for ctas < 1, rounds < 1
 * or a NULL sink. */
ACCR_API int accr_probe_fma(int32_t ctas, int64_t rounds, float *sink, accr_stream_t stream);

/* The same probe issuing packed pairs (two float fused multiply-adds per
 * instruction): 16 independent pair chains per thread, i.e.
 * 2 * 32 * 256 * ctas * rounds flop.  Arguments, results and errors as for
 * accr_probe_fma.  The FP32 peak is the larger of the two probes' rates. */
ACCR_API int accr_probe_fma_packed(int32_t ctas, int64_t rounds, float *sink, accr_stream_t stream);

/* Message of the last error raised on the calling thread ("" if none). */
ACCR_API const char *accr_last_error(void);

/* Number of kernels this library has launched in this process. */
ACCR_API uint64_t accr_launch_count(void);

/* ABI version of this header (major * 100 + minor). */
ACCR_API int32_t accr_version(void);

/* Bounds checks of debug builds (a substitute for a memory checker; no
 * counterpart in the paper).  A library built with ACCR_DEBUG
 * (libaccr_debug.so) checks the index of every global store of the row,
 * batched-region, k-nearest and tensor-core kernels against its bound; a
 * failed check does not trap: it counts a violation, records the first
 * failing site and skips the access.  This call (after the work has finished:
 * synchronise first) returns the number of violations since the last clear,
 * the first failing site (0 if none; the codes are listed in the library's
 * debug.cuh) and whether the library checks at all (*checked = 0 in release
 * builds, where both counts are 0); clear != 0 resets the counts. */
ACCR_API int accr_debug_report(uint64_t *violations, uint32_t *first_site, int32_t *checked, int32_t clear);

#define ACCR_VERSION 100

#ifdef __cplusplus
}
#endif
#endif
