/*
 * oracle.h -- serial CPU oracle for the device side of an OpenACC region.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header or constant with the CUDA
 * path.
 *
 * What it computes (IPMACC, arXiv 1412.1127):
 *  - "Ignoring the directive lines, Listing 1a shows the baseline serial
 *    multiplication" (Sec. 1.3): every function here is the region's serial
 *    C program with the `#pragma acc` lines dropped, loops in index order.
 *  - A `reduction(op:var)` clause (Stage 3.4 item iii, Stage 3.7) folds each
 *    iteration's value into the variable: var = var (op) x[i], i = 0..n-1,
 *    starting from the variable's value before the region.
 *  - The Listing-1a nest (Sec. 1.3): c[i*LEN+j] = sum_l a[i*LEN+l]*b[l*LEN+j]
 *    with a float accumulator and a serial l loop.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *  - operators + * max min & | ^ && ||; types int32, int64, float, double;
 *  - integer arithmetic wraps modulo 2^32 / 2^64 (built with -fwrapv and done
 *    on unsigned values);
 *  - && and || give 0 or 1 in the accumulator's type, C semantics;
 *  - max/min on floating point: the larger/smaller value, with +0 ordered
 *    above -0; NaN inputs are outside the contract;
 *  - an integer input folded into a wider accumulator is converted by the
 *    usual C conversion (sign extension); float into double likewise.
 *
 * Built with -O2 -fwrapv -ffp-contract=off and no fast-math, so that the
 * serial float program is what it says (no fused multiply-add).
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

/* element / accumulator types */
#define ORC_I32 0
#define ORC_I64 1
#define ORC_F32 2
#define ORC_F64 3

/* reduction operators */
#define ORC_ADD 0
#define ORC_MUL 1
#define ORC_MAX 2
#define ORC_MIN 3
#define ORC_BAND 4
#define ORC_BOR 5
#define ORC_BXOR 6
#define ORC_LAND 7
#define ORC_LOR 8

/* Serial fold of one reduction clause over x[0..n) read with stride `stride`
 * elements.  `init` points to the variable's value before the region in the
 * accumulator type, or is NULL for the operator's identity.  The result (in
 * the accumulator type) is written to *out.  Returns 0, or -1 if the operator
 * is undefined for the accumulator type or the conversion is not allowed. */
int oracle_reduce(const void *x, int64_t n, int64_t stride, int in_type,
                  int op, int acc_type, const void *init, void *out);

/* Row nest: for each row r < rows, out[r] = fold over A[r*ld + 0..cols).
 * out has `rows` entries of the accumulator type. */
int oracle_rowreduce(const void *A, int64_t rows, int64_t cols, int64_t ld,
                     int in_type, int op, int acc_type, const void *init,
                     void *out);

/* Many independent regions: segment s covers values[offsets[s]..offsets[s+1]).
 * out has nseg entries of the accumulator type. */
int oracle_segmented_reduce(const void *values, const int64_t *offsets,
                            int64_t nseg, int in_type, int op, int acc_type,
                            const void *init, void *out);

/* Identity element of an operator in an accumulator type, written to *out. */
int oracle_identity(int op, int acc_type, void *out);

/* Exact sum of n float (in_type ORC_F32) or double (ORC_F64) values, rounded
 * once to the nearest double (ties to even).  Finite inputs only.  This is the
 * truth that floating-point sums are measured against. */
double oracle_truth_sum(const void *x, int64_t n, int64_t stride, int in_type);

/* Sum of |x[i]| as an exact-rounded double (the scale for relative errors). */
double oracle_truth_abs_sum(const void *x, int64_t n, int64_t stride,
                            int in_type);

/* Listing 1a with the directives ignored: float accumulator, serial l loop. */
void oracle_matmul_listing1(const float *a, const float *b, float *c,
                            int64_t len);

/* Same nest accumulated in double (products of floats are exact in double):
 * c64 = sum_l a*b, and absab = sum_l |a*b| (componentwise error scale). */
void oracle_matmul_truth(const float *a, const float *b, double *c64,
                         double *absab, int64_t len);

/* Single entries of the two nests above, for sampled checks at sizes where
 * the full O(LEN^3) loop would take too long on one core. */
float oracle_matmul_listing1_at(const float *a, const float *b, int64_t len,
                                int64_t i, int64_t j);
double oracle_matmul_truth_at(const float *a, const float *b, int64_t len,
                              int64_t i, int64_t j, double *absab);

/* Rows [i0, i1) of the two nests, reading b through its transpose bt
 * (bt[j*len + l] == b[l*len + j]); same arithmetic in the same order.  The
 * outputs c / c64 / absab are the full len x len arrays; only rows i0..i1-1
 * are written. */
void oracle_matmul_listing1_rows_bt(const float *a, const float *bt, float *c,
                                    int64_t len, int64_t i0, int64_t i1);
void oracle_matmul_truth_rows_bt(const float *a, const float *bt, double *c64,
                                 double *absab, int64_t len, int64_t i0,
                                 int64_t i1);

/* ---- patterns of the paper's applications (Sec. 4.2) ----------------------- */

/* Nearest Neighbor: squared distances d_i = (x_i-qx)^2 + (y_i-qy)^2 of the n
 * points pts[2i], pts[2i+1] (float arithmetic, each operation rounded), and the
 * k smallest by (d, i) in increasing order.  idx[j] = -1 and d2[j] = +inf for
 * j >= n. */
void oracle_nearest_k(const float *pts, int64_t n, float qx, float qy, int k,
                      int64_t *idx, float *d2);

/* SRAD's reduction region feeding its data-parallel region, restated as the
 * standardisation of an array: mean = sum x / n, var = sum x^2 / n - mean^2
 * (sums in double), and y_i = (x_i - mean_f) * rstd_f with mean_f = (float)
 * mean and rstd_f = (float)(1 / sqrt(var)).  stats = {mean, var}. */
void oracle_standardize(const float *x, int64_t n, float *y, double *stats);

/* BFS on a rows x cols grid (4-neighbour moves between open cells, open[c] !=
 * 0), from the source cell: dist[c] = number of moves, -1 if unreachable
 * (or the cell is closed).  Returns the number of levels (largest distance
 * + 1), 0 if the source is closed. */
int64_t oracle_grid_bfs(const uint8_t *open, int64_t rows, int64_t cols,
                        int64_t src, int32_t *dist);

#endif
