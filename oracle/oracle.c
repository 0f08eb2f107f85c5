/*
 * oracle.c -- serial CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Plain C99.  Each function is the region's serial program with the OpenACC
 * directives ignored (IPMACC Sec. 1.3, Listing 1a), plus an exactly rounded
 * sum used as the truth for floating-point tolerances.  No blocking, no
 * reordering, no parallelism: loops run in index order.
 */
#include "oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Type rules (reading of Stage 3.4 iii; the paper names no types):          */
/* integers fold into an integer accumulator at least as wide, floating       */
/* point into a floating-point accumulator at least as wide.                 */
/* ------------------------------------------------------------------------- */
static int is_int(int t) { return t == ORC_I32 || t == ORC_I64; }
static int is_fp(int t) { return t == ORC_F32 || t == ORC_F64; }
static int width(int t) { return (t == ORC_I32 || t == ORC_F32) ? 4 : 8; }

static int combo_ok(int in_type, int op, int acc_type)
{
    if (in_type < 0 || in_type > 3 || acc_type < 0 || acc_type > 3) return 0;
    if (op < ORC_ADD || op > ORC_LOR) return 0;
    if (is_int(in_type) != is_int(acc_type)) return 0;
    if (width(acc_type) < width(in_type)) return 0;
    if (is_fp(acc_type) && op >= ORC_BAND) return 0; /* bitwise / logical */
    return 1;
}

/* Integer elements widened by the usual C conversion (sign extension). */
static int64_t load_int(const void *x, int t, int64_t i)
{
    if (t == ORC_I32) return (int64_t)((const int32_t *)x)[i];
    return ((const int64_t *)x)[i];
}

static double load_fp(const void *x, int t, int64_t i)
{
    if (t == ORC_F32) return (double)((const float *)x)[i];
    return ((const double *)x)[i];
}

/* FP order for max/min: by value, and +0 above -0 (a reading: the paper is
 * silent on signed zero). */
static int fp_above(double v, double a)
{
    if (v > a) return 1;
    if (v == a && v == 0.0 && signbit(a) && !signbit(v)) return 1;
    return 0;
}

int oracle_identity(int op, int acc_type, void *out)
{
    switch (acc_type) {
    case ORC_I32: {
        int32_t v;
        switch (op) {
        case ORC_ADD: v = 0; break;
        case ORC_MUL: v = 1; break;
        case ORC_MAX: v = INT32_MIN; break;
        case ORC_MIN: v = INT32_MAX; break;
        case ORC_BAND: v = -1; break;
        case ORC_BOR: v = 0; break;
        case ORC_BXOR: v = 0; break;
        case ORC_LAND: v = 1; break;
        case ORC_LOR: v = 0; break;
        default: return -1;
        }
        memcpy(out, &v, sizeof v);
        return 0;
    }
    case ORC_I64: {
        int64_t v;
        switch (op) {
        case ORC_ADD: v = 0; break;
        case ORC_MUL: v = 1; break;
        case ORC_MAX: v = INT64_MIN; break;
        case ORC_MIN: v = INT64_MAX; break;
        case ORC_BAND: v = -1; break;
        case ORC_BOR: v = 0; break;
        case ORC_BXOR: v = 0; break;
        case ORC_LAND: v = 1; break;
        case ORC_LOR: v = 0; break;
        default: return -1;
        }
        memcpy(out, &v, sizeof v);
        return 0;
    }
    case ORC_F32: {
        float v;
        switch (op) {
        case ORC_ADD: v = 0.0f; break;
        case ORC_MUL: v = 1.0f; break;
        case ORC_MAX: v = -INFINITY; break;
        case ORC_MIN: v = INFINITY; break;
        default: return -1;
        }
        memcpy(out, &v, sizeof v);
        return 0;
    }
    case ORC_F64: {
        double v;
        switch (op) {
        case ORC_ADD: v = 0.0; break;
        case ORC_MUL: v = 1.0; break;
        case ORC_MAX: v = -INFINITY; break;
        case ORC_MIN: v = INFINITY; break;
        default: return -1;
        }
        memcpy(out, &v, sizeof v);
        return 0;
    }
    }
    return -1;
}

/* var = var (op) x[i] for i = 0..n-1, integer accumulator of `bits` bits.
 * Arithmetic is on unsigned values so that + and * wrap modulo 2^bits. */
static uint64_t fold_int(const void *x, int64_t n, int64_t stride, int in_type,
                         int op, int bits, uint64_t acc)
{
    const uint64_t mask = bits == 32 ? 0xffffffffULL : ~0ULL;
    int64_t i;
    for (i = 0; i < n; ++i) {
        uint64_t v = (uint64_t)load_int(x, in_type, i * stride) & mask;
        /* signed views for the comparisons */
        int64_t sv = bits == 32 ? (int64_t)(int32_t)(uint32_t)v : (int64_t)v;
        int64_t sa = bits == 32 ? (int64_t)(int32_t)(uint32_t)acc : (int64_t)acc;
        switch (op) {
        case ORC_ADD: acc = (acc + v) & mask; break;
        case ORC_MUL: acc = (acc * v) & mask; break;
        case ORC_MAX: if (sv > sa) acc = v; break;
        case ORC_MIN: if (sv < sa) acc = v; break;
        case ORC_BAND: acc = acc & v; break;
        case ORC_BOR: acc = acc | v; break;
        case ORC_BXOR: acc = acc ^ v; break;
        case ORC_LAND: acc = (acc != 0) && (v != 0); break;
        case ORC_LOR: acc = (acc != 0) || (v != 0); break;
        }
    }
    return acc;
}

/* float accumulator: every step rounds to float, as the serial C program. */
static float fold_f32(const float *x, int64_t n, int64_t stride, int op, float acc)
{
    int64_t i;
    for (i = 0; i < n; ++i) {
        float v = x[i * stride];
        switch (op) {
        case ORC_ADD: acc = acc + v; break;
        case ORC_MUL: acc = acc * v; break;
        case ORC_MAX: if (fp_above(v, acc)) acc = v; break;
        case ORC_MIN: if (fp_above(acc, v)) acc = v; break;
        }
    }
    return acc;
}

static double fold_f64(const void *x, int64_t n, int64_t stride, int in_type,
                       int op, double acc)
{
    int64_t i;
    for (i = 0; i < n; ++i) {
        double v = load_fp(x, in_type, i * stride);
        switch (op) {
        case ORC_ADD: acc = acc + v; break;
        case ORC_MUL: acc = acc * v; break;
        case ORC_MAX: if (fp_above(v, acc)) acc = v; break;
        case ORC_MIN: if (fp_above(acc, v)) acc = v; break;
        }
    }
    return acc;
}

int oracle_reduce(const void *x, int64_t n, int64_t stride, int in_type,
                  int op, int acc_type, const void *init, void *out)
{
    if (!combo_ok(in_type, op, acc_type) || n < 0) return -1;
    switch (acc_type) {
    case ORC_I32: {
        int32_t a;
        if (init) memcpy(&a, init, sizeof a); else oracle_identity(op, acc_type, &a);
        uint64_t r = fold_int(x, n, stride, in_type, op, 32, (uint64_t)(uint32_t)a);
        int32_t v = (int32_t)(uint32_t)r;
        memcpy(out, &v, sizeof v);
        return 0;
    }
    case ORC_I64: {
        int64_t a;
        if (init) memcpy(&a, init, sizeof a); else oracle_identity(op, acc_type, &a);
        uint64_t r = fold_int(x, n, stride, in_type, op, 64, (uint64_t)a);
        int64_t v = (int64_t)r;
        memcpy(out, &v, sizeof v);
        return 0;
    }
    case ORC_F32: {
        float a;
        if (init) memcpy(&a, init, sizeof a); else oracle_identity(op, acc_type, &a);
        a = fold_f32((const float *)x, n, stride, op, a);
        memcpy(out, &a, sizeof a);
        return 0;
    }
    case ORC_F64: {
        double a;
        if (init) memcpy(&a, init, sizeof a); else oracle_identity(op, acc_type, &a);
        a = fold_f64(x, n, stride, in_type, op, a);
        memcpy(out, &a, sizeof a);
        return 0;
    }
    }
    return -1;
}

int oracle_rowreduce(const void *A, int64_t rows, int64_t cols, int64_t ld,
                     int in_type, int op, int acc_type, const void *init,
                     void *out)
{
    const int ib = width(in_type), ob = width(acc_type);
    int64_t r;
    if (rows < 0 || cols < 0 || ld < cols) return -1;
    for (r = 0; r < rows; ++r) {
        const char *row = (const char *)A + (size_t)(r * ld) * (size_t)ib;
        char *o = (char *)out + (size_t)r * (size_t)ob;
        if (oracle_reduce(row, cols, 1, in_type, op, acc_type, init, o) != 0)
            return -1;
    }
    return 0;
}

int oracle_segmented_reduce(const void *values, const int64_t *offsets,
                            int64_t nseg, int in_type, int op, int acc_type,
                            const void *init, void *out)
{
    const int ib = width(in_type), ob = width(acc_type);
    int64_t s;
    for (s = 0; s < nseg; ++s) {
        int64_t lo = offsets[s], hi = offsets[s + 1];
        const char *seg = (const char *)values + (size_t)lo * (size_t)ib;
        char *o = (char *)out + (size_t)s * (size_t)ob;
        if (hi < lo) return -1;
        if (oracle_reduce(seg, hi - lo, 1, in_type, op, acc_type, init, o) != 0)
            return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Exact sum: a fixed-point "long accumulator" whose least significant bit   */
/* is 2^-1074 (the smallest subnormal double), held as 32-bit digits in      */
/* int64 words so that carries can be deferred.  Rounded once at the end.    */
/* ------------------------------------------------------------------------- */
#define LA_DIGITS 72 /* 72*32 = 2304 bits: 2^-1074 .. 2^1229, room for carries */
#define LA_MASK 0xffffffffLL

typedef struct {
    int64_t d[LA_DIGITS];
    int64_t adds; /* additions since the last carry propagation */
} longacc;

static void la_normalize(longacc *A)
{
    int i;
    for (i = 0; i < LA_DIGITS - 1; ++i) {
        int64_t low = A->d[i] & LA_MASK;            /* in [0, 2^32) */
        int64_t carry = (A->d[i] - low) / 4294967296LL; /* exact */
        A->d[i] = low;
        A->d[i + 1] += carry;
    }
    A->adds = 0;
}

static void la_add(longacc *A, double x)
{
    int e, neg, k, sh, off;
    double f;
    uint64_t m, mlo, mhi, t0, t1;
    int64_t c0, c1, c2;
    if (x == 0.0) return;
    neg = x < 0.0;
    f = frexp(fabs(x), &e);            /* |x| = f * 2^e, f in [0.5, 1) */
    m = (uint64_t)ldexp(f, 53);        /* integer < 2^53, |x| = m * 2^(e-53) */
    off = e - 53 + 1074;               /* bit position of m's lsb */
    if (off < 0) {                     /* subnormal: low bits of m are zero */
        m >>= -off;
        off = 0;
    }
    k = off / 32;
    sh = off % 32;
    mlo = m & 0xffffffffULL;
    mhi = m >> 32;
    t0 = mlo << sh;                    /* < 2^64 */
    t1 = mhi << sh;                    /* < 2^53 */
    c0 = (int64_t)(t0 & 0xffffffffULL);
    c1 = (int64_t)((t0 >> 32) + (t1 & 0xffffffffULL));
    c2 = (int64_t)(t1 >> 32);
    if (neg) { c0 = -c0; c1 = -c1; c2 = -c2; }
    A->d[k] += c0;
    A->d[k + 1] += c1;
    A->d[k + 2] += c2;
    if (++A->adds >= (1LL << 28)) la_normalize(A);
}

static int la_bit(const longacc *A, int i)
{
    return (int)((A->d[i / 32] >> (i % 32)) & 1);
}

static double la_round(longacc *A)
{
    int i, p = -1, neg = 0;
    la_normalize(A);
    if (A->d[LA_DIGITS - 1] < 0) { /* negative total: negate every digit */
        neg = 1;
        for (i = 0; i < LA_DIGITS; ++i) A->d[i] = -A->d[i];
        la_normalize(A);
    }
    for (i = LA_DIGITS * 32 - 1; i >= 0; --i)
        if (la_bit(A, i)) { p = i; break; }
    if (p < 0) return 0.0;
    if (p < 53) { /* fits a double exactly (including subnormals) */
        uint64_t v = 0;
        for (i = p; i >= 0; --i) v = (v << 1) | (uint64_t)la_bit(A, i);
        double r = ldexp((double)v, -1074);
        return neg ? -r : r;
    } else {
        uint64_t M = 0;
        int rnd, sticky = 0;
        for (i = p; i >= p - 52; --i) M = (M << 1) | (uint64_t)la_bit(A, i);
        rnd = la_bit(A, p - 53);
        for (i = p - 54; i >= 0 && !sticky; --i) sticky = la_bit(A, i);
        if (rnd && (sticky || (M & 1))) M += 1; /* nearest, ties to even */
        double r = ldexp((double)M, p - 52 - 1074);
        return neg ? -r : r;
    }
}

double oracle_truth_sum(const void *x, int64_t n, int64_t stride, int in_type)
{
    longacc A;
    int64_t i;
    memset(&A, 0, sizeof A);
    for (i = 0; i < n; ++i) la_add(&A, load_fp(x, in_type, i * stride));
    return la_round(&A);
}

double oracle_truth_abs_sum(const void *x, int64_t n, int64_t stride,
                            int in_type)
{
    longacc A;
    int64_t i;
    memset(&A, 0, sizeof A);
    for (i = 0; i < n; ++i) la_add(&A, fabs(load_fp(x, in_type, i * stride)));
    return la_round(&A);
}

/* ------------------------------------------------------------------------- */
/* Listing 1a (Sec. 1.3): the i and j loops are independent, l is serial.    */
/* ------------------------------------------------------------------------- */
float oracle_matmul_listing1_at(const float *a, const float *b, int64_t len,
                                int64_t i, int64_t j)
{
    int64_t l;
    float sum = 0;
    for (l = 0; l < len; ++l) sum += a[i * len + l] * b[l * len + j];
    return sum;
}

void oracle_matmul_listing1(const float *a, const float *b, float *c,
                            int64_t len)
{
    int64_t i, j;
    for (i = 0; i < len; ++i)
        for (j = 0; j < len; ++j)
            c[i * len + j] = oracle_matmul_listing1_at(a, b, len, i, j);
}

/* Products of two floats are exact in double; the double sum adds a relative
 * error of at most about len * 2^-53 of sum |a*b|, far below float rounding. */
double oracle_matmul_truth_at(const float *a, const float *b, int64_t len,
                              int64_t i, int64_t j, double *absab)
{
    int64_t l;
    double s = 0.0, t = 0.0;
    for (l = 0; l < len; ++l) {
        double p = (double)a[i * len + l] * (double)b[l * len + j];
        s += p;
        t += fabs(p);
    }
    if (absab) *absab = t;
    return s;
}

void oracle_matmul_truth(const float *a, const float *b, double *c64,
                         double *absab, int64_t len)
{
    int64_t i, j;
    for (i = 0; i < len; ++i)
        for (j = 0; j < len; ++j)
            c64[i * len + j] = oracle_matmul_truth_at(
                a, b, len, i, j, absab ? &absab[i * len + j] : NULL);
}

/* Rows i0..i1-1 of the two nests above, with b given through its transpose
 * (bt[j * len + l] == b[l * len + j]).  The arithmetic and its order are those
 * of Listing 1a (l ascending, float accumulator rounded after every multiply
 * and add); only the layout of b differs, so that both operands are read
 * along memory and independent row blocks of a large product can run in
 * separate threads. */
void oracle_matmul_listing1_rows_bt(const float *a, const float *bt, float *c,
                                    int64_t len, int64_t i0, int64_t i1)
{
    int64_t i, j, l;
    for (i = i0; i < i1; ++i)
        for (j = 0; j < len; ++j) {
            const float *ar = a + i * len, *bc = bt + j * len;
            float sum = 0;
            for (l = 0; l < len; ++l) sum += ar[l] * bc[l];
            c[i * len + j] = sum;
        }
}

void oracle_matmul_truth_rows_bt(const float *a, const float *bt, double *c64,
                                 double *absab, int64_t len, int64_t i0,
                                 int64_t i1)
{
    int64_t i, j, l;
    for (i = i0; i < i1; ++i)
        for (j = 0; j < len; ++j) {
            const float *ar = a + i * len, *bc = bt + j * len;
            double s = 0.0, t = 0.0;
            for (l = 0; l < len; ++l) {
                double p = (double)ar[l] * (double)bc[l];
                s += p;
                t += fabs(p);
            }
            c64[i * len + j] = s;
            absab[i * len + j] = t;
        }
}

/* ------------------------------------------------------------------------- */
/* Application patterns (Sec. 4.2).                                          */
/* ------------------------------------------------------------------------- */

/* (d, i) order: by distance, ties by index. */
static int pair_less(float da, int64_t ia, float db, int64_t ib)
{
    return da < db || (da == db && ia < ib);
}

void oracle_nearest_k(const float *pts, int64_t n, float qx, float qy, int k,
                      int64_t *idx, float *d2)
{
    int64_t i;
    int j;
    /* k selection passes: each takes the smallest pair above the previous */
    float last_d = -INFINITY;
    int64_t last_i = -1;
    for (j = 0; j < k; ++j) {
        float best_d = INFINITY;
        int64_t best_i = -1;
        for (i = 0; i < n; ++i) {
            float dx = pts[2 * i] - qx;
            float dy = pts[2 * i + 1] - qy;
            float d = dx * dx + dy * dy;
            if (pair_less(last_d, last_i, d, i) &&
                (best_i < 0 || pair_less(d, i, best_d, best_i))) {
                best_d = d;
                best_i = i;
            }
        }
        idx[j] = best_i;
        d2[j] = best_i < 0 ? INFINITY : best_d;
        if (best_i >= 0) {
            last_d = best_d;
            last_i = best_i;
        } else {
            last_d = INFINITY;
            last_i = INT64_MAX;
        }
    }
}

void oracle_standardize(const float *x, int64_t n, float *y, double *stats)
{
    int64_t i;
    double s = 0.0, s2 = 0.0, mean, var;
    float mean_f, rstd_f;
    for (i = 0; i < n; ++i) {
        s += (double)x[i];
        s2 += (double)x[i] * (double)x[i];
    }
    mean = n > 0 ? s / (double)n : 0.0;
    var = n > 0 ? s2 / (double)n - mean * mean : 0.0;
    stats[0] = mean;
    stats[1] = var;
    mean_f = (float)mean;
    rstd_f = var > 0.0 ? (float)(1.0 / sqrt(var)) : 0.0f;
    for (i = 0; i < n; ++i) y[i] = (x[i] - mean_f) * rstd_f;
}

int64_t oracle_grid_bfs(const uint8_t *open, int64_t rows, int64_t cols,
                        int64_t src, int32_t *dist)
{
    int64_t total = rows * cols, head = 0, tail = 0, c, levels = 0;
    int64_t *queue;
    for (c = 0; c < total; ++c) dist[c] = -1;
    if (src < 0 || src >= total || !open[src]) return 0;
    queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)total);
    if (!queue) return -1;
    dist[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int64_t u = queue[head++], r = u / cols, q = u % cols, nb[4];
        int m, cnt = 0;
        if (r > 0) nb[cnt++] = u - cols;
        if (r + 1 < rows) nb[cnt++] = u + cols;
        if (q > 0) nb[cnt++] = u - 1;
        if (q + 1 < cols) nb[cnt++] = u + 1;
        for (m = 0; m < cnt; ++m) {
            int64_t v = nb[m];
            if (open[v] && dist[v] < 0) {
                dist[v] = dist[u] + 1;
                queue[tail++] = v;
            }
        }
        if (dist[u] + 1 > levels) levels = dist[u] + 1;
    }
    free(queue);
    return levels;
}
