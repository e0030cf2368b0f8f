/*
 * cpu_sparseperman.c -- the CPU baseline that bench.py times beside the GPU
 * walk: a plain FP64 re-creation of the paper's CPU-SparsePerman (Sec. VI-B):
 * the Nijenhuis-Wilf walk of Algorithm 1 in Gray order with the columns in
 * ascending nonzero count (the caller passes them sorted), the matrix read
 * column by column (CSC), a running count of the zero entries of x (the
 * product is skipped while one is zero), and POSIX threads over aligned Gray
 * chunks.  It is a reported baseline, not a reference for parity and not part
 * of the library: nothing in the product links or calls it.
 *
 * Build: gcc -O3 -fPIC -shared -pthread cpu_sparseperman.c
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    int n;
    const int *colptr, *rows;
    const double *vals, *x0;
    uint64_t q_lo, q_hi;  /* chunks [q_lo, q_hi) of 2^K indices */
    int K;
    double sum, abs_sum;
} job_t;

static void *walk(void *arg)
{
    job_t *j = (job_t *)arg;
    const int n = j->n;
    double x[64];
    double sum = 0.0, abs_sum = 0.0;
    for (uint64_t q = j->q_lo; q < j->q_hi; ++q) {
        const uint64_t g0 = q << j->K, len = 1ull << j->K;
        for (int i = 0; i < n; ++i) x[i] = j->x0[i];
        uint64_t G = g0 ^ (g0 >> 1);
        while (G) {
            const int c = __builtin_ctzll(G);
            G &= G - 1;
            for (int k = j->colptr[c]; k < j->colptr[c + 1]; ++k) x[j->rows[k]] += j->vals[k];
        }
        int zeros = 0;
        for (int i = 0; i < n; ++i) zeros += x[i] == 0.0;
        double part = 0.0;
        for (uint64_t l = 0; l < len; ++l) {
            const uint64_t g = g0 + l;
            if (l) {
                const int c = __builtin_ctzll(g);
                const double s = ((g >> (c + 1)) & 1ull) ? -1.0 : 1.0;
                for (int k = j->colptr[c]; k < j->colptr[c + 1]; ++k) {
                    const int r = j->rows[k];
                    const double o = x[r], v = o + s * j->vals[k];
                    zeros += (v == 0.0) - (o == 0.0);
                    x[r] = v;
                }
            }
            if (zeros == 0) {
                double p = x[0];
                for (int i = 1; i < n; ++i) p *= x[i];
                part += (g & 1ull) ? -p : p;
                abs_sum += fabs(p);
            }
        }
        sum += part;
    }
    j->sum = sum;
    j->abs_sum = abs_sum;
    return NULL;
}

/* The raw Nijenhuis-Wilf partial sum over Gray indices [g_lo, g_hi) (both
   multiples of 2^K) of the n x n matrix given in CSC (columns in walk order;
   the last column is never flipped) with start values x0, on `threads`
   threads; chunks are dealt out in contiguous blocks.  Returns the sum; the
   sum of |terms| goes to *abs_out. */
double cpu_sparseperman_range(int n, const int *colptr, const int *rows, const double *vals, const double *x0,
                              uint64_t g_lo, uint64_t g_hi, int K, int threads, double *abs_out)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    const uint64_t q_lo = g_lo >> K, q_hi = g_hi >> K, nq = q_hi - q_lo;
    pthread_t tid[256];
    job_t jobs[256];
    for (int t = 0; t < threads; ++t) {
        jobs[t].n = n;
        jobs[t].colptr = colptr;
        jobs[t].rows = rows;
        jobs[t].vals = vals;
        jobs[t].x0 = x0;
        jobs[t].K = K;
        jobs[t].q_lo = q_lo + nq * (uint64_t)t / (uint64_t)threads;
        jobs[t].q_hi = q_lo + nq * (uint64_t)(t + 1) / (uint64_t)threads;
        pthread_create(&tid[t], NULL, walk, &jobs[t]);
    }
    double sum = 0.0, abs_sum = 0.0;
    for (int t = 0; t < threads; ++t) {
        pthread_join(tid[t], NULL);
        sum += jobs[t].sum;
        abs_sum += jobs[t].abs_sum;
    }
    if (abs_out) *abs_out = abs_sum;
    return sum;
}
