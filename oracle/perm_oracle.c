/*
 * perm_oracle.c -- the CPU oracle for the sparse-permanent hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or execute this file; only the test-suite, the smoke check and the
 * bench's CPU-baseline / reference leg use it.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * Everything here is plain, slow and written to be checked against the paper
 * by eye.  Matrices arrive dense and row-major (a[i*n + j] = a_ij), which is
 * equivalent to the CSR/CSC walk of Algorithm 1 because adding an explicit
 * zero changes nothing.
 *
 *   oracle_brute_ld / oracle_brute_u128     Eq. 1 (sum over all permutations)
 *   oracle_ryser_u128                        Eq. 2 (sum over all column subsets)
 *   oracle_ryser_gray_range_u128             Eq. 2 walked in Gray-code order (Sec. II)
 *   oracle_nw_range_ld                       Algorithm 1 (Nijenhuis-Wilf, Gray order)
 *                                            over a Gray-index range, with the
 *                                            per-thread start vector of Sec. II-A
 *   oracle_nw2_range_u128                    Algorithm 1 with every x_i doubled, in
 *                                            integers modulo 2^128 (the same walk,
 *                                            made exact for integer matrices)
 *   oracle_band_dp_ld / oracle_band_dp_u128  an independent permanent for banded
 *                                            matrices (row-by-row DP over the set of
 *                                            used columns in the band window)
 *   oracle_rowdp_ld / oracle_rowdp_u128      an independent permanent for sparse
 *                                            matrices: Eq. 1 expanded row by row,
 *                                            equal subproblems merged
 *   oracle_*_mt                              the range functions above run on T
 *                                            POSIX threads over fixed, aligned chunks
 *                                            that are combined in chunk order, so the
 *                                            result does not depend on T
 *
 * Floating point is long double (x87 80-bit on x86-64, IEEE binary128 on
 * AArch64): at least 11 bits beyond FP64.  Integer arithmetic is unsigned
 * __int128 and wraps modulo 2^128 (a ring homomorphism, so a sum is exact
 * whenever the true value lies in [-2^127, 2^127)).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread perm_oracle.c
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef long double ld;
typedef unsigned __int128 u128;

static u128 u128_from_i64(int64_t v) { return (u128)(__int128)v; }

static void u128_store(u128 v, uint64_t *lo, uint64_t *hi)
{
    *lo = (uint64_t)v;
    *hi = (uint64_t)(v >> 64);
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: perm(A) = sum over permutations sigma of prod_i a_{i,sigma(i)}.     */
/* Row i picks any column not used by rows 0..i-1; every permutation is      */
/* visited exactly once.                                                      */
/* ------------------------------------------------------------------------ */

static void brute_ld_rec(int n, const double *a, int i, int *used, ld prod, ld *acc)
{
    if (i == n) { *acc += prod; return; }
    for (int c = 0; c < n; ++c) {
        if (used[c]) continue;
        used[c] = 1;
        brute_ld_rec(n, a, i + 1, used, prod * (ld)a[i * n + c], acc);
        used[c] = 0;
    }
}

int oracle_brute_ld(int n, const double *a, long double *out)
{
    if (n < 0 || n > 12) return -1;
    int used[12] = {0};
    ld acc = 0;
    brute_ld_rec(n, a, 0, used, 1.0L, &acc);
    *out = acc;
    return 0;
}

static void brute_u128_rec(int n, const int64_t *a, int i, int *used, u128 prod, u128 *acc)
{
    if (i == n) { *acc += prod; return; }
    for (int c = 0; c < n; ++c) {
        if (used[c]) continue;
        used[c] = 1;
        brute_u128_rec(n, a, i + 1, used, prod * u128_from_i64(a[i * n + c]), acc);
        used[c] = 0;
    }
}

int oracle_brute_u128(int n, const int64_t *a, uint64_t *lo, uint64_t *hi)
{
    if (n < 0 || n > 12) return -1;
    int used[12] = {0};
    u128 acc = 0;
    brute_u128_rec(n, a, 0, used, 1, &acc);
    u128_store(acc, lo, hi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 2 (Ryser): perm(A) = (-1)^n sum_{S subset of columns} (-1)^{|S|}       */
/*                          prod_i sum_{j in S} a_ij.                         */
/* Written out directly: every subset, every row sum recomputed.             */
/* ------------------------------------------------------------------------ */

int oracle_ryser_u128(int n, const int64_t *a, uint64_t *lo, uint64_t *hi)
{
    if (n < 1 || n > 30) return -1;
    u128 total = 0;
    for (uint64_t S = 0; S < (1ull << n); ++S) {
        u128 prod = 1;
        for (int i = 0; i < n; ++i) {
            u128 rowsum = 0;
            for (int j = 0; j < n; ++j)
                if ((S >> j) & 1ull) rowsum += u128_from_i64(a[i * n + j]);
            prod *= rowsum;
        }
        if (__builtin_popcountll(S) & 1) total -= prod; else total += prod;
    }
    if (n & 1) total = (u128)0 - total;
    u128_store(total, lo, hi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 2 walked in Gray-code order (Sec. II): subset number k is the set bits */
/* of Gray(k) = k xor (k >> 1); consecutive subsets differ by one column, so  */
/* the row sums are updated instead of recomputed.  Sub-range [k_lo, k_hi)    */
/* of the 2^n subsets; returns sum_k (-1)^{|S_k|} prod_i rowsum_i (without    */
/* the (-1)^n of Eq. 2).                                                      */
/* ------------------------------------------------------------------------ */

int oracle_ryser_gray_range_u128(int n, const int64_t *a, uint64_t k_lo, uint64_t k_hi,
                                 uint64_t *lo, uint64_t *hi)
{
    if (n < 1 || n > 63) return -1;
    if (k_hi > (1ull << n) || k_lo > k_hi) return -1;
    u128 total = 0;
    if (k_lo == k_hi) { u128_store(total, lo, hi); return 0; }
    u128 x[64];
    uint64_t G = k_lo ^ (k_lo >> 1);
    for (int i = 0; i < n; ++i) {
        x[i] = 0;
        for (int j = 0; j < n; ++j)
            if ((G >> j) & 1ull) x[i] += u128_from_i64(a[i * n + j]);
    }
    for (uint64_t k = k_lo; k < k_hi; ++k) {
        if (k != k_lo) {
            uint64_t Gk = k ^ (k >> 1), Gp = (k - 1) ^ ((k - 1) >> 1);
            uint64_t diff = Gk ^ Gp;
            int j = 0;
            while (!((diff >> j) & 1ull)) ++j;          /* log2 of the changed bit */
            int added = (int)((Gk >> j) & 1ull);
            for (int i = 0; i < n; ++i) {
                if (added) x[i] += u128_from_i64(a[i * n + j]);
                else       x[i] -= u128_from_i64(a[i * n + j]);
            }
            G = Gk;
        }
        u128 prod = 1;
        for (int i = 0; i < n; ++i) prod *= x[i];
        if (__builtin_popcountll(G) & 1) total -= prod; else total += prod;
    }
    u128_store(total, lo, hi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (SparsePerman, Nijenhuis-Wilf variant) over Gray indices g in  */
/* [g_lo, g_hi) of the 2^(n-1) indices:                                       */
/*   x-init:  x_i = a_{i,n-1} - (1/2) sum_j a_ij                              */
/*   start:   x_i += sum of a_ij over the set bits j of Gray(g_lo)  (Sec. II-A)*/
/*   term g:  (-1)^g prod_i x_i                                               */
/*   step g:  j = log2(Gray(g) xor Gray(g-1)), s = +1 if bit j of Gray(g) is  */
/*            set else -1, then x_i += s * a_ij                               */
/* Returns the partial sum of the terms and the sum of their magnitudes.      */
/* The permanent is (4 (n mod 2) - 2) times the sum over the whole range.     */
/* The x-init uses a_{i,n-1} itself (zero when row i has no entry in the last */
/* column): Algorithm 1 reads the last stored value of row i, which is the    */
/* same number exactly when row i has a nonzero in column n-1.                */
/* ------------------------------------------------------------------------ */

int oracle_nw_range_ld(int n, const double *a, uint64_t g_lo, uint64_t g_hi,
                       long double *sum_out, long double *abs_out)
{
    if (n < 1 || n > 64) return -1;
    uint64_t total = 1ull << (n - 1);
    if (g_hi > total || g_lo > g_hi) return -1;
    ld x[64];
    for (int i = 0; i < n; ++i) {
        ld rowsum = 0;
        for (int j = 0; j < n; ++j) rowsum += (ld)a[i * n + j];
        x[i] = (ld)a[i * n + (n - 1)] - rowsum / 2;
    }
    uint64_t G = g_lo ^ (g_lo >> 1);
    for (int j = 0; j < n - 1; ++j)
        if ((G >> j) & 1ull)
            for (int i = 0; i < n; ++i) x[i] += (ld)a[i * n + j];
    ld p = 0, pabs = 0;
    for (uint64_t g = g_lo; g < g_hi; ++g) {
        if (g != g_lo) {
            uint64_t Gg = g ^ (g >> 1), Gp = (g - 1) ^ ((g - 1) >> 1);
            uint64_t diff = Gg ^ Gp;
            int j = 0;
            while (!((diff >> j) & 1ull)) ++j;
            ld s = ((Gg >> j) & 1ull) ? 1.0L : -1.0L;
            for (int i = 0; i < n; ++i)
                if (a[i * n + j] != 0.0) x[i] += s * (ld)a[i * n + j];
        }
        ld prod = 1;
        for (int i = 0; i < n; ++i) prod *= x[i];
        if (g & 1ull) p -= prod; else p += prod;
        pabs += prod < 0 ? -prod : prod;
    }
    *sum_out = p;
    *abs_out = pabs;
    return 0;
}

int oracle_nw_perm_ld(int n, const double *a, long double *perm_out, long double *abs_out)
{
    if (n < 1 || n > 40) return -1;
    ld s, sa;
    int rc = oracle_nw_range_ld(n, a, 0, 1ull << (n - 1), &s, &sa);
    if (rc) return rc;
    ld f = (ld)(4 * (n % 2) - 2);
    *perm_out = s * f;
    *abs_out = sa * (f < 0 ? -f : f);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 with every x_i doubled so that integer matrices stay integer:  */
/*   2 x_i = 2 a_{i,n-1} - sum_j a_ij + 2 sum_{j in Gray(g)} a_ij             */
/* The partial sum  sum_g (-1)^g prod_i (2 x_i)  is returned modulo 2^128.    */
/* Over the whole range it equals 2^n * perm / (4 (n mod 2) - 2)              */
/*                              = (-1)^(n-1) 2^(n-1) perm.                    */
/* ------------------------------------------------------------------------ */

int oracle_nw2_range_u128(int n, const int64_t *a, uint64_t g_lo, uint64_t g_hi,
                          uint64_t *lo, uint64_t *hi)
{
    if (n < 1 || n > 64) return -1;
    uint64_t total = 1ull << (n - 1);
    if (g_hi > total || g_lo > g_hi) return -1;
    u128 x2[64];
    for (int i = 0; i < n; ++i) {
        u128 rowsum = 0;
        for (int j = 0; j < n; ++j) rowsum += u128_from_i64(a[i * n + j]);
        x2[i] = 2 * u128_from_i64(a[i * n + (n - 1)]) - rowsum;
    }
    uint64_t G = g_lo ^ (g_lo >> 1);
    for (int j = 0; j < n - 1; ++j)
        if ((G >> j) & 1ull)
            for (int i = 0; i < n; ++i) x2[i] += 2 * u128_from_i64(a[i * n + j]);
    u128 p = 0;
    for (uint64_t g = g_lo; g < g_hi; ++g) {
        if (g != g_lo) {
            uint64_t Gg = g ^ (g >> 1), Gp = (g - 1) ^ ((g - 1) >> 1);
            uint64_t diff = Gg ^ Gp;
            int j = 0;
            while (!((diff >> j) & 1ull)) ++j;
            int added = (int)((Gg >> j) & 1ull);
            for (int i = 0; i < n; ++i) {
                if (added) x2[i] += 2 * u128_from_i64(a[i * n + j]);
                else       x2[i] -= 2 * u128_from_i64(a[i * n + j]);
            }
        }
        u128 prod = 1;
        for (int i = 0; i < n; ++i) prod *= x2[i];
        if (g & 1ull) p -= prod; else p += prod;
    }
    u128_store(p, lo, hi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Banded permanent by dynamic programming over rows (independent of Ryser). */
/* Only a_ij with |i - j| <= w may be nonzero.  Before row i, bit k of the    */
/* state says that column i - w + k is taken (columns outside [0, n) count as */
/* taken).  Row i takes a free column c in [i - w, i + w]; afterwards column  */
/* i - w can never be reached again, so it must be taken, and the window      */
/* slides by one.  The answer is the weight of the all-taken final state.     */
/* ------------------------------------------------------------------------ */

#define BAND_MAXW 6

static int band_check(int n, int w, const void *a, int is_int)
{
    if (n < 1 || n > 4096 || w < 0 || w > BAND_MAXW) return -1;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int off = i - j; if (off < 0) off = -off;
            if (off <= w) continue;
            if (is_int ? ((const int64_t *)a)[i * n + j] != 0 : ((const double *)a)[i * n + j] != 0.0)
                return -2;
        }
    return 0;
}

static int col_exists(int n, int c) { return c >= 0 && c < n; }

int oracle_band_dp_ld(int n, int w, const double *a, long double *out)
{
    int rc = band_check(n, w, a, 0);
    if (rc) return rc;
    int W = 2 * w + 1, NS = 1 << W;
    ld *cur = calloc((size_t)NS, sizeof(ld)), *nxt = calloc((size_t)NS, sizeof(ld));
    if (!cur || !nxt) { free(cur); free(nxt); return -3; }
    /* state before row 0: columns -w..-1 do not exist (taken), columns 0..w-1 free,
       column w is represented once the window slides. */
    int s0 = 0;
    for (int k = 0; k < W; ++k) if (!col_exists(n, 0 - w + k)) s0 |= 1 << k;
    cur[s0] = 1;
    for (int i = 0; i < n; ++i) {
        for (int s = 0; s < NS; ++s) nxt[s] = 0;
        for (int s = 0; s < NS; ++s) {
            if (cur[s] == 0) continue;
            for (int k = 0; k < W; ++k) {
                if ((s >> k) & 1) continue;
                int c = i - w + k;
                if (!col_exists(n, c)) continue;
                ld v = (ld)a[i * n + c];
                if (v == 0) continue;
                int t = s | (1 << k);
                if (!(t & 1)) continue;                   /* column i-w would be lost */
                int u = t >> 1;                           /* slide the window */
                if (!col_exists(n, i + 1 + w)) u |= 1 << (W - 1);
                nxt[u] += cur[s] * v;
            }
        }
        ld *tmp = cur; cur = nxt; nxt = tmp;
    }
    *out = cur[NS - 1];
    free(cur); free(nxt);
    return 0;
}

int oracle_band_dp_u128(int n, int w, const int64_t *a, uint64_t *lo, uint64_t *hi)
{
    int rc = band_check(n, w, a, 1);
    if (rc) return rc;
    int W = 2 * w + 1, NS = 1 << W;
    u128 *cur = calloc((size_t)NS, sizeof(u128)), *nxt = calloc((size_t)NS, sizeof(u128));
    unsigned char *live = calloc((size_t)NS, 1), *nlive = calloc((size_t)NS, 1);
    if (!cur || !nxt || !live || !nlive) { free(cur); free(nxt); free(live); free(nlive); return -3; }
    int s0 = 0;
    for (int k = 0; k < W; ++k) if (!col_exists(n, 0 - w + k)) s0 |= 1 << k;
    cur[s0] = 1; live[s0] = 1;
    for (int i = 0; i < n; ++i) {
        for (int s = 0; s < NS; ++s) { nxt[s] = 0; nlive[s] = 0; }
        for (int s = 0; s < NS; ++s) {
            if (!live[s]) continue;
            for (int k = 0; k < W; ++k) {
                if ((s >> k) & 1) continue;
                int c = i - w + k;
                if (!col_exists(n, c)) continue;
                int64_t v = a[i * n + c];
                if (v == 0) continue;
                int t = s | (1 << k);
                if (!(t & 1)) continue;
                int u = t >> 1;
                if (!col_exists(n, i + 1 + w)) u |= 1 << (W - 1);
                nxt[u] += cur[s] * u128_from_i64(v);
                nlive[u] = 1;
            }
        }
        u128 *tmp = cur; cur = nxt; nxt = tmp;
        unsigned char *tl = live; live = nlive; nlive = tl;
    }
    u128_store(cur[NS - 1], lo, hi);
    free(cur); free(nxt); free(live); free(nlive);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 expanded row by row, with equal subproblems merged (a permanent for  */
/* sparse matrices, independent of Ryser and of the Gray walk).  The rows are */
/* taken in the order `order` (NULL: 0..n-1); a row order does not change a   */
/* permanent.  After k rows a state is the set of columns those rows took;    */
/* its weight is the sum, over the ways of reaching it, of the products of    */
/* the entries taken.  Row order[k] extends every state by each of its        */
/* nonzero columns that the state has not taken.  Two states that agree on    */
/* the columns some later row can still take have the same futures, so a      */
/* state keeps only those columns (reach[k+1]) and merged states add their    */
/* weights.  After the last row the one state left is the empty set, and its  */
/* weight is perm(A).  Returns -4 when more than max_states states are alive. */
/* ------------------------------------------------------------------------ */

#define ROWDP_EMPTY (~0ull)   /* never a state: a state has at most n-1 <= 63 columns */

typedef struct {
    uint64_t *key;
    u128 *iv;           /* integer weights (rowdp_u128) */
    ld *fv;             /* long double weights (rowdp_ld) */
    size_t cap, count;
} rowdp_map;

static int rowdp_map_init(rowdp_map *m, size_t want, int is_int)
{
    size_t cap = 16;
    while (cap < 2 * want) cap <<= 1;
    m->cap = cap;
    m->count = 0;
    m->key = malloc(cap * sizeof(uint64_t));
    m->iv = is_int ? calloc(cap, sizeof(u128)) : NULL;
    m->fv = is_int ? NULL : calloc(cap, sizeof(ld));
    if (!m->key || (is_int ? !m->iv : !m->fv)) return -3;
    for (size_t h = 0; h < cap; ++h) m->key[h] = ROWDP_EMPTY;
    return 0;
}

static void rowdp_map_free(rowdp_map *m)
{
    free(m->key);
    free(m->iv);
    free(m->fv);
}

/* the slot of state k (inserted with weight 0 if absent) */
static size_t rowdp_slot(rowdp_map *m, uint64_t k)
{
    size_t h = (size_t)((k * 0x9E3779B97F4A7C15ull) >> 17) & (m->cap - 1);
    while (m->key[h] != ROWDP_EMPTY && m->key[h] != k) h = (h + 1) & (m->cap - 1);
    if (m->key[h] == ROWDP_EMPTY) {
        m->key[h] = k;
        m->count++;
    }
    return h;
}

static int rowdp(int n, const void *a, int is_int, const int *order, size_t max_states, u128 *iout, ld *fout)
{
    if (n < 1 || n > 64) return -1;
    int row[64], seen[64] = {0};
    for (int k = 0; k < n; ++k) {
        row[k] = order ? order[k] : k;
        if (row[k] < 0 || row[k] >= n || seen[row[k]]++) return -2;
    }
    const int64_t *ai = (const int64_t *)a;
    const double *af = (const double *)a;
    #define ROWDP_NZ(r, j) (is_int ? ai[(r) * n + (j)] != 0 : af[(r) * n + (j)] != 0.0)
    uint64_t reach[65];   /* reach[k]: columns with a nonzero in rows row[k..n-1] */
    reach[n] = 0;
    for (int k = n - 1; k >= 0; --k) {
        reach[k] = reach[k + 1];
        for (int j = 0; j < n; ++j)
            if (ROWDP_NZ(row[k], j)) reach[k] |= 1ull << j;
    }
    rowdp_map cur, nxt;
    if (rowdp_map_init(&cur, 1, is_int)) { rowdp_map_free(&cur); return -3; }
    size_t h0 = rowdp_slot(&cur, 0);
    if (is_int) cur.iv[h0] = 1; else cur.fv[h0] = 1;
    for (int k = 0; k < n; ++k) {
        const int r = row[k];
        int deg = 0;
        for (int j = 0; j < n; ++j) deg += ROWDP_NZ(r, j);
        size_t want = cur.count * (size_t)deg;
        if (want > max_states) want = max_states;
        if (rowdp_map_init(&nxt, want, is_int)) { rowdp_map_free(&cur); rowdp_map_free(&nxt); return -3; }
        for (size_t h = 0; h < cur.cap; ++h) {
            if (cur.key[h] == ROWDP_EMPTY) continue;
            const uint64_t taken = cur.key[h];
            for (int j = 0; j < n; ++j) {
                if (!ROWDP_NZ(r, j) || ((taken >> j) & 1ull)) continue;
                const uint64_t t = (taken | (1ull << j)) & reach[k + 1];
                size_t g = rowdp_slot(&nxt, t);
                if (nxt.count > max_states) { rowdp_map_free(&cur); rowdp_map_free(&nxt); return -4; }
                if (is_int) nxt.iv[g] += cur.iv[h] * u128_from_i64(ai[r * n + j]);
                else nxt.fv[g] += cur.fv[h] * (ld)af[r * n + j];
            }
        }
        rowdp_map_free(&cur);
        cur = nxt;
    }
    #undef ROWDP_NZ
    u128 iv = 0;
    ld fv = 0;
    for (size_t h = 0; h < cur.cap; ++h)
        if (cur.key[h] == 0) {   /* the empty set: every column taken and none reachable */
            if (is_int) iv = cur.iv[h]; else fv = cur.fv[h];
        }
    rowdp_map_free(&cur);
    if (iout) *iout = iv;
    if (fout) *fout = fv;
    return 0;
}

int oracle_rowdp_ld(int n, const double *a, const int *order, uint64_t max_states, long double *out)
{
    return rowdp(n, a, 0, order, (size_t)max_states, NULL, out);
}

int oracle_rowdp_u128(int n, const int64_t *a, const int *order, uint64_t max_states, uint64_t *lo, uint64_t *hi)
{
    u128 v = 0;
    int rc = rowdp(n, a, 1, order, (size_t)max_states, &v, NULL);
    if (rc == 0) u128_store(v, lo, hi);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Multi-threaded drivers.  The range is cut into fixed chunks whose length   */
/* depends only on the range (never on the thread count); each chunk is one   */
/* call of the single-threaded function above; chunk results are combined in  */
/* chunk order.  Threads take chunks round-robin.                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n, kind;                 /* kind 0: nw ld, 1: nw2 u128 */
    const void *a;
    uint64_t g_lo, chunk, nchunks;
    int tid, nthreads;
    ld *sum, *abs;
    u128 *isum;
    int rc;
} mt_job;

static void *mt_worker(void *arg)
{
    mt_job *jb = (mt_job *)arg;
    for (uint64_t c = (uint64_t)jb->tid; c < jb->nchunks; c += (uint64_t)jb->nthreads) {
        uint64_t lo = jb->g_lo + c * jb->chunk, hi = lo + jb->chunk;
        int rc;
        if (jb->kind == 0) {
            rc = oracle_nw_range_ld(jb->n, (const double *)jb->a, lo, hi, &jb->sum[c], &jb->abs[c]);
        } else {
            uint64_t l, h;
            rc = oracle_nw2_range_u128(jb->n, (const int64_t *)jb->a, lo, hi, &l, &h);
            jb->isum[c] = ((u128)h << 64) | l;
        }
        if (rc) jb->rc = rc;
    }
    return NULL;
}

static int run_mt(int kind, int n, const void *a, uint64_t g_lo, uint64_t g_hi, int nthreads,
                  ld *sum_out, ld *abs_out, u128 *isum_out)
{
    if (n < 1 || n > 64 || g_lo > g_hi || g_hi > (1ull << (n - 1))) return -1;
    uint64_t len = g_hi - g_lo;
    if (len == 0) { if (sum_out) { *sum_out = 0; *abs_out = 0; } if (isum_out) *isum_out = 0; return 0; }
    /* chunk = the largest power of two <= len/256 (at least 1) that divides both ends */
    uint64_t chunk = 1;
    while (chunk * 2 <= len / 256 && (g_lo % (chunk * 2)) == 0 && (g_hi % (chunk * 2)) == 0) chunk *= 2;
    uint64_t nchunks = len / chunk;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    ld *sums = calloc((size_t)nchunks, sizeof(ld)), *abss = calloc((size_t)nchunks, sizeof(ld));
    u128 *isums = calloc((size_t)nchunks, sizeof(u128));
    mt_job jobs[256];
    pthread_t th[256];
    if (!sums || !abss || !isums) { free(sums); free(abss); free(isums); return -3; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (mt_job){n, kind, a, g_lo, chunk, nchunks, t, nthreads, sums, abss, isums, 0};
        pthread_create(&th[t], NULL, mt_worker, &jobs[t]);
    }
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) { pthread_join(th[t], NULL); if (jobs[t].rc) rc = jobs[t].rc; }
    ld s = 0, sa = 0; u128 is = 0;
    for (uint64_t c = 0; c < nchunks; ++c) { s += sums[c]; sa += abss[c]; is += isums[c]; }
    if (sum_out) { *sum_out = s; *abs_out = sa; }
    if (isum_out) *isum_out = is;
    free(sums); free(abss); free(isums);
    return rc;
}

int oracle_nw_range_ld_mt(int n, const double *a, uint64_t g_lo, uint64_t g_hi, int nthreads,
                          long double *sum_out, long double *abs_out)
{
    return run_mt(0, n, a, g_lo, g_hi, nthreads, sum_out, abs_out, NULL);
}

int oracle_nw2_range_u128_mt(int n, const int64_t *a, uint64_t g_lo, uint64_t g_hi, int nthreads,
                             uint64_t *lo, uint64_t *hi)
{
    u128 v = 0;
    int rc = run_mt(1, n, a, g_lo, g_hi, nthreads, NULL, NULL, &v);
    u128_store(v, lo, hi);
    return rc;
}

/* sizeof(long double) in bytes, so callers can say which format ran. */
int oracle_long_double_bits(void) { return (int)(8 * sizeof(long double)); }
int oracle_long_double_mant_dig(void) { return __LDBL_MANT_DIG__; }

/* Splits a long double into an unevaluated sum hi + lo of two doubles (so a
   caller that only has doubles keeps the extra precision). */
void oracle_ld_to_dd(const long double *v, double *hi, double *lo)
{
    double h = (double)*v;
    *hi = h;
    *lo = (double)(*v - (long double)h);
}
