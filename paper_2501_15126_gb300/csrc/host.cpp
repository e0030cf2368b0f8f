// host.cpp -- host preprocessing (see host.hpp).
#include "host.hpp"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

namespace perm {

perm_status_t ingest(const perm_matrix_t *A, Matrix &out, const char **errp, void *storage, size_t storage_bytes) {
    const char *dummy = nullptr;
    const char *&err = errp ? *errp : dummy;
    if (!A) { err = "matrix is NULL"; return PERM_ERR_ARG; }
    if (A->n < 1 || A->n > kNMax) { err = "n must be in [1, 64]"; return PERM_ERR_SIZE; }
    if (A->nnz < 0) { err = "nnz < 0"; return PERM_ERR_SIZE; }
    if (A->layout != PERM_CSR && A->layout != PERM_CSC) { err = "bad layout"; return PERM_ERR_ARG; }
    if (A->vtype != PERM_F64 && A->vtype != PERM_I64) { err = "bad value type"; return PERM_ERR_ARG; }
    if (!A->ptr || (A->nnz > 0 && (!A->idx || !A->vals))) { err = "NULL array"; return PERM_ERR_ARG; }
    const int n = A->n;
    if (A->ptr[0] != 0 || A->ptr[n] != A->nnz) { err = "ptr[0] must be 0 and ptr[n] must be nnz"; return PERM_ERR_SIZE; }
    out.n = n;
    out.is_int = A->vtype == PERM_I64;
    for (int i = 0; i < kNMax; ++i) out.rowmask[i] = out.colmask[i] = 0;
    const size_t bytes = (size_t)n * n * 8;
    unsigned char *buf;
    if (storage) {
        if (storage_bytes < bytes) { err = "ingest storage too small"; return PERM_ERR_SIZE; }
        buf = static_cast<unsigned char *>(storage);
    } else {
        out.own.assign(bytes, 0);
        buf = out.own.data();
    }
    std::memset(buf, 0, bytes);
    out.f = out.is_int ? nullptr : reinterpret_cast<double *>(buf);
    out.v = out.is_int ? reinterpret_cast<int64_t *>(buf) : nullptr;
    for (int o = 0; o < n; ++o) {
        const int b = A->ptr[o], e = A->ptr[o + 1];
        if (b > e || b < 0 || e > A->nnz) { err = "ptr not monotone"; return PERM_ERR_PATTERN; }
        int prev = -1;
        for (int k = b; k < e; ++k) {
            const int t = A->idx[k];
            if (t < 0 || t >= n) { err = "index out of range"; return PERM_ERR_PATTERN; }
            if (t <= prev) { err = "indices not strictly increasing"; return PERM_ERR_PATTERN; }
            prev = t;
            const int i = A->layout == PERM_CSR ? o : t;
            const int j = A->layout == PERM_CSR ? t : o;
            if (out.is_int) {
                const int64_t v = ((const int64_t *)A->vals)[k];
                if (v == 0) continue;
                out.v[(size_t)i * n + j] = v;
            } else {
                const double v = ((const double *)A->vals)[k];
                if (!std::isfinite(v)) { err = "non-finite value"; return PERM_ERR_ARG; }
                if (v == 0.0) continue;
                out.f[(size_t)i * n + j] = v;
            }
            out.rowmask[i] |= 1ull << j;
            out.colmask[j] |= 1ull << i;
        }
    }
    return PERM_OK;
}

// Kuhn's augmenting paths on the bipartite row/column graph.
static bool augment(const Matrix &m, int i, uint64_t &seen, int *match_col) {
    uint64_t cand = m.rowmask[i] & ~seen;
    while (cand) {
        const int j = __builtin_ctzll(cand);
        cand &= cand - 1;
        seen |= 1ull << j;
        if (match_col[j] < 0 || augment(m, match_col[j], seen, match_col)) {
            match_col[j] = i;
            return true;
        }
    }
    return false;
}

bool has_perfect_matching(const Matrix &m) {
    int match_col[kNMax];
    for (int j = 0; j < m.n; ++j) match_col[j] = -1;
    for (int i = 0; i < m.n; ++i) {
        uint64_t seen = 0;
        if (!augment(m, i, seen, match_col)) return false;
    }
    return true;
}

void order_none(const Matrix &m, int *col_order) {
    for (int j = 0; j < m.n; ++j) col_order[j] = j;
}

// Ascending nonzero count, ties by index (a stable insertion sort: n <= 64,
// and it allocates nothing).
void order_degree(const Matrix &m, int *col_order) {
    order_none(m, col_order);
    for (int i = 1; i < m.n; ++i) {
        const int c = col_order[i];
        const int d = __builtin_popcountll(m.colmask[c]);
        int j = i - 1;
        while (j >= 0 && __builtin_popcountll(m.colmask[col_order[j]]) > d) {
            col_order[j + 1] = col_order[j];
            --j;
        }
        col_order[j + 1] = c;
    }
}

// Algorithm 3 (PermanentOrdering).  cdeg[j] counts the nonzeros of column j
// on rows not yet ordered; each round picks the column with the smallest
// count (ties: smallest index), orders its unordered rows (in row order, as a
// CSC scan meets them) and lowers the counts of every column sharing one of
// those rows.
void order_alg3(const Matrix &m, int *col_order, int *row_order) {
    const int n = m.n;
    const int kInf = INT_MAX / 2;
    int cdeg[kNMax];
    bool rmark[kNMax];
    for (int j = 0; j < n; ++j) cdeg[j] = __builtin_popcountll(m.colmask[j]);
    for (int i = 0; i < n; ++i) rmark[i] = false;
    int ridx = 0;
    for (int cidx = 0; cidx < n; ++cidx) {
        int col = -1;
        for (int j = 0; j < n; ++j)
            if (cdeg[j] < kInf && (col < 0 || cdeg[j] < cdeg[col])) col = j;
        col_order[cidx] = col;
        cdeg[col] = kInf;
        uint64_t rows = m.colmask[col];
        while (rows) {
            const int row = __builtin_ctzll(rows);
            rows &= rows - 1;
            if (rmark[row]) continue;
            rmark[row] = true;
            row_order[ridx++] = row;
            uint64_t cols = m.rowmask[row];
            while (cols) {
                const int c2 = __builtin_ctzll(cols);
                cols &= cols - 1;
                if (cdeg[c2] < kInf) cdeg[c2] -= 1;
            }
        }
    }
    // rows no column reaches (only with an empty row) go last, in index order
    for (int i = 0; i < n; ++i)
        if (!rmark[i]) row_order[ridx++] = i;
}

Layout make_layout(const Matrix &m, const int *col_order, int ordering) {
    Layout L;
    const int n = m.n;
    L.n = n;
    L.ordering = ordering;
    for (int p = 0; p < n; ++p) L.col_order[p] = col_order[p];
    // first touching position of each original row
    int first[kNMax];
    for (int i = 0; i < n; ++i) first[i] = n - 1;
    bool seen[kNMax] = {};
    int order_seen[kNMax], nseen = 0;
    for (int p = 0; p < n; ++p) {
        uint64_t rows = m.colmask[col_order[p]];
        while (rows) {
            const int r = __builtin_ctzll(rows);
            rows &= rows - 1;
            if (!seen[r]) { seen[r] = true; first[r] = p; order_seen[nseen++] = r; }
        }
    }
    for (int i = 0; i < n; ++i)
        if (!seen[i]) order_seen[nseen++] = i;   // empty rows (perm is 0 anyway)
    // column 0's rows (group 0): their first touching position after 0
    // (n-1 when no flipped column touches them again)
    int second[kNMax];
    for (int i = 0; i < n; ++i) {
        second[i] = n - 1;
        if (first[i] != 0) continue;
        for (int p = 1; p < n - 1; ++p)
            if ((m.colmask[col_order[p]] >> i) & 1ull) { second[i] = p; break; }
    }
    // slots: stable by group, inside a group in first-touch order, except
    // that group 0 is sorted by the second touching position (so each set S_m
    // below is a contiguous slot range)
    int by_group[kNMax], gcount[kNMax + 1] = {};
    for (int i = 0; i < n; ++i) ++gcount[first[i] + 1];
    for (int g = 0; g < n; ++g) gcount[g + 1] += gcount[g];
    for (int g = 0; g <= n; ++g) L.group_begin[g] = gcount[g];
    for (int k = 0; k < n; ++k) {   // counting sort by group, stable in first-touch order
        const int r = order_seen[k];
        by_group[gcount[first[r]]++] = r;
    }
    std::stable_sort(by_group, by_group + L.group_begin[1], [&](int a, int b) { return second[a] < second[b]; });
    for (int slot = 0; slot < n; ++slot) {
        const int r = by_group[slot];
        L.row_order[slot] = r;
        L.slot_of_row[r] = slot;
        L.group_of_slot[slot] = first[r];
    }
    L.top = 0;
    for (int g = 0; g < n; ++g)
        if (L.group_begin[g + 1] > L.group_begin[g]) L.top = g;
    // S_m = rows of column 0 whose next touching position is m: slots
    // [s_begin[m], s_begin[m+1]) inside [0, group_begin[1])
    for (int mm = 0; mm <= n; ++mm) L.s_begin[mm] = 0;
    {
        int k = 0;
        for (int mm = 1; mm <= n - 1; ++mm) {
            L.s_begin[mm] = k;
            while (k < L.group_begin[1] && second[L.row_order[k]] == mm) ++k;
        }
        L.s_begin[n] = k;
    }
    L.top_dual = L.top;
    for (int mm = 1; mm <= n - 1; ++mm)
        if (L.s_begin[mm + 1] > L.s_begin[mm]) L.top_dual = std::max(L.top_dual, mm);
    for (int p = 0; p < n; ++p) {
        uint64_t rows = m.colmask[col_order[p]], mask = 0;
        while (rows) {
            const int r = __builtin_ctzll(rows);
            rows &= rows - 1;
            mask |= 1ull << L.slot_of_row[r];
        }
        L.colmask[p] = mask;
        L.col_nnz[p] = __builtin_popcountll(mask);
    }
    return L;
}

double cost_per_step(const Layout &L, bool paper_scheme) {
    const int n = L.n;
    if (n < 2) return 0.0;
    const double steps = std::ldexp(1.0, n - 1) - 1.0;
    double total = 0.0, prefix = 0.0;
    for (int j = 0; j <= n - 2; ++j) {
        const double w = std::ldexp(1.0, n - j - 2) / steps;   // Lemma 2
        prefix += L.group_begin[j + 1] - L.group_begin[j];
        const double mults = paper_scheme ? (double)(n - 1) : prefix;
        total += w * (L.col_nnz[j] + mults + 1.0);
    }
    return total;
}

double cost_per_step_paired(const Layout &L) {
    const int n = L.n;
    if (n < 3) return cost_per_step(L, false);
    const double steps = std::ldexp(1.0, n - 1) - 1.0;
    const double r0 = L.group_begin[1] - L.group_begin[0];
    double total = 0.0, prefix = 0.0;
    for (int j = 1; j <= n - 2; ++j) {
        const double w = std::ldexp(1.0, n - j - 2) / steps;   // Lemma 2
        prefix += L.group_begin[j + 1] - L.group_begin[j];     // |R_1| + ... + |R_j|
        total += w * (L.col_nnz[j] + prefix);
    }
    const double w0 = std::ldexp(1.0, n - 2) / steps;           // column-0 steps = pairs
    const double pair_ops = r0 == 1 ? 2.0 : 3.0 * r0 - 1.0;
    return total + w0 * pair_ops;
}

double cost_per_step_dual(const Layout &L, bool shared_product) {
    const int n = L.n;
    if (n < 3) return cost_per_step(L, false);
    const double steps = std::ldexp(1.0, n - 1) - 1.0;
    double total = 0.0, rate = 0.0;
    for (int m = n - 2; m >= 1; --m) {
        const double w = std::ldexp(1.0, n - m - 2) / steps;   // Lemma 2: column m's flips per step
        total += w * L.col_nnz[m];
        rate += w;                                             // level m is rebuilt by any column >= m
        const int r = L.group_begin[m + 1] - L.group_begin[m];
        const int sm = L.s_begin[m + 1] - L.s_begin[m];
        // shared: the group's product (r - 1 multiplications) into both chains (2);
        // S_m rows: x and x + a_0 into the two chains (3 operations per row)
        const double level = (shared_product ? (r ? r + 1.0 : 0.0) : 2.0 * r) + 3.0 * sm;
        total += rate * level;
    }
    const double w0 = std::ldexp(1.0, n - 2) / steps;         // pairs of steps
    return total + w0 * 2.0;
}

// The step-cost model of the scheme a plan will run, straight from a column
// order (group sizes, column-0 rows by next column, column sizes: O(n) with
// bit masks), for the order search below.  Same formulas as cost_per_step
// (exact: one chain), cost_per_step_paired and cost_per_step_dual (FP64:
// the cheaper of the two for long walks, two-state chains for short ones).
static double order_cost(const Matrix &m, const int *cols, bool fp64, bool long_walk) {
    const int n = m.n;
    int R[kNMax], d[kNMax], S[kNMax + 1] = {};
    uint64_t seen = 0, r0 = 0;
    for (int p = 0; p < n; ++p) {
        const uint64_t cm = m.colmask[cols[p]];
        d[p] = __builtin_popcountll(cm);
        const uint64_t nw = cm & ~seen;
        R[p] = __builtin_popcountll(nw);
        seen |= cm;
        if (p == 0) r0 = nw;
    }
    uint64_t rem = r0;
    for (int p = 1; p < n - 1; ++p) {
        const uint64_t hit = m.colmask[cols[p]] & rem;
        S[p] = __builtin_popcountll(hit);
        rem &= ~hit;
    }
    const double steps = std::ldexp(1.0, n - 1) - 1.0;
    if (!fp64) {   // one chain, column 0 applied (cost_per_step)
        double total = 0.0, prefix = 0.0;
        for (int j = 0; j <= n - 2; ++j) {
            prefix += R[j];
            total += std::ldexp(1.0, n - j - 2) / steps * (d[j] + prefix + 1.0);
        }
        return total;
    }
    const double w0 = std::ldexp(1.0, n - 2) / steps;
    double dual = 0.0, rate = 0.0;
    for (int j = n - 2; j >= 1; --j) {
        const double w = std::ldexp(1.0, n - j - 2) / steps;
        dual += w * d[j];
        rate += w;
        dual += rate * ((R[j] ? R[j] + 1.0 : 0.0) + 3.0 * S[j]);
    }
    dual += 2.0 * w0;
    if (!long_walk) return dual;
    double paired = 0.0, prefix = 0.0;
    for (int j = 1; j <= n - 2; ++j) {
        prefix += R[j];
        paired += std::ldexp(1.0, n - j - 2) / steps * (d[j] + prefix);
    }
    paired += w0 * (R[0] == 1 ? 2.0 : 3.0 * R[0] - 1.0);
    return std::min(dual, paired);
}

// Pairwise column swaps, first improvement, until none lowers the cost model
// (at most 16 sweeps).
static void search_order(const Matrix &m, int *cols, bool fp64, bool long_walk) {
    const int n = m.n;
    double best = order_cost(m, cols, fp64, long_walk);
    for (int sweep = 0; sweep < 16; ++sweep) {
        bool improved = false;
        for (int i = 0; i + 1 < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                std::swap(cols[i], cols[j]);
                const double c = order_cost(m, cols, fp64, long_walk);
                if (c < best - 1e-12) {
                    best = c;
                    improved = true;
                } else {
                    std::swap(cols[i], cols[j]);
                }
            }
        if (!improved) break;
    }
}

// Four-state chains (a design study; no kernel runs them): columns 0 and 1
// are never applied to x, and four chains hold the products for the four
// settings of the two columns, so every 4-step Gray quad flips only columns
// >= 2.  A flip of column j >= 2 updates its nnz_j rows and rebuilds levels
// j..2 of all four chains: a group of r rows is one product of r factors
// multiplied into four chains (r + 3 operations); a row of column 0 or 1
// whose next column is m joins level m as two variants (one add, four
// multiplications), a row of both as four (three adds, four
// multiplications).  Each quad's four products are combined and accumulated
// (four operations).  Per step, with Lemma 2's flip rates.
double cost_per_step_four_state(const Matrix &m, const int *cols) {
    const int n = m.n;
    if (n < 3) return 0.0;
    int R[kNMax], d[kNMax], S1[kNMax + 1] = {}, S2[kNMax + 1] = {};
    uint64_t seen = 0;
    for (int p = 0; p < n; ++p) {
        const uint64_t cm = m.colmask[cols[p]];
        d[p] = __builtin_popcountll(cm);
        R[p] = __builtin_popcountll(cm & ~seen);
        seen |= cm;
    }
    const uint64_t c0 = m.colmask[cols[0]], c1 = m.colmask[cols[1]];
    uint64_t one = c0 ^ c1, both = c0 & c1;
    for (int p = 2; p < n - 1; ++p) {
        const uint64_t cm = m.colmask[cols[p]];
        S1[p] = __builtin_popcountll(cm & one);
        S2[p] = __builtin_popcountll(cm & both);
        one &= ~cm;
        both &= ~cm;
    }
    const double steps = std::ldexp(1.0, n - 1) - 1.0;
    double total = 0.0, rate = 0.0;
    for (int j = n - 2; j >= 2; --j) {
        const double w = std::ldexp(1.0, n - j - 2) / steps;
        total += w * d[j];
        rate += w;   // level j is rebuilt by a flip of any column >= j
        total += rate * ((R[j] ? R[j] + 3.0 : 0.0) + 5.0 * S1[j] + 7.0 * S2[j]);
    }
    return total + 4.0 * std::ldexp(1.0, n - 3) / steps;
}

// The same pairwise-swap search as search_order, under the four-state model.
double four_state_searched(const Matrix &m, const int *cols_in) {
    const int n = m.n;
    if (n < 3) return 0.0;
    int cols[kNMax];
    for (int p = 0; p < n; ++p) cols[p] = cols_in[p];
    double best = cost_per_step_four_state(m, cols);
    for (int sweep = 0; sweep < 16; ++sweep) {
        bool improved = false;
        for (int i = 0; i + 1 < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                std::swap(cols[i], cols[j]);
                const double c = cost_per_step_four_state(m, cols);
                if (c < best - 1e-12) {
                    best = c;
                    improved = true;
                } else {
                    std::swap(cols[i], cols[j]);
                }
            }
        if (!improved) break;
    }
    return best;
}

double walk_cost_per_step(const Layout &L, bool fp64) {
    if (!fp64) return cost_per_step(L, false);
    const double dual = cost_per_step_dual(L, true);
    return L.n >= 31 ? std::min(dual, cost_per_step_paired(L)) : dual;
}

Layout choose_layout(const Matrix &m, int ordering_opt) {
    int cols[kNMax], rows[kNMax];
    if (ordering_opt == PERM_ORDER_NONE) { order_none(m, cols); return make_layout(m, cols, PERM_ORDER_NONE); }
    if (ordering_opt == PERM_ORDER_DEGREE) { order_degree(m, cols); return make_layout(m, cols, PERM_ORDER_DEGREE); }
    order_alg3(m, cols, rows);
    Layout paper = make_layout(m, cols, PERM_ORDER_PAPER);
    if (ordering_opt == PERM_ORDER_PAPER) return paper;
    order_degree(m, cols);
    Layout deg = make_layout(m, cols, PERM_ORDER_DEGREE);
    Layout start = cost_per_step(deg, false) < cost_per_step(paper, false) ? deg : paper;
    // AUTO / SEARCH: for FP64 walks of 2^21 steps and more, refine the better
    // order under the model of the scheme the walk will run (two-state chains
    // below n = 31, where the generic kernels run; the cheaper of those and the
    // paired chain from n = 31, the generated kernels' range).  The search
    // takes about 0.1-0.2 ms of host time at n = 22..28 and cuts the counted
    // FP64 operations of the batch workload's matrices there by 15-16 % (its
    // FP64 half: 2.15 s -> 1.76 s).  Exact kernels fold runs of rows in 32
    // bits, which the one-chain model does not see (a searched order made the
    // n=48 band's exact walk 7 % slower), so they keep the start order.
    if (m.n < 22 || m.is_int) return start;
    for (int p = 0; p < m.n; ++p) cols[p] = start.col_order[p];
    const bool fp64 = true, long_walk = m.n >= 31;
    const double before = order_cost(m, cols, fp64, long_walk);
    search_order(m, cols, fp64, long_walk);
    if (!(order_cost(m, cols, fp64, long_walk) < before - 1e-12)) return start;
    return make_layout(m, cols, PERM_ORDER_SEARCH);
}

int64_t threads_for_regs(int regs) {
    int r = std::max(regs, 16);
    r = (r + 7) / 8 * 8;                       // allocation granularity
    if (r > 255) return 0;
    int warps = kRegsPerSM / (r * 32);
    warps = std::min(warps, kMaxThreadsPerSM / 32);
    return (int64_t)kSMCount * warps * 32;
}

// Algorithm 4 (Partitioning), with column n-1 excluded (it never flips) and
// CalculateNoThreads given by GB300 occupancy at nregisters + base registers.
void partition_alg4(const Layout &L, double gr_ratio, int base_regs, int *k_out, int *c_out) {
    const int n = L.n;
    int k = 0, c = 0, nrows = 0;
    double best = 0.0;
    for (int j = 0; j <= n - 2; ++j) {
        nrows = std::max(nrows, L.group_begin[j + 1]);
        const int nregisters = nrows * 2;
        const double w = std::ldexp(1.0, -(j + 1));
        const double reg_cost = nregisters * (1.0 - w);
        const double glob_cost = (n - nrows) * w * gr_ratio;
        const double tau = (double)threads_for_regs(nregisters + base_regs);
        const double score = tau / (reg_cost + glob_cost);
        if (score > best || nrows == k) {
            best = score;
            k = nrows;
            c = j + 1;
        }
    }
    if (n < 2) { k = n; c = 0; }
    *k_out = k;
    *c_out = c;
}

// log2(r!) for a row or column count r <= 64, summed directly (no lgamma:
// it writes a process-wide sign variable, and plans are prepared on several
// threads).
static double log2_factorial(int r) {
    double s = 0.0;
    for (int k = 2; k <= r; ++k) s += std::log2((double)k);
    return s;
}

double bound_log2(const Matrix &m) {
    const int n = m.n;
    bool binary = true;
    for (int i = 0; i < n && binary; ++i)
        for (int j = 0; j < n; ++j)
            if (m.nz(i, j) && !(m.is_int ? m.ival(i, j) == 1 : m.fval(i, j) == 1.0)) { binary = false; break; }
    double rows = 0.0, cols = 0.0;
    for (int i = 0; i < n; ++i) {
        double rs = 0.0, cs = 0.0;
        for (int j = 0; j < n; ++j) {
            rs += std::fabs(m.fval(i, j));
            cs += std::fabs(m.fval(j, i));
        }
        if (rs == 0.0 || cs == 0.0) return -INFINITY;
        if (binary) {
            rows += log2_factorial((int)rs) / rs;   // Bregman-Minc
            cols += log2_factorial((int)cs) / cs;
        } else {
            rows += std::log2(rs);
            cols += std::log2(cs);
        }
    }
    return std::min(rows, cols);
}

double ring_ops_per_step(const Matrix &m, const Layout &L, int limbs, int fold) {
    const int n = m.n;
    if (n < 2 || limbs < 2) return 0.0;
    const double ring = limbs == 2 ? 3.0 : (double)limbs;
    double rs[kNMax];
    for (int s = 0; s < n; ++s) {
        double a = 0.0;
        for (int j = 0; j < n; ++j) a += std::fabs(m.fval(L.row_order[s], j));
        rs[s] = std::max(a, 1.0);
    }
    double level[kNMax + 1];
    for (int g = 0; g < n; ++g) {
        const int b = L.group_begin[g], e = L.group_begin[g + 1];
        double c = 0.0;
        int s = b;
        while (s < e) {
            int t = s + 1;
            if (fold == 1) {
                double bound = rs[s];
                while (t < e && bound * rs[t] < 2147483647.0) bound *= rs[t++];
            } else if (fold == 2) {
                while (t < e && (t & 3) != 0) ++t;   // to the end of the slot quadruple
            }
            c += (t - s - 1) + ring;
            s = t;
        }
        level[g] = c;
    }
    const double steps = std::ldexp(1.0, n - 1) - 1.0;
    double total = level[0], prefix = 0.0;
    for (int j = 1; j <= n - 2; ++j) {
        prefix += level[j];
        total += std::ldexp(1.0, n - j - 2) / steps * prefix;
    }
    return total;
}

int abs_shift_for(const Matrix &m) {
    double L = 0.0;
    for (int i = 0; i < m.n; ++i) {
        double rs = 0.0;
        for (int j = 0; j < m.n; ++j) rs += std::fabs(m.fval(i, j));
        if (rs > 0.0) L += std::log2(rs / 2.0);
    }
    const double s = std::ceil(L) - 120.0;
    return (int)std::min(1100.0, std::max(-890.0, s));
}

int exact_words_for(double bound, int n) {
    if (!(bound < 125.0)) return 0;               // result must fit a signed 128-bit integer
    for (int w = 1; w <= 3; ++w)
        if (64.0 * w >= bound + n + 2.0) return w; // (n-1) bits of scale, a sign bit, a margin
    return 0;
}

int exact_limbs_for(double bound, int n) {
    if (!(bound < 125.0)) return 0;
    for (int l = 2; l <= 6; ++l)
        if (32.0 * l >= bound + n + 2.0) return l;
    return 0;
}

std::vector<Launch> alg2_launches(int64_t tau, int n) {
    std::vector<Launch> out;
    int64_t start = 1;
    const int64_t end = (int64_t)1 << (n - 1);
    while (end - start > 0) {
        int64_t delta = 1024;
        while (delta * tau <= end - start) delta *= 2;
        delta /= 2;
        if (delta == 512) {
            out.push_back({start, 1024, end});
            break;
        }
        out.push_back({start, delta, end});
        start += tau * delta;
    }
    return out;
}

double zero_term_fraction(const Matrix &m, const int *col_order, int samples) {
    const int n = m.n;
    if (n < 2 || samples < 1) return 0.0;
    double x0[kNMax];
    for (int i = 0; i < n; ++i) {
        double rs = 0.0;
        for (int j = 0; j < n; ++j) rs += m.fval(i, j);
        x0[i] = m.fval(i, col_order[n - 1]) - 0.5 * rs;
    }
    uint64_t state = 0x9e3779b97f4a7c15ull;   // splitmix64
    auto next = [&state]() {
        uint64_t z = (state += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    };
    int zero = 0;
    for (int t = 0; t < samples; ++t) {
        const uint64_t S = next();
        bool any = false;
        for (int i = 0; i < n && !any; ++i) {
            double x = x0[i];
            for (int p = 0; p < n - 1; ++p)
                if (((S >> p) & 1ull) && m.nz(i, col_order[p])) x += m.fval(i, col_order[p]);
            any = x == 0.0;
        }
        zero += any;
    }
    return (double)zero / samples;
}

}  // namespace perm
