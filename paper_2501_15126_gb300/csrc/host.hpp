// host.hpp -- host-side preprocessing of a permanent plan (C++).
//
// Ingest (CSR/CSC -> dense, validation), the structural guard (perfect
// matching), column ordering (degree sort of Sec. VI-B, PermanentOrdering of
// Algorithm 3), the row grouping behind the product chain, the step-cost
// model (Lemma 2 weights), Partitioning (Algorithm 4), the a-priori bound that
// sizes the exact path, and the Gray-code helpers of Sec. IV.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "perm.h"

namespace perm {

constexpr int kNMax = 64;
constexpr int kBlockLog2 = 5;         // B: 2^B Gray steps unrolled per block
constexpr int kSMCount = 152;         // GB300
constexpr int kRegsPerSM = 65536;
constexpr int kMaxThreadsPerSM = 2048;

// A dense copy of the input.  The n*n entries live either in the matrix's own
// vector or in caller storage (the allocation-free entry point); the matrix is
// not copyable because it may point into its own vector.
struct Matrix {
    int n = 0;
    bool is_int = false;
    double *f = nullptr;      // n*n row-major (FP64 inputs)
    int64_t *v = nullptr;     // n*n row-major (integer inputs)
    std::vector<unsigned char> own;
    uint64_t rowmask[kNMax] = {};
    uint64_t colmask[kNMax] = {};
    Matrix() = default;
    Matrix(const Matrix &) = delete;
    Matrix &operator=(const Matrix &) = delete;
    bool nz(int i, int j) const { return (rowmask[i] >> j) & 1ull; }
    double fval(int i, int j) const { return is_int ? (double)v[(size_t)i * n + j] : f[(size_t)i * n + j]; }
    int64_t ival(int i, int j) const { return v[(size_t)i * n + j]; }
};

// Copies and validates a borrowed matrix.  Explicit zeros are dropped.  With
// `storage` (at least n*n*8 bytes) nothing is allocated.  *err is set to a
// static message on failure.
perm_status_t ingest(const perm_matrix_t *A, Matrix &out, const char **err, void *storage = nullptr,
                     size_t storage_bytes = 0);

// Dense row-major input (internal use by the batch path and tests).
bool has_perfect_matching(const Matrix &m);

// The plan's ordering of rows and columns.
struct Layout {
    int n = 0;
    int ordering = PERM_ORDER_NONE;
    int col_order[kNMax] = {};     // position p -> original column
    int row_order[kNMax] = {};     // slot r -> original row
    int slot_of_row[kNMax] = {};   // original row -> slot
    int group_of_slot[kNMax] = {}; // first column position touching the slot's row
    int group_begin[kNMax + 1] = {};  // slots of group m are [group_begin[m], group_begin[m+1])
    uint64_t colmask[kNMax] = {};  // by position p: slots touched by that column
    int col_nnz[kNMax] = {};
    int top = 0;                   // highest nonempty group
    // Column 0's rows (group 0, slots [0, group_begin[1])) split by the next
    // position that touches them: S_m = slots [s_begin[m], s_begin[m+1]),
    // m = 1..n-1 (m = n-1: no flipped column touches them again).
    int s_begin[kNMax + 1] = {};
    int top_dual = 0;              // highest m with group m or S_m nonempty
};

// Column orders.  PAPER is Algorithm 3; its row order is returned too.
void order_none(const Matrix &m, int *col_order);
void order_degree(const Matrix &m, int *col_order);
void order_alg3(const Matrix &m, int *col_order, int *row_order);

// Builds the slot layout for a column order: slots sorted by group, and
// inside a group in the order the rows were first touched.
Layout make_layout(const Matrix &m, const int *col_order, int ordering);

// Fraction of the walk's terms (Algorithm 1: the subsets of the first n-1
// ordered columns) whose product has a zero factor, estimated from `samples`
// subsets drawn by a fixed-seed generator (each column in with probability
// 1/2): x_i = a_{i,last} - (1/2) sum_j a_ij + the subset's entries of row i.
double zero_term_fraction(const Matrix &m, const int *col_order, int samples);

// Arithmetic ops per Gray step (Lemma 2 weights 2^(n-j-2)/(2^(n-1)-1)):
// chain scheme: nnz_j updates + |R_0|+...+|R_j| multiplies + 1 accumulate;
// paper scheme: nnz_j updates + (n-1) multiplies + 1 accumulate.
double cost_per_step(const Layout &L, bool paper_scheme);
// The same walk with even/odd steps paired (the generated FP64 kernels):
// per pair, column 0's r = |R_0| updates, 2r-2 multiplies/fused multiply-adds
// for prod x - prod (x + s a_0), and one fused multiply-add into the sum; the
// even step's flip rebuilds levels j..1 only.
double cost_per_step_paired(const Layout &L);

// Chooses the ordering (AUTO = cheaper of DEGREE and PAPER under the model).
Layout choose_layout(const Matrix &m, int ordering_opt);

// Algorithm 4 with GB300 occupancy; returns k (register rows) and c.
void partition_alg4(const Layout &L, double gr_ratio, int base_regs, int *k, int *c);

// GB300 resident threads for a kernel using `regs` registers per thread.
int64_t threads_for_regs(int regs);

// log2 of an a-priori bound on |perm(A)|: Bregman-Minc for 0/1 matrices,
// otherwise min over rows/cols of prod of absolute sums.  -inf for zero rows.
double bound_log2(const Matrix &m);

// The scale of the FP64 walks' sum of |terms|: every |x_i(g)| is at most half
// row i's absolute sum, so every term is at most 2^L, L = sum_i log2(r_i / 2);
// the kernels accumulate sum|terms| 2^-shift with shift = ceil(L) - 120
// (clamped to the range the FP32 accumulation can take).
int abs_shift_for(const Matrix &m);

// Smallest w in 1..3 with the doubled-NW sum recoverable modulo 2^(64 w),
// or 0 when even w = 3 is not enough.
int exact_words_for(double bound, int n);
// Operations per Gray step of the generic kernels' two-state chains (column 0
// folded into a second chain): flips of columns >= 1, the levels they
// rebuild, and one difference and accumulation per pair of steps.
double cost_per_step_dual(const Layout &L, bool shared_product);
// The model of the scheme a walk of this layout runs: FP64 two-state chains
// (or, for walks long enough for the generated kernels, the cheaper of those
// and the paired chain); exact: one chain.
double walk_cost_per_step(const Layout &L, bool fp64);
// Integer multiply operations per Gray step of an exact walk (the IMAD pipe's
// work, which bounds it): a ring product of an L-limb value by a 32-bit factor
// is L wide multiply-adds (3 for L = 2: one 64-bit product), and every extra
// row folded into a 32-bit product before it is one more multiplication.
// Level 0 is rebuilt at every step and levels 1..j after a flip of column j
// (Lemma 2 weights).  fold: 0 = one ring product per row, 1 = runs of a
// group's rows whose row-sum product stays below 2^31 (generated kernels),
// 2 = fixed slot quadruples (generic kernels, rows' absolute sums <= 127).
double ring_ops_per_step(const Matrix &m, const Layout &L, int limbs, int fold);
// Four-state chains (a design study): FP64 operations per step on a column
// order, and after a pairwise-swap search for that model.
double cost_per_step_four_state(const Matrix &m, const int *cols);
double four_state_searched(const Matrix &m, const int *cols);

// The fewest 32-bit limbs (2..6) of a ring that holds 2^(n-1) perm with sign
// and margin, or 0.
int exact_limbs_for(double bound, int n);

// Theorem 1: column flipped at step i >= 1 and its sign.
inline int scbs_col(uint64_t i) { return __builtin_ctzll(i); }
inline int scbs_sign(uint64_t i) { int j = __builtin_ctzll(i); return ((i >> (j + 1)) & 1ull) ? -1 : 1; }

// Algorithm 2 (GenerateLaunchParameters).
struct Launch { int64_t start, delta, end; };
std::vector<Launch> alg2_launches(int64_t tau, int n);

}  // namespace perm
