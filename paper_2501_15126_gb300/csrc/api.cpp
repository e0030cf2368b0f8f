// api.cpp -- the C ABI of libperm (see include/perm.h): plans, compute,
// inspection helpers.  Batch and serving live in batch.cpp / server.cpp.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "codegen.hpp"
#include "host.hpp"
#include "kernels.hpp"
#include "plan.hpp"

namespace perm {

// The last error message of the calling thread: a fixed buffer, so that
// reporting an error never allocates.
static thread_local char g_last_error[512];

static void set_error(const char *a, const char *b) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s%s%s", a ? a : "", (a && b) ? ": " : "", b ? b : "");
}

perm_status_t fail(perm_status_t s, const char *msg) {
    set_error(msg, nullptr);
    return s;
}

perm_status_t fail(perm_status_t s, const std::string &msg) { return fail(s, msg.c_str()); }

perm_status_t cuda_fail(cudaError_t e, const char *what) {
    set_error(what, cudaGetErrorString(e));
    return PERM_ERR_CUDA;
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int nmax_bucket(int n) {
    if (n <= 16) return 16;
    if (n <= 32) return 32;
    if (n <= 48) return 48;
    return 0;
}

static int floor_log2(uint64_t v) { return v ? 63 - __builtin_clzll(v) : -1; }

// Builds the shared-memory image read by the generic kernels.
// Image layout (see devmat.h): 16-byte header, column masks, group masks,
// column offsets (u16), x0, then the values of columns 0..n-2 in slot order.
static size_t devmat_head(int nmax) { return 48 + 12 * (size_t)nmax; }
typedef pk::DevMat<16, double> DevMat16F;
typedef pk::DevMat<32, int> DevMat32I;
typedef pk::DevMat<48, double> DevMat48F;
static_assert(offsetof(DevMat16F, x0) == 48 + 12 * 16, "image header");
static_assert(offsetof(DevMat32I, x0) == 48 + 12 * 32, "image header");
static_assert(offsetof(DevMat48F, x0) == 48 + 12 * 48, "image header");
struct HostDD { double h, l; };
static_assert(offsetof(DevMat48F, val) == 48 + 12 * 48 + 8 * 48, "image values");
typedef pk::DevMat<32, double, HostDD> DevMat32DD;
static_assert(offsetof(DevMat32DD, val) == 48 + 12 * 32 + 16 * 32, "double-double image values");

// value and start-value sizes of an image layout (kImgF64, kImgInt, kImgDD)
static size_t img_vsz(int img) { return img == kImgInt ? sizeof(int) : sizeof(double); }
static size_t img_x0sz(int img) { return img == kImgDD ? 2 * sizeof(double) : img_vsz(img); }

size_t devmat_bytes(int img, int nmax, int nnz) {
    const size_t b = devmat_head(nmax) + img_x0sz(img) * (size_t)nmax + img_vsz(img) * (size_t)nnz;
    return (b + 15) & ~(size_t)15;
}

static int devmat_nnz(const Layout &L) {
    int nnz = 0;
    for (int p = 0; p + 1 < L.n; ++p) nnz += L.col_nnz[p];
    return nnz;
}

size_t devmat_bytes_for(const Layout &L, int img, int nmax) { return devmat_bytes(img, nmax, devmat_nnz(L)); }

void build_devmat(const Matrix &m, const Layout &L, int img, int nmax, std::vector<unsigned char> &out) {
    out.assign(devmat_bytes(img, nmax, devmat_nnz(L)), 0);
    build_devmat_into(m, L, img, nmax, out.data());
}

// x0_i = a_{i,last} - (1/2) sum_j a_ij as an exact double-double (hi, lo):
// halving is exact and every partial sum is accumulated with TwoSum, so no bit
// is lost while the value fits 106 bits (values on a common 2^-53 grid do).
static void x0_dd(const Matrix &m, int r, int last, double *hi_out, double *lo_out) {
    double hi = 0.0, lo = 0.0;
    auto add = [&](double v) {
        const double s = hi + v;
        const double bb = s - hi;
        lo += (hi - (s - bb)) + (v - bb);
        hi = s;
    };
    for (int j = 0; j < m.n; ++j) add(-0.5 * m.fval(r, j));
    add(m.fval(r, last));
    const double s = hi + lo;
    *lo_out = lo - (s - hi);
    *hi_out = s;
}

void build_devmat_into(const Matrix &m, const Layout &L, int img, int nmax, unsigned char *dst) {
    const int n = m.n;
    const int last = L.col_order[n - 1];
    const size_t vsz = img_vsz(img), x0sz = img_x0sz(img);
    const int nnz = devmat_nnz(L);
    const size_t bytes = devmat_bytes(img, nmax, nnz);
    std::memset(dst, 0, bytes);
    int32_t *hdr = reinterpret_cast<int32_t *>(dst);
    hdr[0] = n;
    hdr[1] = L.top_dual;
    hdr[2] = nnz;
    hdr[3] = (int32_t)bytes;
    uint64_t *colmask = reinterpret_cast<uint64_t *>(dst + 16);
    uint16_t *colptr = reinterpret_cast<uint16_t *>(colmask + nmax);
    uint8_t *gbegin = reinterpret_cast<uint8_t *>(colptr + nmax);
    uint8_t *sbegin = gbegin + nmax + 16;
    for (int p = 0; p + 1 < n; ++p) colmask[p] = L.colmask[p];
    for (int g = 0; g <= n; ++g) gbegin[g] = (uint8_t)L.group_begin[g];
    for (int g = 0; g <= n; ++g) sbegin[g] = (uint8_t)L.s_begin[g];
    unsigned char *x0 = dst + devmat_head(nmax);
    unsigned char *val = x0 + x0sz * nmax;
    for (int s = 0; s < n; ++s) {
        const int r = L.row_order[s];
        if (img == kImgDD) {
            double v[2];
            x0_dd(m, r, last, &v[0], &v[1]);
            std::memcpy(x0 + x0sz * s, v, x0sz);
        } else if (img == kImgF64) {
            double rowsum = 0.0;
            for (int j = 0; j < n; ++j) rowsum += m.fval(r, j);
            const double v = m.fval(r, last) - rowsum / 2.0;
            std::memcpy(x0 + vsz * s, &v, vsz);
        } else {
            int64_t rowsum = 0;
            for (int j = 0; j < n; ++j) rowsum += m.ival(r, j);
            const int v = (int)(2 * m.ival(r, last) - rowsum);
            std::memcpy(x0 + vsz * s, &v, vsz);
        }
    }
    int k = 0;
    for (int p = 0; p + 1 < n; ++p) {
        const int c = L.col_order[p];
        colptr[p] = (uint16_t)k;
        for (int s = 0; s < n; ++s) {
            if (!((L.colmask[p] >> s) & 1ull)) continue;
            const int r = L.row_order[s];
            unsigned char *d = val + vsz * (size_t)k++;
            if (img != kImgInt) { const double v = m.fval(r, c); std::memcpy(d, &v, vsz); }
            else { const int v = (int)(2 * m.ival(r, c)); std::memcpy(d, &v, vsz); }
        }
    }
}

// The CSC image of the x-in-shared-memory baseline (xshared.cu): header
// (n, nnz, bytes, 0), colptr[n] and rows[nnz] (int32, original rows), then
// 8-byte aligned x0[n] and vals[nnz]; columns are positions 0..n-2 of the
// plan's order, x0 by original row.
void build_xshared_image(const perm_plan_s &P, std::vector<unsigned char> &img) {
    const Matrix &m = P.m;
    const int n = m.n;
    const int last = P.L.col_order[n - 1];
    std::vector<int32_t> colptr(n, 0), rows;
    std::vector<double> vals;
    for (int p = 0; p + 1 < n; ++p) {
        colptr[p] = (int32_t)rows.size();
        const int c = P.L.col_order[p];
        for (int i = 0; i < n; ++i)
            if (m.nz(i, c)) { rows.push_back(i); vals.push_back(m.fval(i, c)); }
    }
    colptr[n - 1] = (int32_t)rows.size();
    const int nnz = (int)rows.size();
    size_t off = 16 + 4 * (size_t)(n + nnz);
    off = (off + 7) & ~(size_t)7;
    const size_t bytes = (off + 8 * (size_t)(n + nnz) + 15) & ~(size_t)15;
    img.assign(bytes, 0);
    int32_t *h = reinterpret_cast<int32_t *>(img.data());
    h[0] = n;
    h[1] = nnz;
    h[2] = (int32_t)bytes;
    std::memcpy(h + 4, colptr.data(), 4 * (size_t)n);
    if (nnz) std::memcpy(h + 4 + n, rows.data(), 4 * (size_t)nnz);
    double *x0 = reinterpret_cast<double *>(img.data() + off);
    for (int i = 0; i < n; ++i) {
        double rowsum = 0.0;
        for (int j = 0; j < n; ++j) rowsum += m.fval(i, j);
        x0[i] = m.fval(i, last) - rowsum / 2.0;
    }
    if (nnz) std::memcpy(x0 + n, vals.data(), 8 * (size_t)nnz);
}

// Checks that the exact walk's doubled row sums fit int32.
static bool exact_fits_int32(const Matrix &m) {
    for (int i = 0; i < m.n; ++i) {
        int64_t s = 0;
        for (int j = 0; j < m.n; ++j) {
            const int64_t v = m.ival(i, j);
            if (v > (1ll << 29) || v < -(1ll << 29)) return false;
            s += v < 0 ? -v : v;
            if (s > (1ll << 29)) return false;
        }
    }
    return true;
}

perm_status_t plan_prepare(const perm_matrix_t *A, const perm_opts_t *opts_in, perm_plan_s &P, void *storage,
                           size_t storage_bytes) {
    const double t0 = now_ms();
    perm_opts_t opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    const char *err = nullptr;
    perm_status_t st = ingest(A, P.m, &err, storage, storage_bytes);
    if (st != PERM_OK) return fail(st, err);
    const int n = P.m.n;
    P.opts = opts;
    P.arith = 0;
    P.total = 1ull << (n - 1);
    P.g_lo = opts.g_lo;
    P.g_hi = opts.g_hi;
    P.subrange = !(opts.g_lo == 0 && opts.g_hi == 0);
    if (!P.subrange) { P.g_lo = 0; P.g_hi = P.total; }
    if (P.g_lo > P.g_hi || P.g_hi > P.total) return fail(PERM_ERR_ARG, "sub-range outside [0, 2^(n-1))");
    if (P.subrange && ((P.g_lo % 32) || ((P.g_hi % 32) && P.g_hi != P.total)))
        return fail(PERM_ERR_ARG, "sub-range ends must be multiples of 32");
    if (opts.ordering < 0 || opts.ordering > PERM_ORDER_SEARCH) return fail(PERM_ERR_ARG, "bad ordering");
    if (opts.ordering == PERM_ORDER_SEARCH) opts.ordering = PERM_ORDER_AUTO;
    if (opts.engine < 0 || opts.engine > PERM_ENGINE_XSHARED) return fail(PERM_ERR_ARG, "bad engine");
    if (opts.engine == PERM_ENGINE_XSHARED && A->vtype != PERM_F64)
        return fail(PERM_ERR_ARG, "the x-in-shared-memory baseline takes FP64 inputs only");
    if (opts.exact_words < 0 || opts.exact_words > 3) return fail(PERM_ERR_ARG, "exact_words must be 0..3");
    if (opts.chunk_log2 < 0 || opts.chunk_log2 > 63) return fail(PERM_ERR_ARG, "bad chunk_log2");
    if (opts.threads < 0) return fail(PERM_ERR_ARG, "threads < 0");
    if (opts.timeout_ms < 0) return fail(PERM_ERR_ARG, "timeout_ms < 0");
    if (opts.precision < PERM_PREC_AUTO || opts.precision > PERM_PREC_DD) return fail(PERM_ERR_ARG, "bad precision");
    if (opts.shared_rows < 0) return fail(PERM_ERR_ARG, "shared_rows < 0");
    P.zero = !has_perfect_matching(P.m);
    if (!P.m.is_int) {
        P.abs_shift = abs_shift_for(P.m);
        P.dd = opts.precision == PERM_PREC_DD;
    }
    P.L = choose_layout(P.m, opts.ordering);
    P.ops_per_step = cost_per_step(P.L, false);
    P.ops_per_step_paper = cost_per_step(P.L, true);
    if (P.m.is_int) {
        const double b = bound_log2(P.m);
        P.bound = b;
        int w = exact_words_for(b, n);
        if (!exact_fits_int32(P.m)) return fail(PERM_ERR_OVERFLOW, "integer entries too large for the exact walk");
        if (!P.zero) {
            if (opts.exact_words) {
                if (!P.subrange && w && opts.exact_words < w)
                    return fail(PERM_ERR_OVERFLOW, "exact_words too small for this matrix's bound");
                w = opts.exact_words;
            } else if (!w) {
                if (P.subrange) w = 3;
                else return fail(PERM_ERR_OVERFLOW, "|perm| bound exceeds the 2^191 exact mode");
            }
        }
        P.arith = w ? w : 1;
        // the narrowest ring of 32-bit limbs that holds the whole sum; a
        // sub-range (a partial sum reported modulo 2^(64 arith)) or an
        // explicit width keeps all 2 arith limbs
        P.limbs = 2 * P.arith;
        if (!opts.exact_words && !P.subrange && !P.zero) {
            const int l = exact_limbs_for(b, n);
            if (l && (l + 1) / 2 == P.arith) P.limbs = l;
        }
        // |x_i| <= sum_j |a_ij| at every Gray index: four factors <= 127 fit 32 bits
        int64_t max_row = 0;
        for (int i = 0; i < n; ++i) {
            int64_t rs = 0;
            for (int j = 0; j < n; ++j) rs += P.m.ival(i, j) < 0 ? -P.m.ival(i, j) : P.m.ival(i, j);
            max_row = std::max(max_row, rs);
        }
        P.fold = max_row <= 127;
    }
    // an empty sub-range [g, g) (g > 0; both ends 0 mean the whole walk) has
    // the partial sum 0: nothing launches, and the ring width above stays
    // the one a non-empty sub-range of this matrix reports
    if (P.subrange && P.g_lo == P.g_hi) P.zero = true;
    P.ms_plan = now_ms() - t0;
    return PERM_OK;
}

// Chooses K, grid and block for a walk over [g_lo, g_hi).
perm_status_t choose_launch(perm_plan_s &P, int block_log2, int blocks_per_sm, int block) {
    const uint64_t len = P.g_hi - P.g_lo;
    const int n = P.m.n;
    int kmax = n - 1;
    if (P.g_lo) kmax = std::min(kmax, __builtin_ctzll(P.g_lo));
    if (P.g_hi != P.total || P.subrange) kmax = std::min(kmax, P.g_hi ? __builtin_ctzll(P.g_hi) : 63);
    kmax = std::min(kmax, floor_log2(len));
    const int64_t resident_warps = (int64_t)kSMCount * blocks_per_sm * (block / 32);
    int K = P.opts.chunk_log2;
    if (!K) {
        // enough 32-chunk tasks for every resident warp several times over, but
        // chunks of at least 2^(B+3) steps so the start vector stays a small cost
        const double want_tasks = 64.0 * (double)resident_warps;   // keeps the last round of tasks short
        K = floor_log2((uint64_t)std::max(1.0, (double)len / (32.0 * want_tasks)));
        int k_floor = block_log2 + 3;
        if (P.arith != 0) {
            // an exact walk too short to give every resident warp a task at that
            // length takes chunks down to 2^(B+1) (its start vector is a few
            // integer adds per column): the n=24 0/1 walk, 2^23 steps, takes
            // 0.081 ms at 2^6-step chunks against 0.132 ms at 2^8, where 72 % of
            // the warps had no task.  FP64 walks keep 2^(B+3) (the same matrix
            // in FP64: 0.220 ms at 2^8, 0.228 at 2^6).
            const int fill = floor_log2((uint64_t)std::max(1.0, (double)len / (32.0 * (double)resident_warps)));
            k_floor = std::max(block_log2 + 1, std::min(k_floor, fill));
        }
        K = std::max(K, k_floor);
    } else {
        K = std::max(K, block_log2);   // a chunk holds whole blocks
    }
    K = std::min(K, kmax);
    if (K < block_log2) return fail(PERM_ERR_ARG, "range too short or misaligned for the chunk size");
    P.K = K;
    P.chunk_lo = P.g_lo >> K;
    P.chunk_hi = P.g_hi >> K;
    P.ntasks = (P.chunk_hi - P.chunk_lo + 31) / 32;
    P.block = block;
    int64_t grid = (int64_t)kSMCount * blocks_per_sm;
    if (P.opts.threads) grid = std::max<int64_t>(1, P.opts.threads / block);
    grid = std::min<int64_t>(grid, ((int64_t)P.ntasks * 32 + block - 1) / block);
    P.grid = (int)std::max<int64_t>(1, grid);
    return PERM_OK;
}

// The register rows requested by the caller, rounded down to whole groups.
void split_for_rows(const Layout &L, int rows, int *k, int *c) {
    const int n = L.n;
    rows = std::min(rows, n);
    int cc = 0;
    while (cc + 1 <= n - 1 && L.group_begin[cc + 1] <= rows) ++cc;
    *c = cc;
    *k = L.group_begin[cc];
}

// The generated kernel keeps every row reached inside the unrolled block in
// registers: c >= B.  k = n means no global rows.
void normalise_split(const Layout &L, int B, int *k, int *c) {
    const int n = L.n;
    if (*c < B) { *c = std::min(B, n - 1); *k = L.group_begin[*c]; }
    if (*c >= n - 1 || *k >= n) { *k = n; *c = n - 1; }
    if (*k < 1) *k = 1;
}

// The generated kernel's layout: the Algorithm 4 split (or the caller's
// register rows) and, for FP64, the cheaper of the paired chain and the
// two-state chains under the cost model.
static void codegen_layout(perm_plan_s &P) {
    const int n = P.m.n;
    int k = n, c = n - 1;
    const double gr = P.opts.gr_ratio > 0 ? P.opts.gr_ratio : kDefaultGRRatio;
    // Walks where most terms are zero (repeated values, Sec. VI-E): FP64 ones
    // keep short blocks, so that the zero skip starts at 2^5 steps, and the
    // kernel widens its skips into zero spans where a warp's lanes can share
    // their zero rows: the 32 chunks of a warp differ in six columns, which
    // must leave rows untouched, i.e. touch fewer than n rows on average
    // (density below 1/6).  Elsewhere the span code only costs registers (the
    // mycielskian6 shape, density 0.21: 255 instead of 128, 16 % slower).
    P.zero_frac = zero_term_fraction(P.m, P.L.col_order, 1024);
    P.zero_heavy = P.zero_frac > 0.25;
    int nnz = 0;
    for (int i = 0; i < n; ++i) nnz += __builtin_popcountll(P.m.rowmask[i]);
    P.zero_spans = P.zero_heavy && 6 * nnz < n * n;
    partition_alg4(P.L, gr, kCodegenBaseRegs, &k, &c);   // Algorithm 4
    if (P.opts.reg_rows > 0) split_for_rows(P.L, P.opts.reg_rows, &k, &c);
    normalise_split(P.L, codegen_block_log2(P), &k, &c);
    P.pure_reg = (P.opts.flags & PERM_FLAG_PURE_REG) != 0;
    // the middle tier: shared memory holds up to 96 KB of x per 256-thread block
    // (two blocks per SM), i.e. 48 FP64 or 96 int32 rows
    const int cap = (int)(96 * 1024 / (256 * (P.arith == 0 ? 8 : 4)));
    P.k2 = P.pure_reg ? 0 : std::max(0, std::min({P.opts.shared_rows, n - k, cap}));
    // sum|terms| costs the generated FP64 kernels about a tenth of their speed:
    // they keep it where precision AUTO may need it (whole walks of n <= 32),
    // or when asked (PERM_FLAG_ABS_SUM)
    P.want_abs = P.arith == 0 && ((P.opts.flags & PERM_FLAG_ABS_SUM) ||
                                  (P.opts.precision == PERM_PREC_AUTO && !P.subrange && n <= kAutoDDMaxN));
    if (P.pure_reg) {   // CodeGen-PureReg: every row in registers, no chain
        k = n;
        c = n - 1;
    }
    P.k = k;
    P.c = c;
    P.dual = false;
    if (P.pure_reg) {
        P.ops_per_step = cost_per_step(P.L, true);
    } else if (P.arith == 0) {
        const double paired = cost_per_step_paired(P.L), dual = cost_per_step_dual(P.L, true);
        P.dual = dual < paired && !(P.opts.flags & PERM_FLAG_PAIRED_CHAIN);
        P.ops_per_step = P.dual ? dual : paired;
    }
}

perm_status_t plan_device_setup(perm_plan_s &P) {
    const int n = P.m.n;
    cudaError_t e;
    const double t0 = now_ms();
    if (P.zero) return PERM_OK;
    int engine = P.opts.engine;
    const bool tiny = n <= 8;
    if (engine == PERM_ENGINE_AUTO) engine = (n > 48 || (!tiny && P.len() >= (1ull << 30))) ? PERM_ENGINE_CODEGEN
                                                                                            : PERM_ENGINE_GENERIC;
    if (P.dd) {   // double-double walks run the precompiled generic kernels only
        if (n > 48) return fail(PERM_ERR_SIZE, "double-double walks cover n <= 48");
        engine = PERM_ENGINE_GENERIC;
    }
    if (engine == PERM_ENGINE_GENERIC && n > 48) return fail(PERM_ERR_SIZE, "generic kernels cover n <= 48");
    const int nmax = nmax_bucket(std::min(n, 48));
    if (tiny && engine != PERM_ENGINE_XSHARED) engine = PERM_ENGINE_GENERIC;
    if (P.dd && engine == PERM_ENGINE_XSHARED) return fail(PERM_ERR_ARG, "the x-in-shared-memory baseline is FP64 only");
    P.engine = engine;
    P.words = result_words(P.arith);

    if (engine == PERM_ENGINE_XSHARED) {
        std::vector<unsigned char> img;
        build_xshared_image(P, img);
        P.img_bytes = img.size();
        if ((e = cudaMalloc(&P.d_devmat, img.size())) != cudaSuccess) return cuda_fail(e, "cudaMalloc(CSC image)");
        if ((e = cudaMemcpy(P.d_devmat, img.data(), img.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy(CSC image)");
        cudaFuncAttributes attr;
        if ((e = xshared_attr(&attr)) != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
        P.regs = attr.numRegs;
        int bps = 0;
        if ((e = xshared_occupancy(n, (int)P.img_bytes, 256, &bps)) != cudaSuccess) return cuda_fail(e, "occupancy");
        perm_status_t st = choose_launch(P, 0, std::max(bps, 1), 256);
        if (st != PERM_OK) return st;
    } else if (engine == PERM_ENGINE_GENERIC) {
        P.gf = generic_fns(nmax, P.kind());
        if (!P.gf.walk) return fail(PERM_ERR_INTERNAL, "no generic kernel for this size");
        P.nmax = nmax;
        std::vector<unsigned char> img;
        build_devmat(P.m, P.L, P.img_kind(), nmax, img);
        P.img_bytes = img.size();
        if ((e = cudaMalloc(&P.d_devmat, img.size())) != cudaSuccess) return cuda_fail(e, "cudaMalloc(devmat)");
        if ((e = cudaMemcpy(P.d_devmat, img.data(), img.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy(devmat)");
        cudaFuncAttributes attr;
        if ((e = P.gf.attr(&attr)) != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
        P.regs = attr.numRegs;
        if (tiny) {
            P.direct = true;
            P.block = 256;
            P.grid = (int)((P.g_hi - P.g_lo + 255) / 256);
            P.ntasks = (uint64_t)P.grid;
            P.K = 0;
        } else {
            int bps = 0;
            if ((e = P.gf.occ(256, img.size(), &bps)) != cudaSuccess) return cuda_fail(e, "occupancy");
            perm_status_t st = choose_launch(P, P.gf.block_log2, std::max(bps, 1), 256);
            if (st != PERM_OK) return st;
        }
    } else {
        codegen_layout(P);
        std::string err;
        perm_status_t st = codegen_build(P, err);
        if (st != PERM_OK) return fail(st, err);
        st = choose_launch(P, P.cg.block_log2, std::max(P.cg.blocks_per_sm, 1), P.cg.block);
        if (st != PERM_OK) return st;
        if (P.k + P.k2 < n) {
            const size_t bytes = (size_t)(n - P.k - P.k2) * (size_t)P.grid * P.block * (P.arith == 0 ? 8 : 4);
            if ((e = cudaMalloc(&P.d_xglob, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(x global rows)");
        }
    }
    const size_t ws_words = kWsTaskOut + (size_t)P.ntasks * P.words;
    if ((e = cudaMalloc(&P.d_ws, ws_words * 8)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
    if (engine == PERM_ENGINE_GENERIC && !P.direct) {
        pk::BatchMat bm;
        std::memset(&bm, 0, sizeof(bm));
        bm.task_begin = 0;
        bm.out_offset = 0;
        bm.image = 0;
        bm.chunk_lo = P.chunk_lo;
        bm.chunk_hi = P.chunk_hi;
        bm.K = P.K;
        bm.abs_shift = P.abs_shift;
        if ((e = cudaMemcpy(P.d_ws + kWsBatchMat, &bm, sizeof(bm), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy(batch table)");
    }
    if ((e = cudaMallocHost(&P.h_res, 8 * 8)) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    if ((e = cudaEventCreate(&P.ev0)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&P.ev1)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    P.ms_plan += now_ms() - t0 - P.ms_compile;
    return PERM_OK;
}

// Launches the walk and the reduction; no synchronisation.  With
// record_events false (graph capture) the timing events are left out: a
// replayed graph is timed by events around its launch instead.
perm_status_t plan_launch(perm_plan_s &P, cudaStream_t st, bool record_events) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(P.d_ws, 0, 8 * 8, st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    uint64_t *task_out = P.d_ws + kWsTaskOut;
    if (record_events && (e = cudaEventRecord(P.ev0, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if (P.direct) {
        e = P.gf.direct(P.d_devmat, P.g_lo, P.g_hi, task_out, P.grid, P.block, st, P.abs_shift);
        if (e != cudaSuccess) return cuda_fail(e, "direct kernel launch");
    } else if (P.engine == PERM_ENGINE_XSHARED) {
        pk::WalkArgs wa;
        wa.chunk_lo = P.chunk_lo;
        wa.chunk_hi = P.chunk_hi;
        wa.ntasks = P.ntasks;
        wa.task_counter = reinterpret_cast<unsigned long long *>(P.d_ws);
        wa.task_out = reinterpret_cast<unsigned long long *>(task_out);
        wa.skip_counter = reinterpret_cast<unsigned long long *>(P.d_ws + 1);
        wa.K = P.K;
        wa.zero_skip = 1;
        wa.timeout_ns = (unsigned long long)std::max(0, P.opts.timeout_ms) * 1000000ull;
        wa.deadline_word = reinterpret_cast<unsigned long long *>(P.d_ws + kWsDeadline);
        wa.abort_flag = reinterpret_cast<unsigned int *>(P.d_ws + kWsAbort);
        e = debug_fail(kSiteLaunch) ? cudaErrorLaunchFailure
                                    : xshared_launch(wa, P.d_devmat, (int)P.img_bytes, P.m.n, P.abs_shift, P.grid,
                                                     P.block, st);
        if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch");
    } else if (P.engine == PERM_ENGINE_GENERIC) {
        pk::BatchArgs ba;
        ba.mats = reinterpret_cast<const pk::BatchMat *>(P.d_ws + kWsBatchMat);
        ba.devmats = P.d_devmat;
        ba.ntasks = P.ntasks;
        ba.task_counter = reinterpret_cast<unsigned long long *>(P.d_ws);
        ba.task_out = reinterpret_cast<unsigned long long *>(task_out);
        ba.skip_counter = reinterpret_cast<unsigned long long *>(P.d_ws + 1);
        ba.slot_bytes = P.img_bytes;
        ba.nmat = 1;
        ba.zero_skip = P.opts.zero_skip ? 0 : 1;
        ba.timeout_ns = (unsigned long long)std::max(0, P.opts.timeout_ms) * 1000000ull;
        ba.deadline_word = reinterpret_cast<unsigned long long *>(P.d_ws + kWsDeadline);
        ba.abort_flag = reinterpret_cast<unsigned int *>(P.d_ws + kWsAbort);
        e = debug_fail(kSiteLaunch) ? cudaErrorLaunchFailure : P.gf.walk(ba, P.grid, P.block, st);
        if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch");
    } else {
        pk::WalkArgs wa;
        wa.chunk_lo = P.chunk_lo;
        wa.chunk_hi = P.chunk_hi;
        wa.ntasks = P.ntasks;
        wa.task_counter = reinterpret_cast<unsigned long long *>(P.d_ws);
        wa.task_out = reinterpret_cast<unsigned long long *>(task_out);
        wa.skip_counter = reinterpret_cast<unsigned long long *>(P.d_ws + 1);
        wa.K = P.K;
        wa.zero_skip = P.opts.zero_skip ? 0 : 1;
        wa.timeout_ns = (unsigned long long)std::max(0, P.opts.timeout_ms) * 1000000ull;
        wa.deadline_word = reinterpret_cast<unsigned long long *>(P.d_ws + kWsDeadline);
        wa.abort_flag = reinterpret_cast<unsigned int *>(P.d_ws + kWsAbort);
        e = debug_fail(kSiteLaunch) ? cudaErrorLaunchFailure : codegen_launch(P, wa, st);
        if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch");
    }
    if ((e = reduce_launch(P.arith, task_out, P.ntasks, P.d_ws + 2, st)) != cudaSuccess)
        return cuda_fail(e, "reduce kernel launch");
    if (record_events && (e = cudaEventRecord(P.ev1, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaMemcpyAsync(P.h_res, P.d_ws, 8 * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(result)");
    return PERM_OK;
}

// Fills the descriptive fields of a result from a prepared plan.
void describe(const perm_plan_s &P, perm_result_t *out) {
    std::memset(out, 0, sizeof(*out));
    const int n = P.m.n;
    out->vtype = P.m.is_int ? PERM_I64 : PERM_F64;
    out->engine = P.engine;
    out->ordering = P.L.ordering;
    out->reg_rows = P.engine == PERM_ENGINE_CODEGEN ? P.k : n;
    out->reg_cols = P.engine == PERM_ENGINE_CODEGEN ? P.c : n - 1;
    out->shared_rows = P.engine == PERM_ENGINE_CODEGEN ? P.k2 : 0;
    out->chunk_log2 = P.K;
    out->threads = P.grid * P.block;
    out->regs_per_thread = P.regs;
    out->steps = P.zero ? 0 : P.g_hi - P.g_lo;
    out->ms_plan = P.ms_plan;
    out->ms_compile = P.ms_compile;
    out->fp_ops_per_step = (P.engine == PERM_ENGINE_GENERIC && !P.direct && P.arith == 0 && P.m.n <= 32)
                               ? cost_per_step_dual(P.L, true)
                           : P.engine == PERM_ENGINE_XSHARED ? P.ops_per_step_paper   // a full product every step
                                                             : P.ops_per_step;
    if (P.m.is_int && !P.zero) {   // integer multiply operations of the kernel that runs
        const int fold = P.engine == PERM_ENGINE_CODEGEN ? (codegen_no_fold() ? 0 : 1) : (P.fold ? 2 : 0);
        out->fp_ops_per_step = ring_ops_per_step(P.m, P.L, P.limbs, fold);
    }
    out->exact_words = P.m.is_int ? P.arith : 0;
    out->precision = P.m.is_int ? 0 : (P.dd ? PERM_PREC_DD : PERM_PREC_F64);
}

// Turns a reduced raw sum (2 words FP64 hi/lo, or w exact words) into the
// permanent (or the sub-range partial sum).
// The skip counter's meaning per engine: the shared-memory walk counts the
// steps each thread skipped; the block walks count warp blocks (a skip is
// warp-wide, and lane 0 counts it once), out of ntasks 2^(K-B) warp blocks
// (a range's idle lanes of its last task walk in step with the warp).
double zero_skip_fraction(const perm_plan_s &P, uint64_t skipped) {
    if (P.direct) return 0.0;
    if (P.engine == PERM_ENGINE_XSHARED) return P.g_hi > P.g_lo ? (double)skipped / (double)(P.g_hi - P.g_lo) : 0.0;
    const int B = P.engine == PERM_ENGINE_GENERIC ? P.gf.block_log2 : P.cg.block_log2;
    const uint64_t warp_blocks = P.ntasks << std::max(0, P.K - B);
    return warp_blocks ? (double)skipped / (double)warp_blocks : 0.0;
}

perm_status_t finish_raw(const perm_plan_s &P, const uint64_t *r, perm_result_t *out) {
    const int n = P.m.n;
    if (P.zero) { out->status = PERM_OK; return PERM_OK; }
    if (!P.m.is_int) {
        double hi, lo, ab;
        std::memcpy(&hi, &r[0], 8);
        std::memcpy(&lo, &r[1], 8);
        std::memcpy(&ab, &r[2], 8);
        ab = std::ldexp(ab, P.abs_shift);
        if (P.subrange) { out->f64 = hi; out->f64_lo = lo; out->abs_term_sum = ab; }
        else {
            const double f = (n % 2) ? 2.0 : -2.0;    // 4 (n mod 2) - 2, Algorithm 1
            out->f64 = hi * f;
            out->f64_lo = lo * f;
            out->abs_term_sum = 2.0 * ab;
        }
        out->status = PERM_OK;
        return PERM_OK;
    }
    const int W = P.arith;
    for (int i = 0; i < W; ++i) out->partial[i] = r[i];
    if (P.subrange) { out->status = PERM_OK; return PERM_OK; }
    // S = (-1)^(n-1) 2^(n-1) perm  (mod 2^(32 limbs)): the low n-1 bits must vanish
    const int ring_bits = 32 * (P.limbs ? P.limbs : 2 * W);
    uint64_t s[3] = {0, 0, 0};
    for (int i = 0; i < W; ++i) s[i] = r[i];
    if (ring_bits < 64 * W) s[W - 1] &= (1ull << (ring_bits - 64 * (W - 1))) - 1;   // odd limb count
    const unsigned __int128 lo128 = ((unsigned __int128)s[1] << 64) | s[0];
    const uint64_t top = s[2];
    const int shift = n - 1;
    if (shift && (s[0] & ((1ull << shift) - 1))) {
        out->status = PERM_ERR_INTERNAL;
        return fail(PERM_ERR_INTERNAL, "exact sum not divisible by 2^(n-1)");
    }
    // value = S >> (n-1) as a (ring_bits - n + 1)-bit two's complement number
    const unsigned __int128 v0 = shift ? (lo128 >> shift) | ((unsigned __int128)top << (128 - shift)) : lo128;
    unsigned __int128 v = v0;
    const int bits = ring_bits - shift;
    if (bits < 128) {
        const unsigned __int128 one = 1;
        const unsigned __int128 mask = (one << bits) - 1;
        v &= mask;
        if ((v >> (bits - 1)) & 1) v |= ~mask;   // sign-extend
    }
    if ((n - 1) % 2) v = (unsigned __int128)0 - v;   // times (-1)^(n-1)
    out->i128_lo = (uint64_t)v;
    out->i128_hi = (int64_t)(uint64_t)(v >> 64);
    out->status = PERM_OK;
    return PERM_OK;
}

perm_status_t plan_finish(perm_plan_s &P, perm_result_t *out) {
    describe(P, out);
    if (P.zero) { out->status = PERM_OK; return PERM_OK; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, P.ev0, P.ev1);
    out->ms_kernel = ms;
    if (P.h_res[kWsAbort]) {
        out->status = PERM_ERR_TIMEOUT;
        return fail(PERM_ERR_TIMEOUT, "device-side deadline passed; the walk stopped early");
    }
    out->zero_skip_frac = zero_skip_fraction(P, P.h_res[1]);
    return finish_raw(P, P.h_res + 2, out);
}

static std::atomic<int> g_inject[kSiteCount];

bool debug_fail(int site) {
    if (site <= 0 || site >= kSiteCount) return false;
    int v = g_inject[site].load();
    while (v > 0)
        if (g_inject[site].compare_exchange_weak(v, v - 1)) return true;
    return false;
}

bool needs_dd(int n, double perm, double abs_term_sum) {
    if (!(std::fabs(perm) > 0.0)) return true;   // zero or not a number
    return (double)n * std::ldexp(1.0, -53) * abs_term_sum > kAutoDDError * std::fabs(perm);
}

perm_matrix_t matrix_view(const Matrix &m, std::vector<int32_t> &ptr, std::vector<int32_t> &idx,
                          std::vector<unsigned char> &vals) {
    const int n = m.n;
    const size_t vsz = m.is_int ? sizeof(int64_t) : sizeof(double);
    ptr.assign(n + 1, 0);
    idx.clear();
    vals.clear();
    for (int i = 0; i < n; ++i) {
        uint64_t cols = m.rowmask[i];
        while (cols) {
            const int j = __builtin_ctzll(cols);
            cols &= cols - 1;
            idx.push_back(j);
            const size_t o = vals.size();
            vals.resize(o + vsz);
            if (m.is_int) { const int64_t v = m.ival(i, j); std::memcpy(&vals[o], &v, vsz); }
            else { const double v = m.fval(i, j); std::memcpy(&vals[o], &v, vsz); }
        }
        ptr[i + 1] = (int32_t)idx.size();
    }
    perm_matrix_t A;
    A.n = n;
    A.nnz = (int32_t)idx.size();
    A.layout = PERM_CSR;
    A.ptr = ptr.data();
    A.idx = idx.data();
    A.vtype = m.is_int ? PERM_I64 : PERM_F64;
    A.vals = vals.data();
    return A;
}

// Precision AUTO: whether a whole FP64 walk of this plan may be rerun in
// double-double, and the double-double plan of the same matrix.
static bool auto_dd_eligible(const perm_plan_s &P) {
    return !P.m.is_int && !P.dd && !P.subrange && !P.zero && P.opts.precision == PERM_PREC_AUTO &&
           P.m.n <= kAutoDDMaxN;
}

static perm_status_t make_dd_plan(perm_plan_s &P) {
    std::vector<int32_t> ptr, idx;
    std::vector<unsigned char> vals;
    const perm_matrix_t A = matrix_view(P.m, ptr, idx, vals);
    perm_opts_t o = P.opts;
    o.precision = PERM_PREC_DD;
    o.engine = PERM_ENGINE_GENERIC;
    o.ordering = P.L.ordering == PERM_ORDER_SEARCH ? PERM_ORDER_AUTO : P.L.ordering;
    perm_plan_s *D = new (std::nothrow) perm_plan_s();
    if (!D) return fail(PERM_ERR_NOMEM, "out of host memory");
    perm_status_t st = plan_prepare(&A, &o, *D);
    if (st == PERM_OK) st = plan_device_setup(*D);
    if (st != PERM_OK) { delete D; return st; }
    P.dd_plan = D;
    return PERM_OK;
}

}  // namespace perm

perm_plan_s::~perm_plan_s() {
    if (d_devmat) cudaFree(d_devmat);
    if (d_ws) cudaFree(d_ws);
    if (d_xglob) cudaFree(d_xglob);
    if (h_res) cudaFreeHost(h_res);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (graph) cudaGraphExecDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    perm::codegen_release(*this);
    delete dd_plan;
}

using namespace perm;

extern "C" {

perm_status_t perm_plan_create(const perm_matrix_t *A, const perm_opts_t *opts, perm_plan_t *out) {
    if (!out) return fail(PERM_ERR_ARG, "out is NULL");
    *out = nullptr;
    perm_plan_s *P = new (std::nothrow) perm_plan_s();
    if (!P) return fail(PERM_ERR_NOMEM, "out of host memory");
    perm_status_t st = plan_prepare(A, opts, *P);
    if (st == PERM_OK) st = plan_device_setup(*P);
    if (st != PERM_OK) { delete P; return st; }
    *out = P;
    return PERM_OK;
}

// Captures the plan's launches into a CUDA graph (on a plan-owned stream).
static bool capture_graph(perm_plan_s &P) {
    if (!P.cap_stream && cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    const perm_status_t s = plan_launch(P, P.cap_stream, false);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(P.cap_stream, &g);
    if (s != PERM_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    const cudaError_t ie = cudaGraphInstantiate(&P.graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) { P.graph = nullptr; cudaGetLastError(); return false; }
    return true;
}

static perm_status_t compute_one(perm_plan_t plan, void *stream, perm_result_t *out);

perm_status_t perm_compute(perm_plan_t plan, void *stream, perm_result_t *out) {
    if (!plan || !out) return fail(PERM_ERR_ARG, "NULL plan or result");
    // precision AUTO: a matrix whose FP64 walk proved too ill-conditioned goes
    // straight to its double-double plan
    if (plan->dd_plan) {
        const perm_status_t s = compute_one(plan->dd_plan, stream, out);
        out->ms_plan = plan->ms_plan + plan->dd_plan->ms_plan;
        return s;
    }
    perm_status_t s = compute_one(plan, stream, out);
    if (s != PERM_OK || !auto_dd_eligible(*plan) || !needs_dd(plan->m.n, out->f64 + out->f64_lo, out->abs_term_sum))
        return s;
    const double ms_fp64 = out->ms_kernel;
    s = make_dd_plan(*plan);
    if (s != PERM_OK) { out->status = s; return s; }
    s = compute_one(plan->dd_plan, stream, out);
    out->ms_kernel += ms_fp64;
    out->ms_plan = plan->ms_plan + plan->dd_plan->ms_plan;
    return s;
}

static perm_status_t compute_one(perm_plan_t plan, void *stream, perm_result_t *out) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!plan->zero) {
        const bool use_graph = !(plan->opts.flags & PERM_FLAG_NO_GRAPH) && plan->computes >= 1;
        if (use_graph && !plan->graph && !plan->graph_failed) plan->graph_failed = !capture_graph(*plan);
        perm_status_t s = PERM_OK;
        if (use_graph && plan->graph) {
            cudaEventRecord(plan->ev0, st);
            const cudaError_t e = cudaGraphLaunch(plan->graph, st);
            if (e != cudaSuccess) s = cuda_fail(e, "cudaGraphLaunch");
            cudaEventRecord(plan->ev1, st);
        } else {
            s = plan_launch(*plan, st);
        }
        if (s != PERM_OK) { std::memset(out, 0, sizeof(*out)); out->status = s; return s; }
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { out->status = PERM_ERR_CUDA; return cuda_fail(e, "cudaStreamSynchronize"); }
        plan->computes += 1;
    }
    return plan_finish(*plan, out);
}

void perm_plan_destroy(perm_plan_t plan) { delete plan; }

perm_status_t perm_inspect(const perm_matrix_t *A, const perm_opts_t *opts_in, perm_inspect_t *out) {
    if (!out) return fail(PERM_ERR_ARG, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    perm_opts_t opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    Matrix m;
    const char *err = nullptr;
    perm_status_t st = ingest(A, m, &err);
    if (st != PERM_OK) return fail(st, err);
    if (opts.ordering < 0 || opts.ordering > PERM_ORDER_SEARCH) return fail(PERM_ERR_ARG, "bad ordering");
    if (opts.ordering == PERM_ORDER_SEARCH) opts.ordering = PERM_ORDER_AUTO;
    const Layout L = choose_layout(m, opts.ordering);
    out->n = m.n;
    out->structurally_zero = has_perfect_matching(m) ? 0 : 1;
    out->ordering = L.ordering;
    for (int i = 0; i < m.n; ++i) {
        out->col_order[i] = L.col_order[i];
        out->row_order[i] = L.row_order[i];
        out->group_of_row[i] = L.group_of_slot[i];
        out->group_size[i] = L.group_begin[i + 1] - L.group_begin[i];
        out->col_nnz[i] = L.col_nnz[i];
    }
    int k = m.n, c = m.n - 1;
    partition_alg4(L, opts.gr_ratio > 0 ? opts.gr_ratio : kDefaultGRRatio, kCodegenBaseRegs, &k, &c);
    out->reg_rows = k;
    out->reg_cols = c;
    out->bound_log2 = bound_log2(m);
    out->exact_words = m.is_int ? exact_words_for(out->bound_log2, m.n) : 0;
    out->exact_limbs = out->exact_words ? exact_limbs_for(out->bound_log2, m.n) : 0;
    out->ops_per_step_walk = walk_cost_per_step(L, !m.is_int);
    out->ring_ops_per_step = m.is_int && out->exact_limbs ? ring_ops_per_step(m, L, out->exact_limbs, 1) : 0.0;
    out->ops_per_step = cost_per_step(L, false);
    out->ops_per_step_paper = cost_per_step(L, true);
    out->ops_per_step_four_state = cost_per_step_four_state(m, L.col_order);
    out->ops_per_step_four_state_searched = four_state_searched(m, L.col_order);
    return PERM_OK;
}

perm_status_t perm_scbs(int32_t k, int32_t *out) {
    if (!out || k < 1 || k > 24) return fail(PERM_ERR_ARG, "k must be in [1, 24]");
    const uint64_t len = (1ull << k) - 1;
    for (uint64_t i = 1; i <= len; ++i) out[i - 1] = scbs_sign(i) * (scbs_col(i) + 1);
    return PERM_OK;
}

perm_status_t perm_alg2_launches(int64_t tau, int32_t n, int64_t *start, int64_t *delta, int64_t *end,
                                 int32_t max_launches, int32_t *count) {
    if (tau < 1 || n < 2 || n > 62 || !count) return fail(PERM_ERR_ARG, "bad Algorithm 2 arguments");
    std::vector<Launch> v = alg2_launches(tau, n);
    *count = (int32_t)v.size();
    for (int i = 0; i < (int)v.size() && i < max_launches; ++i) {
        if (start) start[i] = v[i].start;
        if (delta) delta[i] = v[i].delta;
        if (end) end[i] = v[i].end;
    }
    return PERM_OK;
}

perm_status_t perm_codegen_source(const perm_matrix_t *A, const perm_opts_t *opts, char *buf, int64_t cap,
                                  int64_t *len) {
    perm_plan_s P;
    perm_status_t st = plan_prepare(A, opts, P);
    if (st != PERM_OK) return st;
    codegen_layout(P);
    std::string src = codegen_source(P);
    if (len) *len = (int64_t)src.size();
    if (buf && cap > 0) {
        const size_t nb = std::min<size_t>((size_t)cap - 1, src.size());
        std::memcpy(buf, src.data(), nb);
        buf[nb] = 0;
    }
    return PERM_OK;
}

perm_status_t perm_generic_image(const perm_matrix_t *A, const perm_opts_t *opts, void *buf, int64_t cap,
                                 int64_t *len, int32_t *nmax, int32_t *kind, int32_t *abs_shift) {
    perm_plan_s P;
    perm_status_t st = plan_prepare(A, opts, P);
    if (st != PERM_OK) return st;
    if (P.m.n > 48) return fail(PERM_ERR_SIZE, "generic kernels cover n <= 48");
    const int nm = nmax_bucket(P.m.n);
    std::vector<unsigned char> img;
    build_devmat(P.m, P.L, P.img_kind(), nm, img);
    if (len) *len = (int64_t)img.size();
    if (nmax) *nmax = nm;
    if (kind) *kind = P.kind();
    if (abs_shift) *abs_shift = P.abs_shift;
    if (buf && cap > 0) std::memcpy(buf, img.data(), std::min<size_t>((size_t)cap, img.size()));
    return PERM_OK;
}

const char *perm_status_string(perm_status_t s) {
    switch (s) {
    case PERM_OK: return "ok";
    case PERM_ERR_ARG: return "invalid argument";
    case PERM_ERR_SIZE: return "invalid size";
    case PERM_ERR_PATTERN: return "invalid sparsity pattern";
    case PERM_ERR_OVERFLOW: return "exact result may overflow";
    case PERM_ERR_CUDA: return "CUDA error";
    case PERM_ERR_NVRTC: return "kernel generation/compilation failed";
    case PERM_ERR_NOMEM: return "out of memory";
    case PERM_ERR_TIMEOUT: return "timed out";
    case PERM_ERR_BUSY: return "busy";
    case PERM_ERR_NOT_READY: return "not ready";
    case PERM_ERR_CANCELLED: return "cancelled";
    case PERM_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char *perm_last_error(void) { return g_last_error; }

perm_status_t perm_debug_inject_failures(int32_t site, int32_t count) {
    if (site <= 0 || site >= kSiteCount || count < 0) return fail(PERM_ERR_ARG, "bad injection site or count");
    g_inject[site].store(count);
    return PERM_OK;
}

int32_t perm_device_available(void) {
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) { cudaGetLastError(); return 0; }
    return count > 0 ? 1 : 0;
}

const char *perm_version(void) { return "1.1.0"; }

int64_t perm_sizeof(int32_t which) {
    switch (which) {
    case 0: return (int64_t)sizeof(perm_matrix_t);
    case 1: return (int64_t)sizeof(perm_opts_t);
    case 2: return (int64_t)sizeof(perm_result_t);
    case 3: return (int64_t)sizeof(perm_inspect_t);
    case 4: return (int64_t)sizeof(perm_server_opts_t);
    case 5: return (int64_t)sizeof(perm_server_stats_t);
    default: return -1;
    }
}

}  // extern "C"
