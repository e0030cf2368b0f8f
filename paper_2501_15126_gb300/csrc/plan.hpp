// plan.hpp -- the internal state behind a perm_plan_t.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "codegen.hpp"
#include "host.hpp"
#include "kernels.hpp"

namespace perm {

// Layouts of the matrix image (devmat.h): FP64 values and start values,
// doubled int32 values and start values, or FP64 values with exact
// double-double start values.
constexpr int kImgF64 = 0, kImgInt = 1, kImgDD = 2;

// 64-bit words of one task result: the FP64 accumulator (hi, lo, sum|terms|)
// or the exact ring's words.
inline int result_words(int arith) { return arith == 0 ? 3 : arith; }

// Precision AUTO reruns an FP64 walk in double-double arithmetic when its
// rounding-error estimate n 2^-53 sum|terms| / |perm| exceeds the 1e-9
// relative target, for walks of at most 2^31 steps.  The measured error of
// FP64 walks is at most 0.076 of the estimate (0.0067 among the most
// ill-conditioned matrices of the batch and serving workloads), so a walk
// that is not rerun is within about 1e-10.
constexpr double kAutoDDError = 1e-9;
constexpr int kAutoDDMaxN = 32;
bool needs_dd(int n, double perm, double abs_term_sum);

// Host-side failure injection for tests (perm_debug_inject_failures): each
// call consumes one pending injected failure of `site`, if any, and the
// caller then behaves as if the call made there had failed.
enum { kSiteWaveLaunch = 1, kSiteNvrtc = 2, kSiteFinish = 3, kSiteUpload = 4, kSiteLaunch = 5, kSiteCount = 6 };
bool debug_fail(int site);

}  // namespace perm

struct perm_plan_s {
    perm::Matrix m;
    perm::Layout L;
    perm_opts_t opts{};
    int arith = 0;            // 0 = FP64, 1..3 = exact, results stored as `arith` 64-bit words
    int limbs = 0;            // 0 = FP64, else the walk's ring Z/2^(32 limbs): 2 arith - 1 or 2 arith
    bool fold = false;        // exact: every row's absolute sum <= 127 (folded products)
    bool dual = false;        // generated FP64 kernel with two-state chains (cheaper than pairing)
    bool dd = false;          // FP64 input walked in double-double arithmetic
    bool pure_reg = false;    // codegen: a full product of all n rows every step (CodeGen-PureReg)
    bool zero_heavy = false;  // codegen: most sampled terms have a zero factor (FP64: shorter blocks)
    double zero_frac = 0.0;   // codegen: fraction of sampled terms with a zero factor
    bool zero_spans = false;  // codegen: the kernel widens zero skips into zero spans (core.cuh)
    bool want_abs = true;     // FP64 walks: accumulate sum|terms| (generated kernels: see codegen_layout)
    int abs_shift = 0;        // FP64 / double-double: sum|terms| is accumulated as sum|terms| 2^-abs_shift
    int kind() const { return dd ? perm::kKindDD : 2 * limbs + (fold ? 1 : 0); }   // generic kernel family
    int img_kind() const { return dd ? perm::kImgDD : (arith ? perm::kImgInt : perm::kImgF64); }   // matrix image layout
    uint64_t total = 0;       // 2^(n-1)
    uint64_t g_lo = 0, g_hi = 0;
    bool subrange = false;
    bool zero = false;        // no perfect matching: perm is 0, nothing launches
    bool direct = false;      // tiny n: one thread per Gray index
    double bound = 0.0;
    double ops_per_step = 0.0, ops_per_step_paper = 0.0;
    double ms_plan = 0.0, ms_compile = 0.0;
    int engine = 0, nmax = 0, words = 2;
    size_t img_bytes = 0;     // generic kernels: size of the matrix image
    int K = 0, grid = 1, block = 256, regs = 0;
    int k = 0, c = 0;         // Algorithm 4 split (codegen)
    int k2 = 0;               // codegen: rows [k, k + k2) of x in shared memory, the rest global
    uint64_t chunk_lo = 0, chunk_hi = 0, ntasks = 0;
    perm::GenericFns gf;
    perm::CodegenKernel cg;
    void *d_devmat = nullptr;
    uint64_t *d_ws = nullptr;   // [0] task counter, [1] skipped blocks, [2..4] result, [8..] task results
    void *d_xglob = nullptr;    // codegen: rows of x kept in global memory
    size_t xs_bytes() const { return (size_t)k2 * 256 * (arith == 0 ? 8 : 4); }   // per block
    uint64_t *h_res = nullptr;  // pinned copy of d_ws[0..7]
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int computes = 0;                      // perm_compute calls so far
    cudaStream_t cap_stream = nullptr;     // stream the graph is captured on
    cudaGraphExec_t graph = nullptr;       // the captured launches (second call on)
    bool graph_failed = false;
    // precision AUTO: the double-double plan of this matrix, made when a
    // compute's FP64 result proved too ill-conditioned; later computes use it
    // directly
    perm_plan_s *dd_plan = nullptr;
    uint64_t len() const { return g_hi - g_lo; }
    ~perm_plan_s();
};

namespace perm {

// Workspace layout (64-bit words): [0] task counter, [1] skipped blocks,
// [2..4] reduced result, [5] deadline, [6] abort flag, [8..13] the
// single-matrix BatchMat, [16..] task results.  Words 0..7 are cleared
// before every launch.
constexpr size_t kWsDeadline = 5;
constexpr size_t kWsAbort = 6;
constexpr size_t kWsBatchMat = 8;
constexpr size_t kWsTaskOut = 16;

perm_status_t fail(perm_status_t s, const char *msg);
perm_status_t fail(perm_status_t s, const std::string &msg);
perm_status_t cuda_fail(cudaError_t e, const char *what);
double now_ms();

// Stages of perm_plan_create / perm_compute, reused by batch and serving.
// storage: optional caller memory (>= n*n*8 bytes) for the dense copy.
perm_status_t plan_prepare(const perm_matrix_t *A, const perm_opts_t *opts, perm_plan_s &P,
                           void *storage = nullptr, size_t storage_bytes = 0);
perm_status_t plan_device_setup(perm_plan_s &P);
perm_status_t plan_launch(perm_plan_s &P, cudaStream_t st, bool record_events = true);
perm_status_t plan_finish(perm_plan_s &P, perm_result_t *out);
void describe(const perm_plan_s &P, perm_result_t *out);
perm_status_t finish_raw(const perm_plan_s &P, const uint64_t *raw, perm_result_t *out);
// perm_result_t.zero_skip_frac from the walk's skip counter
double zero_skip_fraction(const perm_plan_s &P, uint64_t skipped);
int nmax_bucket(int n);
// Matrix images; img is kImgF64, kImgInt or kImgDD.
void build_devmat(const Matrix &m, const Layout &L, int img, int nmax, std::vector<unsigned char> &img_out);
size_t devmat_bytes(int img, int nmax, int nnz);
size_t devmat_bytes_for(const Layout &L, int img, int nmax);
void build_devmat_into(const Matrix &m, const Layout &L, int img, int nmax, unsigned char *dst);
// A CSR view of a prepared matrix (for re-planning it), backed by the vectors.
perm_matrix_t matrix_view(const Matrix &m, std::vector<int32_t> &ptr, std::vector<int32_t> &idx,
                          std::vector<unsigned char> &vals);
perm_status_t choose_launch(perm_plan_s &P, int block_log2, int blocks_per_sm, int block);

}  // namespace perm
