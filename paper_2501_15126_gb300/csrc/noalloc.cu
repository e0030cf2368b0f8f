// noalloc.cu -- perm_compute_noalloc: one permanent without allocating memory.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or budget, or a process that has reserved every
// byte of HBM for itself ahead of time, or callers that are not allowed to
// call cudaMalloc/cudaFree at all.  For them this entry point runs the
// precompiled generic walk with its scratch memory (counters, per-task
// partial sums, the matrix image and the task table) in one file-scope
// device array instead of device allocations.  It allocates no device or
// pinned host memory; its host-side temporaries are on the stack or in the
// plan's host-only bookkeeping.
//
// The array is kNoAllocScratchBytes (1 MiB) on every GPU that loads this
// library and stays allocated until the process exits.  Its device address
// is looked up once per device with cudaGetSymbolAddress, on the first call
// made with that device current (so the first call on a device should not be
// made while a stream is being captured).  Every call shares the one array:
// the call clears the words that must start at zero, and two calls whose GPU
// work overlaps (on different streams or threads) race on it.
#include <algorithm>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "kernels.hpp"
#include "plan.hpp"

namespace {

constexpr size_t kNoAllocScratchBytes = 1u << 20;
constexpr int kNoAllocMaxN = 48;                  // the generic kernels' largest bucket
constexpr size_t kOffCounters = 0;                // [0] task counter, [1] skipped blocks, [2] deadline, [3] abort
constexpr size_t kOffResult = 128;                // up to 3 words
constexpr size_t kOffBatchMat = 192;              // one pk::BatchMat
constexpr size_t kOffImage = 256;                 // the matrix image (<= 20480 bytes)
constexpr size_t kImageBytes = 20480;
constexpr size_t kOffTasks = kOffImage + kImageBytes;   // per-task partial sums
constexpr int kMaxDevices = 64;
static_assert(sizeof(pk::BatchMat) <= kOffImage - kOffBatchMat, "task table entry");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// The device address of g_noalloc_scratch on the current device.
perm_status_t scratch_for_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return perm::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return perm::fail(PERM_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return perm::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return PERM_OK;
}

// The smallest chunk length (log2) whose 32-chunk tasks fit the scratch
// array's task area, or -1 when the range's alignment does not allow one:
// chunks must tile [g_lo, g_hi) exactly, so K is at most the number of
// trailing zero bits of both ends.
int chunk_log2_that_fits(const perm_plan_s &P, uint64_t max_tasks, int K_from) {
    int kmax = P.m.n - 1;
    if (P.g_lo) kmax = std::min(kmax, __builtin_ctzll(P.g_lo));
    if (P.g_hi != P.total || P.subrange) kmax = std::min(kmax, P.g_hi ? __builtin_ctzll(P.g_hi) : 63);
    const uint64_t len = P.g_hi - P.g_lo;
    if (len) kmax = std::min(kmax, 63 - __builtin_clzll(len));
    for (int K = K_from; K <= kmax; ++K) {
        const uint64_t chunks = (P.g_hi >> K) - (P.g_lo >> K);
        if ((chunks + 31) / 32 <= max_tasks) return K;
    }
    return -1;
}

// One walk of a prepared plan (FP64, double-double or exact) in the scratch
// array; fills *out.  Every error return sets out->status too.
perm_status_t walk_in_scratch(perm_plan_s &P, unsigned char *scratch, cudaStream_t st_, perm_result_t *out) {
    using namespace perm;
    auto failed = [&](perm_status_t s) { out->status = s; return s; };
    const int n = P.m.n;
    P.engine = PERM_ENGINE_GENERIC;
    P.words = result_words(P.arith);
    const int nmax = nmax_bucket(n);
    P.nmax = nmax;
    P.gf = generic_fns(nmax, P.kind());
    if (!P.gf.walk) return failed(fail(PERM_ERR_INTERNAL, "no generic kernel"));
    const size_t img_bytes = devmat_bytes_for(P.L, P.img_kind(), nmax);
    if (img_bytes > kImageBytes) return failed(fail(PERM_ERR_INTERNAL, "image too large for the scratch array"));
    const uint64_t max_tasks = (kNoAllocScratchBytes - kOffTasks) / (8ull * P.words);
    cudaError_t e;
    cudaFuncAttributes attr;
    if ((e = P.gf.attr(&attr)) != cudaSuccess) return failed(cuda_fail(e, "cudaFuncGetAttributes"));
    P.regs = attr.numRegs;
    unsigned char *d_tasks = scratch + kOffTasks;
    uint64_t *d_counters = reinterpret_cast<uint64_t *>(scratch + kOffCounters);
    uint64_t *d_result = reinterpret_cast<uint64_t *>(scratch + kOffResult);

    if (n <= 8) {
        // one thread per Gray index; block partial sums go to the task area
        P.direct = true;
        P.block = 256;
        P.grid = (int)((P.g_hi - P.g_lo + 255) / 256);
        P.ntasks = (uint64_t)P.grid;
    } else {
        int bps = 0;
        if ((e = P.gf.occ(256, img_bytes, &bps)) != cudaSuccess) return failed(cuda_fail(e, "occupancy"));
        perm_status_t s = choose_launch(P, P.gf.block_log2, bps > 0 ? bps : 1, 256);
        if (s != PERM_OK) return failed(s);
        if (P.ntasks > max_tasks) {
            // the longest chunks the alignment allows, and no longer than needed
            const int K = chunk_log2_that_fits(P, max_tasks, P.K + 1);
            if (K < 0) return failed(fail(PERM_ERR_SIZE, "range too long (or its ends too finely aligned) for the scratch array"));
            P.opts.chunk_log2 = K;
            s = choose_launch(P, P.gf.block_log2, bps > 0 ? bps : 1, 256);
            if (s != PERM_OK) return failed(s);
        }
    }
    if (P.ntasks > max_tasks) return failed(fail(PERM_ERR_SIZE, "too many tasks for the scratch array"));

    alignas(16) unsigned char image[kImageBytes];
    build_devmat_into(P.m, P.L, P.img_kind(), nmax, image);
    if ((e = cudaMemcpyAsync(scratch + kOffImage, image, img_bytes, cudaMemcpyHostToDevice, st_)) != cudaSuccess)
        return failed(cuda_fail(e, "cudaMemcpyAsync(image)"));
    if ((e = cudaMemsetAsync(scratch + kOffCounters, 0, kOffResult + 32, st_)) != cudaSuccess)
        return failed(cuda_fail(e, "cudaMemsetAsync(counters)"));
    if (P.direct) {
        e = P.gf.direct(scratch + kOffImage, P.g_lo, P.g_hi, reinterpret_cast<uint64_t *>(d_tasks), P.grid, P.block,
                        st_, P.abs_shift);
        if (e != cudaSuccess) return failed(cuda_fail(e, "direct kernel launch"));
    } else {
        pk::BatchMat bm;
        std::memset(&bm, 0, sizeof(bm));
        bm.chunk_lo = P.chunk_lo;
        bm.chunk_hi = P.chunk_hi;
        bm.K = P.K;
        bm.abs_shift = P.abs_shift;
        // a stack source: the copy is staged before cudaMemcpyAsync returns
        if ((e = cudaMemcpyAsync(scratch + kOffBatchMat, &bm, sizeof(bm), cudaMemcpyHostToDevice, st_)) != cudaSuccess)
            return failed(cuda_fail(e, "cudaMemcpyAsync(task table)"));
        pk::BatchArgs ba;
        ba.mats = reinterpret_cast<const pk::BatchMat *>(scratch + kOffBatchMat);
        ba.devmats = scratch + kOffImage;
        ba.ntasks = P.ntasks;
        ba.task_counter = reinterpret_cast<unsigned long long *>(d_counters);
        ba.task_out = reinterpret_cast<unsigned long long *>(d_tasks);
        ba.skip_counter = reinterpret_cast<unsigned long long *>(d_counters + 1);
        ba.slot_bytes = img_bytes;
        ba.nmat = 1;
        ba.zero_skip = P.opts.zero_skip ? 0 : 1;
        ba.timeout_ns = (unsigned long long)std::max(0, P.opts.timeout_ms) * 1000000ull;
        ba.deadline_word = reinterpret_cast<unsigned long long *>(d_counters + 2);
        ba.abort_flag = reinterpret_cast<unsigned int *>(d_counters + 3);
        if ((e = P.gf.walk(ba, P.grid, P.block, st_)) != cudaSuccess) return failed(cuda_fail(e, "walk kernel launch"));
    }
    if ((e = reduce_launch(P.arith, reinterpret_cast<const uint64_t *>(d_tasks), P.ntasks, d_result, st_)) !=
        cudaSuccess)
        return failed(cuda_fail(e, "reduce kernel launch"));
    uint64_t host[4];
    if ((e = cudaMemcpyAsync(host, d_counters, sizeof(host), cudaMemcpyDeviceToHost, st_)) != cudaSuccess)
        return failed(cuda_fail(e, "cudaMemcpyAsync(counters)"));
    uint64_t raw[3];
    if ((e = cudaMemcpyAsync(raw, d_result, sizeof(raw), cudaMemcpyDeviceToHost, st_)) != cudaSuccess)
        return failed(cuda_fail(e, "cudaMemcpyAsync(result)"));
    if ((e = cudaStreamSynchronize(st_)) != cudaSuccess) return failed(cuda_fail(e, "cudaStreamSynchronize"));
    describe(P, out);
    if (host[3]) return failed(fail(PERM_ERR_TIMEOUT, "device-side deadline passed; the walk stopped early"));
    out->zero_skip_frac = zero_skip_fraction(P, host[1]);
    return finish_raw(P, raw, out);
}

}  // namespace

using namespace perm;

extern "C" perm_status_t perm_compute_noalloc(const perm_matrix_t *A, const perm_opts_t *opts, void *stream,
                                              perm_result_t *out) {
    if (!A || !out) return fail(PERM_ERR_ARG, "NULL matrix or result");
    std::memset(out, 0, sizeof(*out));
    auto failed = [&](perm_status_t s) { out->status = s; return s; };
    if (A->n > kNoAllocMaxN)
        return failed(fail(PERM_ERR_SIZE, "perm_compute_noalloc: n must be <= 48 (its scratch holds one 48x48 image)"));
    if (opts && opts->engine == PERM_ENGINE_CODEGEN)
        return failed(fail(PERM_ERR_ARG, "perm_compute_noalloc runs the precompiled kernels only"));
    unsigned char *scratch = nullptr;
    perm_status_t st = scratch_for_current_device(&scratch);
    if (st != PERM_OK) return failed(st);

    alignas(16) unsigned char dense[kNoAllocMaxN * kNoAllocMaxN * 8];
    perm_plan_s P;   // host bookkeeping only: nothing on the device is allocated through it
    st = plan_prepare(A, opts, P, dense, sizeof(dense));
    if (st != PERM_OK) return failed(st);
    if (P.zero) { describe(P, out); out->status = PERM_OK; return PERM_OK; }
    cudaStream_t st_ = reinterpret_cast<cudaStream_t>(stream);
    st = walk_in_scratch(P, scratch, st_, out);
    // precision AUTO: an ill-conditioned whole FP64 walk runs again in
    // double-double, in the same scratch array
    if (st == PERM_OK && !P.m.is_int && !P.dd && !P.subrange && P.opts.precision == PERM_PREC_AUTO &&
        P.m.n <= kAutoDDMaxN && needs_dd(P.m.n, out->f64 + out->f64_lo, out->abs_term_sum)) {
        P.dd = true;
        P.direct = false;
        P.opts.chunk_log2 = opts ? opts->chunk_log2 : 0;
        st = walk_in_scratch(P, scratch, st_, out);
    }
    return st;
}
