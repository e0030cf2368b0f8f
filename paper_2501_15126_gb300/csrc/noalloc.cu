// noalloc.cu -- perm_compute_noalloc: one permanent without allocating.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or budget, or a process that has reserved every
// byte of HBM for itself ahead of time, or callers that are not allowed to
// call cudaMalloc/cudaFree at all.  For them this entry point runs the
// precompiled generic walk with its scratch memory (task counter, per-task
// partial sums, the matrix image and the task table) in one file-scope
// device array instead of device allocations, and it keeps every host-side
// temporary on the stack.
//
// The array is kNoAllocScratchBytes (1 MiB) on every GPU that loads this
// library and stays allocated until the process exits.  Its device address
// is looked up once per device with cudaGetSymbolAddress, on the first call
// made with that device current (so the first call on a device should not be
// made while a stream is being captured).  Every call shares the one array:
// the call clears the words that must start at zero, and two calls whose GPU
// work overlaps (on different streams or threads) race on it.
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "kernels.hpp"
#include "plan.hpp"

namespace {

constexpr size_t kNoAllocScratchBytes = 1u << 20;
constexpr int kNoAllocMaxN = 48;                  // the generic kernels' largest bucket
constexpr size_t kOffCounters = 0;                // [0] task counter, [1] skipped blocks
constexpr size_t kOffResult = 64;                 // up to 3 words
constexpr size_t kOffBatchMat = 128;              // one pk::BatchMat
constexpr size_t kOffImage = 256;                 // the matrix image (<= 19600 bytes)
constexpr size_t kOffTasks = 256 + 20480;         // per-task partial sums
constexpr int kMaxDevices = 64;

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

}  // namespace

using namespace perm;

extern "C" perm_status_t perm_compute_noalloc(const perm_matrix_t *A, const perm_opts_t *opts, void *stream,
                                              perm_result_t *out) {
    if (!A || !out) return fail(PERM_ERR_ARG, "NULL matrix or result");
    std::memset(out, 0, sizeof(*out));
    if (A->n > kNoAllocMaxN) {
        out->status = PERM_ERR_SIZE;
        return fail(PERM_ERR_SIZE, "perm_compute_noalloc: n must be <= 48 (its scratch holds one 48x48 image)");
    }
    if (opts && opts->engine == PERM_ENGINE_CODEGEN) {
        out->status = PERM_ERR_ARG;
        return fail(PERM_ERR_ARG, "perm_compute_noalloc runs the precompiled kernels only");
    }
    unsigned char *scratch = nullptr;
    perm_status_t st = scratch_for_current_device(&scratch);
    if (st != PERM_OK) { out->status = st; return st; }

    alignas(16) unsigned char dense[kNoAllocMaxN * kNoAllocMaxN * 8];
    perm_plan_s P;   // host bookkeeping only: nothing on the device is allocated through it
    st = plan_prepare(A, opts, P, dense, sizeof(dense));
    if (st != PERM_OK) { out->status = st; return st; }
    const int n = P.m.n;
    P.engine = PERM_ENGINE_GENERIC;
    P.words = P.arith == 0 ? 2 : P.arith;
    if (P.zero) { describe(P, out); out->status = PERM_OK; return PERM_OK; }
    const int nmax = nmax_bucket(n);
    P.nmax = nmax;
    P.gf = generic_fns(nmax, P.kind());
    if (!P.gf.walk) { out->status = PERM_ERR_INTERNAL; return fail(PERM_ERR_INTERNAL, "no generic kernel"); }
    const size_t img_bytes = devmat_bytes_for(P.L, P.arith, nmax);
    if (img_bytes > kOffTasks - kOffImage) { out->status = PERM_ERR_INTERNAL; return fail(PERM_ERR_INTERNAL, "image too large"); }
    const uint64_t max_tasks = (kNoAllocScratchBytes - kOffTasks) / (8ull * P.words);
    cudaStream_t st_ = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    cudaFuncAttributes attr;
    if ((e = P.gf.attr(&attr)) != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
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
        if ((e = P.gf.occ(256, img_bytes, &bps)) != cudaSuccess) return cuda_fail(e, "occupancy");
        st = choose_launch(P, P.gf.block_log2, bps > 0 ? bps : 1, 256);
        // raise the chunk length until the task results fit the scratch array
        while (st == PERM_OK && P.ntasks > max_tasks) {
            if (P.K >= n - 1) { st = fail(PERM_ERR_SIZE, "range too long for the scratch array"); break; }
            P.opts.chunk_log2 = P.K + 1;
            st = choose_launch(P, P.gf.block_log2, bps > 0 ? bps : 1, 256);
        }
        if (st != PERM_OK) { out->status = st; return st; }
    }
    if (P.ntasks > max_tasks) { out->status = PERM_ERR_SIZE; return fail(PERM_ERR_SIZE, "too many tasks for the scratch array"); }

    alignas(16) unsigned char image[20480];
    build_devmat_into(P.m, P.L, P.arith, nmax, image);
    if ((e = cudaMemcpyAsync(scratch + kOffImage, image, img_bytes, cudaMemcpyHostToDevice, st_)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(image)");
    if ((e = cudaMemsetAsync(scratch + kOffCounters, 0, 128, st_)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync(counters)");
    if (P.direct) {
        e = P.gf.direct(scratch + kOffImage, P.g_lo, P.g_hi, reinterpret_cast<uint64_t *>(d_tasks), P.grid, P.block,
                        st_);
        if (e != cudaSuccess) return cuda_fail(e, "direct kernel launch");
    } else {
        pk::BatchMat bm;
        std::memset(&bm, 0, sizeof(bm));
        bm.chunk_lo = P.chunk_lo;
        bm.chunk_hi = P.chunk_hi;
        bm.K = P.K;
        if ((e = cudaMemcpyAsync(scratch + kOffBatchMat, &bm, sizeof(bm), cudaMemcpyHostToDevice, st_)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(task table)");
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
        ba.timeout_ns = 0;
        ba.deadline_word = nullptr;
        ba.abort_flag = nullptr;
        if ((e = P.gf.walk(ba, P.grid, P.block, st_)) != cudaSuccess) return cuda_fail(e, "walk kernel launch");
    }
    if ((e = reduce_launch(P.arith, reinterpret_cast<const uint64_t *>(d_tasks), P.ntasks, d_result, st_)) !=
        cudaSuccess)
        return cuda_fail(e, "reduce kernel launch");
    uint64_t host[8];
    if ((e = cudaMemcpyAsync(host, d_counters, 64, cudaMemcpyDeviceToHost, st_)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(counters)");
    uint64_t raw[3];
    if ((e = cudaMemcpyAsync(raw, d_result, 24, cudaMemcpyDeviceToHost, st_)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(result)");
    if ((e = cudaStreamSynchronize(st_)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    describe(P, out);
    const uint64_t blocks = (P.g_hi - P.g_lo) >> P.gf.block_log2;
    out->zero_skip_frac = (!P.direct && blocks) ? (double)host[1] / (double)blocks : 0.0;
    return finish_raw(P, raw, out);
}
