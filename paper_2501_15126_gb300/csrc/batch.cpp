// batch.cpp -- many permanents in one persistent launch per kernel family.
//
// perm_batch: every matrix is prepared on the host (ingest, structural guard,
// ordering, exact width); matrices are grouped by (NMAX bucket, arithmetic);
// each group becomes one launch of the generic multi-matrix walk, fed by one
// device task table (32-chunk tasks of every matrix of the group), followed by
// one segmented reduction (one warp per matrix).  The chunk length of each
// group comes from the autotuner (tune.cpp) unless the caller fixes it.
// Tiny (n <= 8) and large (n > 48) matrices take their own plans.
//
// perm_batch_sequential: the plain form -- plan, launch, synchronise and
// destroy one matrix at a time -- used as the comparison baseline.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "batch.hpp"
#include "plan.hpp"

namespace perm {

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

int batch_chunk_log2(int n, int B, int K_target) {
    // 32 chunks fill a warp task; keep at least one full task when n allows
    int K = std::min(K_target, n - 1 - 5);
    K = std::max(K, B);
    return std::min(K, n - 1);
}

int BatchGroup::setup(int nmax_, int kind_, int K_target) {
    nmax = nmax_;
    kind = kind_;
    arith = ((kind >> 1) + 1) / 2;
    img = kind == kKindDD ? kImgDD : (arith ? kImgInt : kImgF64);
    gf = generic_fns(nmax, kind);
    if (!gf.walk) return fail(PERM_ERR_INTERNAL, "no generic kernel for this group");
    words = result_words(arith);
    // task table
    mats.resize(plans.size());
    ntasks = 0;
    for (size_t i = 0; i < plans.size(); ++i) {
        perm_plan_s &P = *plans[i];
        const int K = batch_chunk_log2(P.m.n, gf.block_log2, K_target);
        P.K = K;
        P.chunk_lo = 0;
        P.chunk_hi = P.total >> K;
        P.ntasks = (P.chunk_hi + 31) / 32;
        P.engine = PERM_ENGINE_GENERIC;
        P.gf = gf;
        P.nmax = nmax;
        std::memset(&mats[i], 0, sizeof(mats[i]));
        mats[i].task_begin = ntasks;
        mats[i].chunk_lo = 0;
        mats[i].chunk_hi = P.chunk_hi;
        mats[i].out_offset = ntasks;
        mats[i].K = K;
        mats[i].abs_shift = P.abs_shift;
        ntasks += P.ntasks;
    }
    // images packed back to back (each a multiple of 16 bytes)
    size_t total = 0;
    slot_bytes = 16;
    for (size_t i = 0; i < plans.size(); ++i) {
        const size_t b = devmat_bytes_for(plans[i]->L, img, nmax);
        mats[i].image = (int)(total / 16);
        total += b;
        slot_bytes = std::max(slot_bytes, b);
    }
    images.assign(total, 0);
    for (size_t i = 0; i < plans.size(); ++i)
        build_devmat_into(plans[i]->m, plans[i]->L, img, nmax, images.data() + (size_t)mats[i].image * 16);
    cudaFuncAttributes attr;
    if (gf.attr(&attr) == cudaSuccess) regs = attr.numRegs;
    int bps = 0;
    cudaError_t e = gf.occ(256, slot_bytes, &bps);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    block = 256;
    int64_t g = (int64_t)kSMCount * std::max(bps, 1);
    g = std::min<int64_t>(g, ((int64_t)ntasks * 32 + block - 1) / block);
    grid = (int)std::max<int64_t>(1, g);
    return PERM_OK;
}

size_t BatchGroup::arena_bytes() const {
    return align256(images.size()) + align256(mats.size() * sizeof(pk::BatchMat)) +
           align256((size_t)ntasks * words * 8) + align256(mats.size() * (size_t)words * 8) + 256;
}

void BatchGroup::bind(unsigned char *base) {
    size_t off = 0;
    d_images = base + off; off += align256(images.size());
    d_mats = reinterpret_cast<pk::BatchMat *>(base + off); off += align256(mats.size() * sizeof(pk::BatchMat));
    d_task_out = reinterpret_cast<uint64_t *>(base + off); off += align256((size_t)ntasks * words * 8);
    d_result = reinterpret_cast<uint64_t *>(base + off); off += align256(mats.size() * (size_t)words * 8);
    d_counters = reinterpret_cast<uint64_t *>(base + off);
}

int BatchGroup::upload(cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_images, images.data(), images.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(images)");
    if ((e = cudaMemcpyAsync(d_mats, mats.data(), mats.size() * sizeof(pk::BatchMat), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(task table)");
    return PERM_OK;
}

int BatchGroup::launch(cudaStream_t st, int zero_skip) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_counters, 0, 32, st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    pk::BatchArgs ba;
    ba.mats = d_mats;
    ba.devmats = d_images;
    ba.ntasks = ntasks;
    ba.task_counter = reinterpret_cast<unsigned long long *>(d_counters);
    ba.task_out = reinterpret_cast<unsigned long long *>(d_task_out);
    ba.skip_counter = reinterpret_cast<unsigned long long *>(d_counters + 1);
    ba.slot_bytes = slot_bytes;
    ba.nmat = (int)mats.size();
    ba.zero_skip = zero_skip;
    ba.timeout_ns = timeout_ns;
    ba.deadline_word = reinterpret_cast<unsigned long long *>(d_counters + 2);
    ba.abort_flag = reinterpret_cast<unsigned int *>(d_counters + 3);
    if ((e = gf.walk(ba, grid, block, st)) != cudaSuccess) return cuda_fail(e, "batch walk launch");
    if ((e = batch_reduce_launch(arith, d_mats, (int)mats.size(), ntasks, d_task_out, d_result, st)) != cudaSuccess)
        return cuda_fail(e, "batch reduce launch");
    return PERM_OK;
}

}  // namespace perm

using namespace perm;

namespace perm {

// The batch's device work captured as one CUDA graph on a library stream:
// `st` is joined to it with events before and after, so the caller's stream
// (the legacy default stream included, which cannot be captured) sees the
// usual ordering.
struct GraphLaunch {
    cudaStream_t cs = nullptr;
    cudaEvent_t before = nullptr, after = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool capture(std::map<std::pair<int, int>, BatchGroup> &groups, int zero_skip, cudaStream_t) {
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return fail_clean();
        if (cudaEventCreateWithFlags(&before, cudaEventDisableTiming) != cudaSuccess) return fail_clean();
        if (cudaEventCreateWithFlags(&after, cudaEventDisableTiming) != cudaSuccess) return fail_clean();
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail_clean();
        bool ok = true;
        for (auto &kv : groups) ok = ok && kv.second.launch(cs, zero_skip) == PERM_OK;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (!ok || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return fail_clean();
        }
        const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) { exec = nullptr; return fail_clean(); }
        return true;
    }
    cudaError_t launch(cudaStream_t st) {
        cudaError_t e = cudaEventRecord(before, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, before, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, cs);
        if (e == cudaSuccess) e = cudaEventRecord(after, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, after, 0);
        return e;
    }
    bool fail_clean() {
        cudaGetLastError();   // a failed capture leaves no sticky error behind
        return false;
    }
    ~GraphLaunch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
        if (before) cudaEventDestroy(before);
        if (after) cudaEventDestroy(after);
    }
};

// Launches every group (one persistent walk and one segmented reduction
// each, all in one device arena), reads the results back and finishes
// out[i] for every matrix of the groups.
static perm_status_t run_groups(std::map<std::pair<int, int>, BatchGroup> &groups, const perm_opts_t &opts,
                                cudaStream_t st, double ms_plan_each,
                                std::vector<std::unique_ptr<perm_plan_s>> &plans, perm_result_t *out) {
    if (groups.empty()) return PERM_OK;
    size_t total = 0;
    for (auto &kv : groups) {
        BatchGroup &G = kv.second;
        G.timeout_ns = (unsigned long long)std::max(0, opts.timeout_ms) * 1000000ull;
        int K_target = opts.chunk_log2;
        if (!K_target) {
            if (!chunk_log2_is_tuned(kv.first.first, kv.first.second)) {
                G.nmax = kv.first.first;
                G.kind = kv.first.second;
                G.arith = ((G.kind >> 1) + 1) / 2;
                G.img = G.kind == kKindDD ? kImgDD : (G.arith ? kImgInt : kImgF64);
                autotune_group(G, st);
            }
            K_target = tuned_chunk_log2(kv.first.first, kv.first.second);
        }
        perm_status_t s = (perm_status_t)G.setup(kv.first.first, kv.first.second, K_target);
        if (s != PERM_OK) return s;
        total += G.arena_bytes();
    }
    DeviceArena arena;
    cudaError_t e = arena.alloc(total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch arena)");
    size_t off = 0;
    for (auto &kv : groups) {
        kv.second.bind(arena.base + off);
        off += kv.second.arena_bytes();
    }
    EventPair ev;
    if ((e = ev.create()) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventRecord(ev.e0, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (auto &kv : groups) {
        perm_status_t s = (perm_status_t)kv.second.upload(st);
        if (s != PERM_OK) return s;
    }
    // every family's launches (counter reset, walk, reduction) as one CUDA
    // graph; launched directly if the capture is not possible
    GraphLaunch gl;
    const bool graphed = !(opts.flags & PERM_FLAG_NO_GRAPH) && gl.capture(groups, opts.zero_skip ? 0 : 1, st);
    if (!graphed) {
        for (auto &kv : groups) {
            const perm_status_t s = (perm_status_t)kv.second.launch(st, opts.zero_skip ? 0 : 1);
            if (s != PERM_OK) return s;
        }
    } else if ((e = gl.launch(st)) != cudaSuccess) {
        return cuda_fail(e, "batch graph launch");
    }
    if ((e = cudaEventRecord(ev.e1, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    // results back in one copy per group, then the group's counters
    std::vector<std::vector<uint64_t>> raw;
    raw.reserve(groups.size());
    for (auto &kv : groups) {
        BatchGroup &G = kv.second;
        raw.emplace_back(G.mats.size() * (size_t)G.words + 4);
        if ((e = cudaMemcpyAsync(raw.back().data(), G.d_result, G.mats.size() * (size_t)G.words * 8,
                                 cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(batch results)");
        if ((e = cudaMemcpyAsync(raw.back().data() + G.mats.size() * (size_t)G.words, G.d_counters, 32,
                                 cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(batch counters)");
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize(batch)");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.e0, ev.e1);
    size_t gi = 0;
    bool timed_out = false;
    for (auto &kv : groups) {
        BatchGroup &G = kv.second;
        const bool aborted = raw[gi][G.mats.size() * (size_t)G.words + 3] != 0;
        timed_out |= aborted;
        for (size_t j = 0; j < G.idx.size(); ++j) {
            const int i = G.idx[j];
            perm_plan_s &P = *plans[i];
            P.grid = G.grid;
            P.block = G.block;
            P.regs = G.regs;
            describe(P, &out[i]);
            out[i].ms_kernel = ms;
            out[i].ms_plan = ms_plan_each;
            if (aborted) out[i].status = PERM_ERR_TIMEOUT;
            else finish_raw(P, raw[gi].data() + j * (size_t)G.words, &out[i]);
        }
        ++gi;
    }
    if (timed_out) fail(PERM_ERR_TIMEOUT, "device-side deadline passed in a batch walk");
    return PERM_OK;
}

}  // namespace perm

extern "C" perm_status_t perm_batch_sequential(const perm_matrix_t *mats, int32_t count, const perm_opts_t *opts,
                                               void *stream, perm_result_t *out) {
    if (count < 0) return fail(PERM_ERR_SIZE, "count < 0");
    if (count > 0 && (!mats || !out)) return fail(PERM_ERR_ARG, "NULL matrices or results");
    for (int32_t i = 0; i < count; ++i) {
        perm_plan_t p = nullptr;
        perm_status_t st = perm_plan_create(&mats[i], opts, &p);
        if (st != PERM_OK) {
            std::memset(&out[i], 0, sizeof(out[i]));
            out[i].status = st;
            if (st == PERM_ERR_CUDA) return st;
            continue;
        }
        st = perm_compute(p, stream, &out[i]);
        perm_plan_destroy(p);
        if (st == PERM_ERR_CUDA) return st;
    }
    return PERM_OK;
}

extern "C" perm_status_t perm_batch(const perm_matrix_t *mats, int32_t count, const perm_opts_t *opts_in,
                                    void *stream, perm_result_t *out) {
    if (count < 0) return fail(PERM_ERR_SIZE, "count < 0");
    if (count == 0) return PERM_OK;
    if (!mats || !out) return fail(PERM_ERR_ARG, "NULL matrices or results");
    perm_opts_t opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    if (opts.g_lo || opts.g_hi) return fail(PERM_ERR_ARG, "sub-ranges are not available in a batch");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double t0 = now_ms();

    // host preprocessing (validation, matching check, ordering, exact width)
    // of every matrix, spread over host threads: plans are independent
    std::vector<std::unique_ptr<perm_plan_s>> plans(count);
    std::vector<perm_status_t> prep(count, PERM_OK);
    {
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nthreads = count >= 256 ? (int)std::min(hw, 16u) : 1;
        auto work = [&](int t) {
            for (int32_t i = t; i < count; i += nthreads) {
                plans[i].reset(new perm_plan_s());
                prep[i] = plan_prepare(&mats[i], &opts, *plans[i]);
            }
        };
        std::vector<std::thread> pool;
        for (int t = 1; t < nthreads; ++t) pool.emplace_back(work, t);
        work(0);
        for (std::thread &th : pool) th.join();
    }
    std::map<std::pair<int, int>, BatchGroup> groups;
    std::vector<int> singles;
    for (int32_t i = 0; i < count; ++i) {
        perm_plan_s &P = *plans[i];
        const perm_status_t s = prep[i];
        std::memset(&out[i], 0, sizeof(out[i]));
        if (s != PERM_OK) {
            out[i].status = s;
            plans[i].reset();
            fail(s, ("batch item " + std::to_string(i) + ": " + perm_status_string(s)).c_str());
            continue;
        }
        if (P.zero) { describe(P, &out[i]); out[i].status = PERM_OK; plans[i].reset(); continue; }
        if (P.m.n <= 8 || P.m.n > 48) { singles.push_back(i); continue; }
        groups[{nmax_bucket(P.m.n), P.kind()}].add(i, &P);
    }
    const double t_prep = now_ms() - t0;
    if (opts.timeout_ms < 0) return fail(PERM_ERR_ARG, "timeout_ms < 0");

    perm_status_t s = run_groups(groups, opts, st, t_prep / count, plans, out);
    if (s != PERM_OK) return s;

    // precision AUTO: FP64 matrices whose results proved too ill-conditioned
    // run again, in double-double, as one more launch per NMAX bucket
    std::map<std::pair<int, int>, BatchGroup> redo;
    for (auto &kv : groups)
        for (size_t j = 0; j < kv.second.idx.size(); ++j) {
            const int i = kv.second.idx[j];
            perm_plan_s &P = *plans[i];
            if (!P.m.is_int && !P.dd && opts.precision == PERM_PREC_AUTO && P.m.n <= kAutoDDMaxN &&
                out[i].status == PERM_OK && needs_dd(P.m.n, out[i].f64 + out[i].f64_lo, out[i].abs_term_sum)) {
                P.dd = true;
                redo[{nmax_bucket(P.m.n), P.kind()}].add(i, &P);
            }
        }
    if (!redo.empty()) {
        std::vector<double> ms_first(count, 0.0);
        for (auto &kv : redo)
            for (int i : kv.second.idx) ms_first[i] = out[i].ms_kernel;
        s = run_groups(redo, opts, st, t_prep / count, plans, out);
        if (s != PERM_OK) return s;
        for (auto &kv : redo)
            for (int i : kv.second.idx) out[i].ms_kernel += ms_first[i];
    }

    // tiny and very large matrices: their own plans (perm_compute applies AUTO)
    for (int i : singles) {
        perm_plan_s &P = *plans[i];
        s = plan_device_setup(P);
        if (s == PERM_OK) {
            perm_plan_s *raw = plans[i].release();
            s = perm_compute(raw, stream, &out[i]);
            perm_plan_destroy(raw);
        }
        if (s != PERM_OK) { out[i].status = s; if (s == PERM_ERR_CUDA) return s; }
    }
    return PERM_OK;
}
