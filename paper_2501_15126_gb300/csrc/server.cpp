// server.cpp -- continuous-batching serving loop (perm_submit / perm_poll).
//
// A request is prepared on the caller's thread (ingest, structural guard,
// ordering, exact width) and queued.  One scheduler thread owns the GPU side:
//
//   admission  a queued request becomes active when its kernel family (NMAX
//              bucket x arithmetic) has a free image slot, its task results fit
//              the family's result pool, and the Gray steps of all active
//              requests stay under the step budget (the compute budget);
//              otherwise it waits in the queue (perm_submit answers BUSY only
//              when the queue itself is full);
//   waves      active requests' tasks (32 aligned 2^K-chunks each) are packed
//              into launches of the generic multi-matrix walk: every active
//              request first gets a small share, the rest of the wave goes to
//              the oldest requests, so large requests progress in slices
//              while small ones that arrive meanwhile are not held back;
//              waves alternate between two streams, so a new wave overlaps
//              the tail of the previous one on the device; image uploads and
//              final reductions go on a third stream, so neither waits behind
//              a wave;
//   results    each task writes its sum to a fixed place in the request's own
//              result range, whatever wave ran it; when all of a request's
//              waves are done one fixed-order reduction produces its value.
//              A request's chunking depends only on its n and its family, so
//              its result is bit-identical alone and in any mix.
//
// No kernel here waits on anything: completion is observed on the host with
// CUDA events, and a request older than timeout_ms is failed with TIMEOUT
// (its result is discarded when its waves finish).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "batch.hpp"
#include "plan.hpp"

namespace perm {

namespace {

constexpr int kStreams = 2;                   // wave streams; one more (aux) takes uploads and reductions
constexpr uint64_t kSmallShare = 64;          // tasks every active request gets per wave
constexpr double kWaveSteps = 268435456.0;    // Gray steps per wave (2^28, a few ms): short waves let
                                              // requests that arrive meanwhile start soon
constexpr int kServeChunkLog2 = 12;           // chunk length target: tasks of 2^17 steps fill short waves
constexpr int kAdmitScan = 256;               // queued requests looked at past a blocked one
constexpr double kNoSkipAfterMs = 200.0;      // a request blocked this long stops being overtaken
constexpr size_t kQueueMax = 1 << 20;

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Makes `dev` current for a scope and restores the caller's device after it:
// perm_server_create and perm_submit run on the caller's thread, whose
// current device is the caller's business.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct Request {
    uint64_t ticket = 0;
    std::unique_ptr<perm_plan_s> P;
    int family = -1;            // -1: own plan (n <= 8 or n > 48)
    int slot = -1;
    uint64_t ntasks = 0, next_task = 0, done_tasks = 0;
    uint64_t out_offset = 0;    // first task of the request's result range in the family pool
    size_t img_bytes = 0;       // size of the request's matrix image
    double t_submit = 0.0;
    int inflight_waves = 0;
    bool failed = false;
    bool retired = false;
    perm_status_t fail_status = PERM_OK;
};

// First-fit allocator of task ranges in a family's result pool.
struct RangeAlloc {
    std::map<uint64_t, uint64_t> free_;   // start -> length
    void init(uint64_t n) { free_.clear(); if (n) free_[0] = n; }
    bool alloc(uint64_t n, uint64_t *out) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *out = it->first;
                const uint64_t s = it->first + n, l = it->second - n;
                free_.erase(it);
                if (l) free_[s] = l;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t s, uint64_t n) {
        auto it = free_.emplace(s, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }
};

struct Family {
    int nmax = 0, kind = 0, arith = 0, words = 3, K_target = 14;   // kind: generic kernel family
    int img = 0;                                                  // image layout (kImgF64, kImgInt, kImgDD)
    GenericFns gf;
    int grid_max = 1;
    unsigned char *d_images = nullptr;
    uint64_t *d_pool = nullptr;
    uint64_t pool_tasks = 0;
    std::vector<int> free_slots;
    RangeAlloc ranges;
    bool ready = false;
};

// A request's slice of a wave: tasks [first, first + count) of the request.
struct Part {
    Request *req;
    uint64_t first, count;
};

struct Wave {
    int stream = 0;
    cudaEvent_t done = nullptr;
    std::vector<Part> parts;                             // at most one slice per request
    pk::BatchMat *h_table = nullptr;                     // pinned
    pk::BatchMat *d_table = nullptr;
    uint64_t *d_counters = nullptr;
    bool busy = false;
};

struct Finish {
    cudaEvent_t done = nullptr;
    std::vector<Request *> reqs;
    uint64_t *h_seg = nullptr, *d_seg = nullptr;   // pinned / device
    uint64_t *h_res = nullptr, *d_res = nullptr;
    int family = 0;
    bool busy = false;
};

}  // namespace

}  // namespace perm

using namespace perm;

struct perm_server_s {
    perm_server_opts_t opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread thread;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<Request *> queue;                          // prepared, not yet admitted
    std::vector<Request *> active;                        // admitted, not finished
    std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
    std::unordered_map<uint64_t, perm_result_t> results;  // finished, not yet polled
    std::vector<Family> fam;
    cudaStream_t streams[kStreams] = {};
    cudaStream_t aux = nullptr;   // image uploads and final reductions, never queued behind a wave
    static constexpr int kWaves = 4, kFinishes = 4;
    Wave waves[kWaves];
    Finish finishes[kFinishes];
    double step_budget = 0.0, steps_active = 0.0;
    // statistics
    std::vector<double> lat_ms;
    uint64_t completed = 0, rejected = 0, failed = 0;
    double t_first = 0.0, t_last = 0.0;
    perm_status_t init_status = PERM_OK;

    static int family_index(int nmax, int kind) { return (nmax / 16 - 1) * 14 + kind; }

    perm_status_t init_device() {   // on the creating thread, with `device` current
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate");
        for (int i = 0; i < kStreams; ++i)
            if ((e = cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreate");
        const int maxn = opts.max_inflight;
        for (Wave &w : waves) {
            if ((e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "event");
            if ((e = cudaMallocHost(&w.h_table, sizeof(pk::BatchMat) * 2 * maxn)) != cudaSuccess) return cuda_fail(e, "pinned");
            if ((e = cudaMalloc(&w.d_table, sizeof(pk::BatchMat) * 2 * maxn)) != cudaSuccess) return cuda_fail(e, "table");
            if ((e = cudaMalloc(&w.d_counters, 256)) != cudaSuccess) return cuda_fail(e, "counters");
        }
        for (Finish &f : finishes) {
            if ((e = cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "event");
            if ((e = cudaMallocHost(&f.h_seg, 16 * (size_t)maxn)) != cudaSuccess) return cuda_fail(e, "pinned");
            if ((e = cudaMalloc(&f.d_seg, 16 * (size_t)maxn)) != cudaSuccess) return cuda_fail(e, "seg");
            if ((e = cudaMallocHost(&f.h_res, 32 * (size_t)maxn)) != cudaSuccess) return cuda_fail(e, "pinned");
            if ((e = cudaMalloc(&f.d_res, 32 * (size_t)maxn)) != cudaSuccess) return cuda_fail(e, "res");
        }
        fam.resize(42);
        return PERM_OK;
    }

    perm_status_t ensure_family(int fi, int nmax, int kind) {
        Family &F = fam[fi];
        if (F.ready) return PERM_OK;
        DeviceScope scope(device);
        F.nmax = nmax;
        F.kind = kind;
        F.arith = ((kind >> 1) + 1) / 2;
        F.words = result_words(F.arith);
        F.img = kind == kKindDD ? kImgDD : (F.arith ? kImgInt : kImgF64);
        F.gf = generic_fns(nmax, kind);
        if (!F.gf.walk) return fail(PERM_ERR_INTERNAL, "no generic kernel for this family");
        F.K_target = tuned_chunk_log2(nmax, kind);
        int bps = 0;
        cudaError_t e = F.gf.occ(256, F.gf.devmat_bytes, &bps);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy");
        F.grid_max = kSMCount * std::max(bps, 1);
        const int slots = opts.max_inflight;
        if ((e = cudaMalloc(&F.d_images, (size_t)slots * F.gf.devmat_bytes)) != cudaSuccess) return cuda_fail(e, "images");
        // result pool: every slot's largest request at once would be too much; size it for the step budget
        F.pool_tasks = std::max<uint64_t>(1ull << 21, (uint64_t)(step_budget / std::ldexp(1.0, F.K_target + 5)) * 2 + 4096);
        F.pool_tasks = std::min<uint64_t>(F.pool_tasks, 1ull << 23);
        if ((e = cudaMalloc(&F.d_pool, F.pool_tasks * F.words * 8)) != cudaSuccess) return cuda_fail(e, "result pool");
        F.ranges.init(F.pool_tasks);
        F.free_slots.clear();
        for (int s = slots - 1; s >= 0; --s) F.free_slots.push_back(s);
        F.ready = true;
        return PERM_OK;
    }

    void release_family_resources() {
        for (Family &F : fam) {
            if (F.d_images) cudaFree(F.d_images);
            if (F.d_pool) cudaFree(F.d_pool);
            F.d_images = nullptr;
            F.d_pool = nullptr;
        }
        for (Wave &w : waves) {
            if (w.done) cudaEventDestroy(w.done);
            if (w.h_table) cudaFreeHost(w.h_table);
            if (w.d_table) cudaFree(w.d_table);
            if (w.d_counters) cudaFree(w.d_counters);
        }
        for (Finish &f : finishes) {
            if (f.done) cudaEventDestroy(f.done);
            if (f.h_seg) cudaFreeHost(f.h_seg);
            if (f.d_seg) cudaFree(f.d_seg);
            if (f.h_res) cudaFreeHost(f.h_res);
            if (f.d_res) cudaFree(f.d_res);
        }
        for (int i = 0; i < kStreams; ++i)
            if (streams[i]) cudaStreamDestroy(streams[i]);
        if (aux) cudaStreamDestroy(aux);
    }

    // ---- called with mu held
    void publish(Request *r, const perm_result_t &res) {
        results[r->ticket] = res;
        const double t = now_ms();
        if (res.status == PERM_OK) {
            ++completed;
            lat_ms.push_back(t - r->t_submit);
        } else {
            ++failed;
        }
        t_last = t;
        cv_done.notify_all();
    }

    // Admits queued requests while budget, slots and pool space allow.
    // Tries to admit one queued request; false when it does not fit now.
    bool try_admit(Request *r) {
        perm_plan_s &P = *r->P;
        const double steps = (double)P.total;
        if (!active.empty() && steps_active + steps > step_budget) return false;
        if (r->family >= 0) {
            Family &F = fam[r->family];
            if (F.free_slots.empty()) return false;
            // at most 2^20 tasks per request, so the largest n fits the result pool
            const int K = batch_chunk_log2(P.m.n, F.gf.block_log2, std::max(kServeChunkLog2, P.m.n - 26));
            const uint64_t chunks = P.total >> K;
            const uint64_t ntasks = (chunks + 31) / 32;
            uint64_t off = 0;
            if (!F.ranges.alloc(ntasks, &off)) return false;
            r->slot = F.free_slots.back();
            F.free_slots.pop_back();
            P.K = K;
            P.chunk_lo = 0;
            P.chunk_hi = chunks;
            P.ntasks = ntasks;
            P.engine = PERM_ENGINE_GENERIC;
            P.gf = F.gf;
            P.nmax = F.nmax;
            r->ntasks = ntasks;
            r->out_offset = off;
            // the image goes up on the aux stream; every wave waits for the uploads made so far
            std::vector<unsigned char> img;
            build_devmat(P.m, P.L, F.img, F.nmax, img);
            r->img_bytes = img.size();
            const cudaError_t e = debug_fail(kSiteUpload) ? cudaErrorInvalidValue
                                  : cudaMemcpyAsync(F.d_images + (size_t)r->slot * F.gf.devmat_bytes, img.data(),
                                                    img.size(), cudaMemcpyHostToDevice, aux);
            if (e != cudaSuccess) fail_request(r, cuda_fail(e, "serving: image upload"));
        }
        steps_active += steps;
        active.push_back(r);
        return true;
    }

    // Admits queued requests in arrival order while budget, slots and pool
    // space allow.  A request that does not fit may be overtaken by later,
    // smaller ones (up to kAdmitScan of them), until it has waited
    // kNoSkipAfterMs; then everything behind it waits too.
    void admit() {
        const double t = now_ms();
        int scanned = 0;
        for (auto it = queue.begin(); it != queue.end() && scanned < kAdmitScan;) {
            Request *r = *it;
            if (try_admit(r)) {
                it = queue.erase(it);
                continue;
            }
            if (t - r->t_submit > kNoSkipAfterMs) break;
            ++it;
            ++scanned;
        }
    }

    void run_own_plan(Request *r, std::unique_lock<std::mutex> &lk) {
        perm_plan_s &P = *r->P;
        lk.unlock();
        perm_result_t res;
        std::memset(&res, 0, sizeof(res));
        perm_status_t s = plan_device_setup(P);
        if (s == PERM_OK) s = perm_compute(&P, streams[0], &res);   // applies precision AUTO too
        if (s != PERM_OK) res.status = s;
        lk.lock();
        steps_active -= (double)P.total;
        r->retired = true;
        active.erase(std::find(active.begin(), active.end(), r));
        publish(r, res);
    }

    // Packs one wave of tasks for family fi; returns false when there is nothing to run.
    bool launch_wave(int fi) {
        Family &F = fam[fi];
        Wave *w = nullptr;
        for (Wave &c : waves)
            if (!c.busy) { w = &c; break; }
        if (!w) return false;
        std::vector<Part> parts;
        std::unordered_map<Request *, size_t> where;
        double budget = kWaveSteps;
        const int maxent = opts.max_inflight * 2;
        // pass 1: a small share for everyone; pass 2: the rest to the oldest.
        // A request's two shares are contiguous, so they merge into one slice.
        for (int pass = 0; pass < 2 && budget > 0; ++pass) {
            for (Request *r : active) {
                if (r->family != fi || r->failed) continue;
                const uint64_t left = r->ntasks - r->next_task;
                if (!left) continue;
                const double task_steps = std::ldexp(32.0, r->P->K);
                uint64_t take = pass == 0 ? std::min(left, kSmallShare) : left;
                take = std::min<uint64_t>(take, std::max<uint64_t>(1, (uint64_t)(budget / task_steps)));
                auto it = where.find(r);
                if (it != where.end()) {
                    parts[it->second].count += take;
                } else {
                    if ((int)parts.size() >= maxent) break;
                    where[r] = parts.size();
                    parts.push_back(Part{r, r->next_task, take});
                }
                r->next_task += take;
                budget -= (double)take * task_steps;
                if (budget <= 0) break;
            }
        }
        if (parts.empty()) return false;
        uint64_t t = 0;
        for (size_t i = 0; i < parts.size(); ++i) {
            Request *r = parts[i].req;
            const uint64_t take = parts[i].count;
            const uint64_t first = parts[i].first;
            pk::BatchMat &bm = w->h_table[i];
            std::memset(&bm, 0, sizeof(bm));
            bm.task_begin = t;
            bm.chunk_lo = first * 32;
            bm.chunk_hi = std::min<uint64_t>((first + take) * 32, r->P->chunk_hi);
            bm.out_offset = r->out_offset + first;
            bm.image = (int)((size_t)r->slot * F.gf.devmat_bytes / 16);
            bm.K = r->P->K;
            bm.abs_shift = r->P->abs_shift;
            r->inflight_waves += 1;
            t += take;
        }
        w->parts = std::move(parts);
        w->stream = (int)(w - waves) % kStreams;
        cudaStream_t st = streams[w->stream];
        cudaError_t e = cudaStreamWaitEvent(st, upload_done, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(w->d_table, w->h_table, sizeof(pk::BatchMat) * w->parts.size(), cudaMemcpyHostToDevice,
                                st);
        if (e == cudaSuccess) e = cudaMemsetAsync(w->d_counters, 0, 16, st);
        pk::BatchArgs ba;
        ba.mats = w->d_table;
        ba.devmats = F.d_images;
        ba.ntasks = t;
        ba.task_counter = reinterpret_cast<unsigned long long *>(w->d_counters);
        ba.task_out = reinterpret_cast<unsigned long long *>(F.d_pool);
        ba.skip_counter = nullptr;
        size_t slot_bytes = 16;
        for (const Part &pt : w->parts) slot_bytes = std::max(slot_bytes, pt.req->img_bytes);
        ba.slot_bytes = slot_bytes;
        ba.nmat = (int)w->parts.size();
        ba.zero_skip = 1;
        ba.timeout_ns = 0;
        ba.deadline_word = nullptr;
        ba.abort_flag = nullptr;
        int bps = 1;
        if (e == cudaSuccess) e = F.gf.occ(256, slot_bytes, &bps);
        const uint64_t grid_occ = (uint64_t)kSMCount * std::max(bps, 1);
        const int grid = (int)std::min<uint64_t>(grid_occ, (t * 32 + 255) / 256);
        if (e == cudaSuccess) e = debug_fail(kSiteWaveLaunch) ? cudaErrorLaunchFailure : F.gf.walk(ba, std::max(grid, 1), 256, st);
        if (e == cudaSuccess) e = cudaEventRecord(w->done, st);
        if (e != cudaSuccess) {
            // nothing of this wave counts: its requests fail instead of
            // publishing whatever their result ranges hold
            const perm_status_t fs = cuda_fail(e, "serving: wave launch");
            for (Part &pt : w->parts) {
                pt.req->inflight_waves -= 1;
                fail_request(pt.req, fs);
            }
            w->parts.clear();
            return true;
        }
        w->busy = true;
        return true;
    }

    cudaEvent_t upload_done = nullptr;

    // Reduces every request of family fi whose tasks are all done.
    void launch_finish(int fi, std::vector<Request *> &ready) {
        Family &F = fam[fi];
        while (!ready.empty()) {
            Finish *f = nullptr;
            for (Finish &c : finishes)
                if (!c.busy) { f = &c; break; }
            if (!f) return;
            const size_t cnt = std::min<size_t>(ready.size(), (size_t)opts.max_inflight);
            f->reqs.assign(ready.begin(), ready.begin() + cnt);
            ready.erase(ready.begin(), ready.begin() + cnt);
            for (size_t i = 0; i < cnt; ++i) {
                f->h_seg[2 * i] = f->reqs[i]->out_offset;
                f->h_seg[2 * i + 1] = f->reqs[i]->ntasks;
            }
            f->family = fi;
            cudaStream_t st = aux;   // its requests' waves are done (their events were seen)
            cudaError_t e = cudaMemcpyAsync(f->d_seg, f->h_seg, 16 * cnt, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = debug_fail(kSiteFinish) ? cudaErrorLaunchFailure
                                            : segment_reduce_launch(F.arith, f->d_seg, (int)cnt, F.d_pool, f->d_res, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(f->h_res, f->d_res, 32 * cnt, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaEventRecord(f->done, st);
            if (e != cudaSuccess) {
                const perm_status_t fs = cuda_fail(e, "serving: final reduction");
                for (Request *r : f->reqs) {
                    perm_result_t res;
                    std::memset(&res, 0, sizeof(res));
                    res.status = fs;
                    retire(r);
                    publish(r, res);
                }
                f->reqs.clear();
                continue;
            }
            f->busy = true;
        }
    }

    bool in_finish(Request *r) const {
        for (const Finish &f : finishes)
            if (f.busy && std::find(f.reqs.begin(), f.reqs.end(), r) != f.reqs.end()) return true;
        return false;
    }

    // Marks a request failed: nothing more of it is scheduled, and it is
    // published with `st` once none of its waves or reductions is in flight.
    void fail_request(Request *r, perm_status_t st) {
        if (!r->failed) r->fail_status = st;
        r->failed = true;
        r->next_task = r->ntasks;
    }

    // Precision AUTO: an FP64 request whose result proved too ill-conditioned
    // gives back its slot and result range and goes to the front of the queue
    // as a double-double request.  False if that family cannot be set up.
    bool requeue_dd(Request *r) {
        perm_plan_s &P = *r->P;
        if (P.m.is_int || P.dd || opts.precision != PERM_PREC_AUTO || P.m.n > kAutoDDMaxN || r->family < 0) return false;
        Family &F = fam[r->family];
        F.free_slots.push_back(r->slot);
        F.ranges.release(r->out_offset, r->ntasks);
        steps_active -= (double)P.total;
        auto it = std::find(active.begin(), active.end(), r);
        if (it != active.end()) active.erase(it);
        const int nmax = nmax_bucket(P.m.n);
        P.dd = true;
        r->family = family_index(nmax, P.kind());
        r->slot = -1;
        r->ntasks = r->next_task = r->done_tasks = 0;
        r->inflight_waves = 0;
        if (ensure_family(r->family, nmax, P.kind()) != PERM_OK) {
            r->retired = true;   // holds nothing any more
            return false;
        }
        queue.push_front(r);
        return true;
    }

    void retire(Request *r) {
        if (r->retired) return;
        r->retired = true;
        if (r->family >= 0) {
            Family &F = fam[r->family];
            F.free_slots.push_back(r->slot);
            F.ranges.release(r->out_offset, r->ntasks);
        }
        steps_active -= (double)r->P->total;
        auto it = std::find(active.begin(), active.end(), r);
        if (it != active.end()) active.erase(it);
    }

    void loop() {
        cudaSetDevice(device);
        cudaEventCreateWithFlags(&upload_done, cudaEventDisableTiming);
        std::unique_lock<std::mutex> lk(mu);
        std::vector<std::vector<Request *>> ready(fam.size());
        while (true) {
            if (stop) break;
            admit();
            cudaEventRecord(upload_done, aux);   // waves wait for the uploads only
            // requests that run their own plan
            for (size_t i = 0; i < active.size(); ++i) {
                Request *r = active[i];
                if (r->family < 0) { run_own_plan(r, lk); --i; if (stop) break; }
            }
            // timeouts
            if (opts.timeout_ms > 0) {
                const double t = now_ms();
                for (Request *r : active)
                    if (!r->failed && t - r->t_submit > opts.timeout_ms) fail_request(r, PERM_ERR_TIMEOUT);
                // a timed-out request waiting in the queue fails there
                for (auto it = queue.begin(); it != queue.end();) {
                    if (t - (*it)->t_submit > opts.timeout_ms) {
                        perm_result_t res;
                        std::memset(&res, 0, sizeof(res));
                        res.status = PERM_ERR_TIMEOUT;
                        publish(*it, res);
                        it = queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            }
            // failed requests (timeout, a failed upload or launch) are published
            // once none of their waves or reductions is in flight
            for (size_t i = 0; i < active.size(); ++i) {
                Request *r = active[i];
                if (r->failed && r->inflight_waves == 0 && r->family >= 0 &&
                    std::find(ready[r->family].begin(), ready[r->family].end(), r) == ready[r->family].end() &&
                    !in_finish(r)) {
                    perm_result_t res;
                    std::memset(&res, 0, sizeof(res));
                    res.status = r->fail_status;
                    retire(r);
                    publish(r, res);
                    --i;
                }
            }
            bool launched = false;
            for (size_t fi = 0; fi < fam.size(); ++fi)
                if (fam[fi].ready) while (launch_wave((int)fi)) launched = true;
            // harvest finished waves (a wave whose event reports an error fails
            // its requests)
            bool progressed = false;
            for (Wave &w : waves) {
                if (!w.busy) continue;
                const cudaError_t q = cudaEventQuery(w.done);
                if (q == cudaErrorNotReady) continue;
                const perm_status_t fs = q == cudaSuccess ? PERM_OK : cuda_fail(q, "serving: wave");
                for (Part &pr : w.parts) {
                    pr.req->done_tasks += pr.count;
                    pr.req->inflight_waves -= 1;
                    if (fs != PERM_OK) fail_request(pr.req, fs);
                }
                for (Part &pr : w.parts) {
                    Request *r = pr.req;
                    if (r->retired) continue;
                    if (r->inflight_waves == 0 && (r->done_tasks == r->ntasks || r->failed) &&
                        std::find(ready[r->family].begin(), ready[r->family].end(), r) == ready[r->family].end()) {
                        if (r->failed) {
                            perm_result_t res;
                            std::memset(&res, 0, sizeof(res));
                            res.status = r->fail_status;
                            retire(r);
                            publish(r, res);
                        } else {
                            ready[r->family].push_back(r);
                        }
                    }
                }
                w.parts.clear();
                w.busy = false;
                progressed = true;
            }
            for (size_t fi = 0; fi < fam.size(); ++fi)
                if (!ready[fi].empty()) launch_finish((int)fi, ready[fi]);
            // harvest finished reductions
            for (Finish &f : finishes) {
                if (!f.busy) continue;
                const cudaError_t q = cudaEventQuery(f.done);
                if (q == cudaErrorNotReady) continue;
                const perm_status_t fs = q == cudaSuccess ? PERM_OK : cuda_fail(q, "serving: final reduction");
                for (size_t i = 0; i < f.reqs.size(); ++i) {
                    Request *r = f.reqs[i];
                    perm_result_t res;
                    r->P->grid = fam[f.family].grid_max;
                    r->P->block = 256;
                    describe(*r->P, &res);
                    if (fs != PERM_OK) res.status = fs;
                    else finish_raw(*r->P, f.h_res + 4 * i, &res);
                    if (fs == PERM_OK && res.status == PERM_OK && !r->P->m.is_int && !r->P->dd &&
                        needs_dd(r->P->m.n, res.f64 + res.f64_lo, res.abs_term_sum) && requeue_dd(r))
                        continue;
                    retire(r);
                    publish(r, res);
                }
                f.reqs.clear();
                f.busy = false;
                progressed = true;
            }
            const bool gpu_busy = std::any_of(std::begin(waves), std::end(waves), [](const Wave &w) { return w.busy; }) ||
                                  std::any_of(std::begin(finishes), std::end(finishes), [](const Finish &f) { return f.busy; });
            if (!gpu_busy && queue.empty() && !launched && !progressed) {
                cv_work.wait_for(lk, std::chrono::milliseconds(50));
            } else if (!progressed) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            }
        }
        // shutdown: drain the device, cancel what is left
        lk.unlock();
        for (int i = 0; i < kStreams; ++i) cudaStreamSynchronize(streams[i]);
        cudaStreamSynchronize(aux);
        lk.lock();
        perm_result_t res;
        std::memset(&res, 0, sizeof(res));
        res.status = PERM_ERR_CANCELLED;
        for (Request *r : active) results[r->ticket] = res;
        for (Request *r : queue) results[r->ticket] = res;
        active.clear();
        queue.clear();
        cudaEventDestroy(upload_done);
        cv_done.notify_all();
    }
};

extern "C" {

perm_status_t perm_server_create(const perm_server_opts_t *opts, perm_server_t *out) {
    if (!out) return fail(PERM_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::unique_ptr<perm_server_s> s(new (std::nothrow) perm_server_s());
    if (!s) return fail(PERM_ERR_NOMEM, "out of host memory");
    if (opts) s->opts = *opts;
    if (s->opts.max_inflight <= 0) s->opts.max_inflight = 4096;
    if (s->opts.max_n <= 0) s->opts.max_n = 40;
    if (s->opts.max_n > 64) return fail(PERM_ERR_ARG, "max_n must be <= 64");
    if (s->opts.timeout_ms < 0) return fail(PERM_ERR_ARG, "timeout_ms < 0");
    if (s->opts.precision < PERM_PREC_AUTO || s->opts.precision > PERM_PREC_DD) return fail(PERM_ERR_ARG, "bad precision");
    s->device = s->opts.device;
    s->step_budget = s->opts.step_budget > 0 ? s->opts.step_budget : 1.5e11;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || s->device < 0 || s->device >= ndev) {
        cudaGetLastError();
        return fail(ndev > 0 ? PERM_ERR_ARG : PERM_ERR_CUDA, "no such CUDA device");
    }
    DeviceScope scope(s->device);
    perm_status_t st = s->init_device();
    if (st != PERM_OK) { s->release_family_resources(); return st; }
    s->thread = std::thread([p = s.get()] { p->loop(); });
    *out = s.release();
    return PERM_OK;
}

perm_status_t perm_submit(perm_server_t s, const perm_matrix_t *A, uint64_t *ticket) {
    if (!s || !A || !ticket) return fail(PERM_ERR_ARG, "NULL argument");
    if (A->n > s->opts.max_n) return fail(PERM_ERR_SIZE, "n above the server's max_n");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return fail(PERM_ERR_NOMEM, "out of host memory");
    r->P.reset(new (std::nothrow) perm_plan_s());
    if (!r->P) return fail(PERM_ERR_NOMEM, "out of host memory");
    perm_opts_t po;
    std::memset(&po, 0, sizeof(po));
    po.precision = s->opts.precision;
    perm_status_t st = plan_prepare(A, &po, *r->P);
    if (st != PERM_OK) return st;
    perm_plan_s &P = *r->P;
    r->t_submit = now_ms();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(PERM_ERR_CANCELLED, "server is shutting down");
    if (s->queue.size() >= kQueueMax) { ++s->rejected; return fail(PERM_ERR_BUSY, "admission queue full"); }
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    if (!s->t_first) s->t_first = r->t_submit;
    Request *raw = r.get();
    s->all[r->ticket] = std::move(r);
    if (P.zero) {
        perm_result_t res;
        describe(P, &res);
        res.status = PERM_OK;
        s->publish(raw, res);
        return PERM_OK;
    }
    if (P.m.n > 8 && P.m.n <= 48) {
        const int nmax = nmax_bucket(P.m.n);
        raw->family = perm_server_s::family_index(nmax, P.kind());
        st = s->ensure_family(raw->family, nmax, P.kind());
        if (st != PERM_OK) { s->all.erase(raw->ticket); return st; }
    }
    s->queue.push_back(raw);
    s->cv_work.notify_one();
    return PERM_OK;
}

perm_status_t perm_poll(perm_server_t s, uint64_t ticket, int32_t timeout_ms, perm_result_t *out) {
    if (!s || !out) return fail(PERM_ERR_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->all.count(ticket)) return fail(PERM_ERR_ARG, "unknown ticket");
    auto ready = [&] { return s->results.count(ticket) > 0; };
    if (!ready()) {
        if (timeout_ms == 0) return PERM_ERR_NOT_READY;
        if (timeout_ms < 0) s->cv_done.wait(lk, ready);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return PERM_ERR_NOT_READY;
    }
    *out = s->results[ticket];
    s->results.erase(ticket);
    s->all.erase(ticket);
    return PERM_OK;
}

perm_status_t perm_server_stats(perm_server_t s, perm_server_stats_t *out) {
    if (!s || !out) return fail(PERM_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->failed = s->failed;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto q = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = v.back();
    }
    if (s->t_last > s->t_first) out->perms_per_s = 1e3 * (double)s->completed / (s->t_last - s->t_first);
    return PERM_OK;
}

void perm_server_destroy(perm_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->thread.joinable()) s->thread.join();
    {
        DeviceScope scope(s->device);
        s->release_family_resources();
    }
    delete s;
}

}  // extern "C"
