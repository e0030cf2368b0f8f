// tune.cpp -- autotuned chunk length for the multi-matrix (batch) walk.
//
// The chunk length 2^K trades the start-vector cost (one per 2^K Gray steps)
// against load balance and the number of 32-chunk tasks that feed the
// persistent grid.  The first large batch of each (NMAX, arithmetic) family
// runs its own group on a sample of its matrices at each candidate K, timed
// with CUDA events, and keeps the fastest; later batches reuse the choice.
// Results do not depend on the choice (exact sums are exact; FP64 sums only
// change in rounding order), so tuning never changes what is computed.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "batch.hpp"
#include "plan.hpp"

namespace perm {

namespace {
std::mutex g_mu;
std::map<std::pair<int, int>, int> g_choice;
constexpr int kDefaultK = 12;
constexpr int kCandidates[] = {8, 10, 12, 14};
constexpr size_t kSampleMats = 256;
constexpr size_t kMinMatsToTune = 64;
}  // namespace

int tuned_chunk_log2(int nmax, int kind) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_choice.find({nmax, kind});
    return it != g_choice.end() ? it->second : kDefaultK;
}

bool chunk_log2_is_tuned(int nmax, int kind) {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_choice.count({nmax, kind}) > 0;
}

void set_tuned_chunk_log2(int nmax, int kind, int K) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_choice[{nmax, kind}] = K;
}

// Times `group` restricted to an evenly spaced sample of its matrices at each
// candidate K on `st`, and records the fastest.  Returns the chosen K.
int autotune_group(const BatchGroup &group, cudaStream_t st) {
    if (group.plans.size() < kMinMatsToTune) return tuned_chunk_log2(group.nmax, group.kind);
    BatchGroup sample;
    const size_t step = std::max<size_t>(1, group.plans.size() / kSampleMats);
    for (size_t i = 0; i < group.plans.size() && sample.plans.size() < kSampleMats; i += step)
        sample.add(group.idx[i], group.plans[i]);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return kDefaultK;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return kDefaultK; }
    int best_k = kDefaultK;
    float best_ms = 1e30f;
    for (int K : kCandidates) {
        if (sample.setup(group.nmax, group.kind, K) != PERM_OK) continue;
        DeviceArena arena;
        if (arena.alloc(sample.arena_bytes()) != cudaSuccess) continue;
        sample.bind(arena.base);
        if (sample.upload(st) != PERM_OK) continue;
        if (sample.launch(st, 1) != PERM_OK) continue;   // warm-up
        cudaEventRecord(e0, st);
        if (sample.launch(st, 1) != PERM_OK) continue;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best_k = K; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    set_tuned_chunk_log2(group.nmax, group.kind, best_k);
    return best_k;
}

}  // namespace perm
