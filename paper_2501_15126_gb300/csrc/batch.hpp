// batch.hpp -- grouping of matrices for the multi-matrix generic walk.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "devmat.h"
#include "kernels.hpp"

struct perm_plan_s;

namespace perm {

// Chunk length (log2) of an n x n matrix in a batch: the group's target,
// lowered so that the matrix still fills a 32-lane task, never below B.
int batch_chunk_log2(int n, int B, int K_target);

// The autotuned chunk target of a (NMAX, kernel family) pair (tune.cpp); the
// family is perm_plan_s::kind().
int tuned_chunk_log2(int nmax, int kind);
bool chunk_log2_is_tuned(int nmax, int kind);
struct BatchGroup;
int autotune_group(const BatchGroup &group, cudaStream_t st);

// Matrices of one NMAX bucket and one arithmetic: one launch.
struct BatchGroup {
    std::vector<int> idx;                 // positions in the caller's array
    std::vector<perm_plan_s *> plans;
    int nmax = 0, kind = 0, arith = 0, words = 3;   // kind: generic kernel family (perm_plan_s::kind())
    int img = 0;                          // image layout (kImgF64, kImgInt, kImgDD)
    GenericFns gf;
    std::vector<pk::BatchMat> mats;
    std::vector<unsigned char> images;
    uint64_t ntasks = 0;
    size_t slot_bytes = 16;                // the largest image of the group
    unsigned long long timeout_ns = 0;     // device-side deadline (0 = none)
    int grid = 1, block = 256, regs = 0;
    unsigned char *d_images = nullptr;
    pk::BatchMat *d_mats = nullptr;
    uint64_t *d_task_out = nullptr, *d_result = nullptr, *d_counters = nullptr;

    void add(int i, perm_plan_s *p) { idx.push_back(i); plans.push_back(p); }
    int setup(int nmax, int kind, int K_target);   // perm_status_t
    size_t arena_bytes() const;
    void bind(unsigned char *base);
    int upload(cudaStream_t st);
    int launch(cudaStream_t st, int zero_skip);
};

// A device allocation freed on scope exit.
struct DeviceArena {
    unsigned char *base = nullptr;
    cudaError_t alloc(size_t bytes) { return cudaMalloc(reinterpret_cast<void **>(&base), bytes); }
    ~DeviceArena() { if (base) cudaFree(base); }
};

// Two timing events destroyed on scope exit.
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t create() {
        cudaError_t e = cudaEventCreate(&e0);
        return e != cudaSuccess ? e : cudaEventCreate(&e1);
    }
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

}  // namespace perm
