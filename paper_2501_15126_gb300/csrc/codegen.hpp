// codegen.hpp -- per-matrix kernel generation (Sec. III-B, Sec. V) and NVRTC.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "devmat.h"
#include "perm.h"

struct perm_plan_s;

namespace perm {

// Algorithm 4 constants re-measured for GB300 (see DESIGN notes in codegen.cpp).
constexpr double kDefaultGRRatio = 2.0;
constexpr int kCodegenBaseRegs = 48;

struct CodegenKernel {
    void *module = nullptr;     // CUmodule (owned by the process-wide cache)
    void *function = nullptr;   // CUfunction
    int regs = 0;
    int block = 256;
    int blocks_per_sm = 0;
    int block_log2 = 5;
    bool cached = false;
    bool owned = false;         // not in the cache: unloaded with the plan
};

// log2 of the generated kernel's unrolled block for the plan's arithmetic.
int codegen_block_log2(const perm_plan_s &P);

// The CUDA C++ text for the plan's matrix, order and split (P.k, P.c).
std::string codegen_source(const perm_plan_s &P);

// Generates, compiles (NVRTC, sm_103a) and loads the kernel, or takes it from
// the cache; fills P.cg, P.regs and P.ms_compile.
perm_status_t codegen_build(perm_plan_s &P, std::string &err);

cudaError_t codegen_launch(perm_plan_s &P, const pk::WalkArgs &wa, cudaStream_t st);

void codegen_release(perm_plan_s &P);

// PERM_CODEGEN_NO_FOLD=1 in the environment: exact generated kernels multiply
// every row into the ring on its own.
bool codegen_no_fold();

}  // namespace perm
