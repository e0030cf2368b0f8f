// kernels.hpp -- host-side entry points of the precompiled kernels.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "devmat.h"

namespace perm {

// Launchers of one precompiled generic kernel family member.
struct GenericFns {
    cudaError_t (*walk)(const pk::BatchArgs &ba, int grid, int block, cudaStream_t st) = nullptr;
    cudaError_t (*direct)(const void *devmat, uint64_t g_lo, uint64_t g_hi, uint64_t *block_out, int grid, int block,
                          cudaStream_t st, int abs_shift) = nullptr;
    cudaError_t (*attr)(cudaFuncAttributes *attr) = nullptr;
    cudaError_t (*occ)(int block, size_t slot_bytes, int *blocks_per_sm) = nullptr;
    int block_log2 = 0;   // B of this family: 2^B steps unrolled per block
    size_t devmat_bytes = 0;   // the largest possible image (every value stored)
};

// kind = 2 limbs + fold: limbs 0 = FP64 (fold 0) or double-double (fold 1,
// kKindDD), 2..6 = exact modulo 2^(32 limbs); fold = 1 selects the exact
// kernels that multiply slot quadruples in 32 bits first (every row's
// absolute sum <= 127).  nmax in {16, 32, 48}.
constexpr int kKindDD = 1;
GenericFns generic_fns(int nmax, int kind);

// Per-matrix sums of a multi-matrix walk: result[m] = sum of task results
// [mats[m].task_begin, mats[m+1].task_begin) (the last ends at ntasks), in a
// fixed order, one warp per matrix.
cudaError_t batch_reduce_launch(int arith, const pk::BatchMat *mats, int nmat, uint64_t ntasks,
                                const uint64_t *task_out, uint64_t *result, cudaStream_t st);

// Serving: result[4 m ..] = sum of pool task results [seg[2m], seg[2m] + seg[2m+1]).
cudaError_t segment_reduce_launch(int arith, const uint64_t *seg, int nseg, const uint64_t *pool, uint64_t *result,
                                  cudaStream_t st);

// The GPU-SparsePerman baseline (xshared.cu): x in shared memory, a full
// product per step.  img is the CSC image built by build_xshared_image.
cudaError_t xshared_occupancy(int n, int img_bytes, int block, int *blocks_per_sm);
cudaError_t xshared_launch(const pk::WalkArgs &wa, const void *img, int img_bytes, int n, int abs_shift, int grid,
                           int block, cudaStream_t st);
cudaError_t xshared_attr(cudaFuncAttributes *attr);

// Sums ntasks task results (words per task: 2 for FP64, arith for exact) in a
// fixed order into result.
cudaError_t reduce_launch(int arith, const uint64_t *task_out, uint64_t ntasks, uint64_t *result, cudaStream_t st);

}  // namespace perm
