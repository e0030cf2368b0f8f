// generic.cu -- dispatch to the precompiled generic kernels, and the final
// reduction kernels.
#include <cuda_runtime.h>

#include "core.cuh"
#include "kernels.hpp"

namespace pk {

template <class A>
__global__ void __launch_bounds__(1024) k_reduce(const u64 *task_out, u64 ntasks, u64 *result) {
    reduce_tasks<A>(task_out, ntasks, result);
}

// One warp per matrix, lane-strided then a fixed shuffle tree: deterministic.
template <class A>
__global__ void __launch_bounds__(256) k_batch_reduce(const BatchMat *mats, int nmat, u64 ntasks,
                                                      const u64 *task_out, u64 *result) {
    const int m = (int)((blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (m >= nmat) return;
    const u64 b = mats[m].task_begin;
    const u64 e = (m + 1 < nmat) ? mats[m + 1].task_begin : ntasks;
    typename A::Acc acc = A::acc_zero();
    for (u64 t = b + lane; t < e; t += 32) acc = A::acc_add(acc, A::acc_load(task_out + t * (u64)A::ACC_WORDS));
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) acc = A::acc_add(acc, A::shfl_down(acc, d));
    if (lane == 0) A::acc_store(result + (u64)m * A::ACC_WORDS, acc);
}

// Serving: segment m sums pool[seg[2m] .. seg[2m] + seg[2m+1]) (task units),
// one warp per segment, fixed order.
template <class A>
__global__ void __launch_bounds__(256) k_segment_reduce(const u64 *seg, int nseg, const u64 *pool, u64 *result) {
    const int m = (int)((blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (m >= nseg) return;
    const u64 b = seg[2 * m], e = b + seg[2 * m + 1];
    typename A::Acc acc = A::acc_zero();
    for (u64 t = b + lane; t < e; t += 32) acc = A::acc_add(acc, A::acc_load(pool + t * (u64)A::ACC_WORDS));
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) acc = A::acc_add(acc, A::shfl_down(acc, d));
    if (lane == 0) A::acc_store(result + (u64)m * 4, acc);
}

}  // namespace pk

namespace perm {

cudaError_t segment_reduce_launch(int arith, const uint64_t *seg, int nseg, const uint64_t *pool, uint64_t *result,
                                  cudaStream_t st) {
    const unsigned long long *sg = reinterpret_cast<const unsigned long long *>(seg);
    const unsigned long long *in = reinterpret_cast<const unsigned long long *>(pool);
    unsigned long long *out = reinterpret_cast<unsigned long long *>(result);
    const int grid = (nseg * 32 + 255) / 256;
    if (nseg <= 0) return cudaSuccess;
    switch (arith) {
    case 0: pk::k_segment_reduce<pk::ArithF64><<<grid, 256, 0, st>>>(sg, nseg, in, out); break;
    case 1: pk::k_segment_reduce<pk::ArithExact<2>><<<grid, 256, 0, st>>>(sg, nseg, in, out); break;
    case 2: pk::k_segment_reduce<pk::ArithExact<4>><<<grid, 256, 0, st>>>(sg, nseg, in, out); break;
    case 3: pk::k_segment_reduce<pk::ArithExact<6>><<<grid, 256, 0, st>>>(sg, nseg, in, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t batch_reduce_launch(int arith, const pk::BatchMat *mats, int nmat, uint64_t ntasks,
                                const uint64_t *task_out, uint64_t *result, cudaStream_t st) {
    const unsigned long long *in = reinterpret_cast<const unsigned long long *>(task_out);
    unsigned long long *out = reinterpret_cast<unsigned long long *>(result);
    const int grid = (nmat * 32 + 255) / 256;
    if (nmat <= 0) return cudaSuccess;
    switch (arith) {
    case 0: pk::k_batch_reduce<pk::ArithF64><<<grid, 256, 0, st>>>(mats, nmat, ntasks, in, out); break;
    case 1: pk::k_batch_reduce<pk::ArithExact<2>><<<grid, 256, 0, st>>>(mats, nmat, ntasks, in, out); break;
    case 2: pk::k_batch_reduce<pk::ArithExact<4>><<<grid, 256, 0, st>>>(mats, nmat, ntasks, in, out); break;
    case 3: pk::k_batch_reduce<pk::ArithExact<6>><<<grid, 256, 0, st>>>(mats, nmat, ntasks, in, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

GenericFns generic_fns_f64(int nmax);
GenericFns generic_fns_dd(int nmax);
GenericFns generic_fns_r64(int nmax, int fold);
GenericFns generic_fns_r96(int nmax, int fold);
GenericFns generic_fns_r128(int nmax, int fold);
GenericFns generic_fns_r160(int nmax, int fold);
GenericFns generic_fns_r192(int nmax, int fold);

GenericFns generic_fns(int nmax, int kind) {
    const int limbs = kind >> 1, fold = kind & 1;
    switch (limbs) {
    case 0: return fold ? generic_fns_dd(nmax) : generic_fns_f64(nmax);
    case 2: return generic_fns_r64(nmax, fold);
    case 3: return generic_fns_r96(nmax, fold);
    case 4: return generic_fns_r128(nmax, fold);
    case 5: return generic_fns_r160(nmax, fold);
    case 6: return generic_fns_r192(nmax, fold);
    default: return GenericFns();
    }
}

cudaError_t reduce_launch(int arith, const uint64_t *task_out, uint64_t ntasks, uint64_t *result, cudaStream_t st) {
    const unsigned long long *in = reinterpret_cast<const unsigned long long *>(task_out);
    unsigned long long *out = reinterpret_cast<unsigned long long *>(result);
    switch (arith) {
    case 0: pk::k_reduce<pk::ArithF64><<<1, 1024, 0, st>>>(in, ntasks, out); break;
    case 1: pk::k_reduce<pk::ArithExact<2>><<<1, 1024, 0, st>>>(in, ntasks, out); break;
    case 2: pk::k_reduce<pk::ArithExact<4>><<<1, 1024, 0, st>>>(in, ntasks, out); break;
    case 3: pk::k_reduce<pk::ArithExact<6>><<<1, 1024, 0, st>>>(in, ntasks, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace perm
