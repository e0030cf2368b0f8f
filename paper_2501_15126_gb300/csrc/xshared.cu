// xshared.cu -- the GPU-SparsePerman baseline of Sec. VI-B (an ablation, not
// the library's fast path): the same Gray-code walk with each thread's x in
// shared memory (the x_shared layout of Table I: x[row * blockDim + thread]),
// the matrix read column by column from a CSC image, a running count of the
// zero entries of x (zero tracking), and the product of all n entries of x at
// every step whose x has no zero.  Chunks, tasks and the reduction are those of
// the other kernels, so results are comparable bit for bit in structure and
// within rounding in value.
#include <cuda_runtime.h>

#include "core.cuh"
#include "kernels.hpp"

namespace pk {

// Image layout (16-byte aligned sections): int n, nnz, bytes, pad;
// int colptr[n]; int rows[nnz]; (align 8) double x0[n]; double vals[nnz].
// Columns are positions 0..n-2 of the plan's order; rows are original rows.
struct XsView {
    int n, nnz;
    const int *colptr, *rows;
    const double *x0, *vals;
};

__device__ __forceinline__ XsView xs_view(const unsigned char *img) {
    XsView v;
    const int *h = reinterpret_cast<const int *>(img);
    v.n = h[0];
    v.nnz = h[1];
    v.colptr = h + 4;
    v.rows = v.colptr + v.n;
    size_t off = 16 + 4 * (size_t)(v.n + v.nnz);
    off = (off + 7) & ~(size_t)7;
    v.x0 = reinterpret_cast<const double *>(img + off);
    v.vals = v.x0 + v.n;
    return v;
}

__device__ __forceinline__ bool is_zero_bits(double d) { return (__double_as_longlong(d) << 1) == 0; }

__global__ void __launch_bounds__(256) k_walk_xshared(WalkArgs wa, const unsigned char *img, int img_bytes,
                                                       int abs_shift) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int words = img_bytes / 16;
    for (int i = threadIdx.x; i < words; i += blockDim.x)
        reinterpret_cast<uint4 *>(smem)[i] = reinterpret_cast<const uint4 *>(img)[i];
    __syncthreads();
    const XsView m = xs_view(smem);
    const int n = m.n, bd = blockDim.x, t = threadIdx.x;
    double *xs = reinterpret_cast<double *>(smem + img_bytes) + t;   // x_i at xs[i * bd]
    const int lane = t & 31;
    u64 skipped = 0;
    for (;;) {
        u64 task = 0;
        if (lane == 0) task = past_deadline(wa.timeout_ns, wa.deadline_word, wa.abort_flag) ? ~0ull : atomicAdd(wa.task_counter, 1ull);
        task = __shfl_sync(PERM_FULLMASK, task, 0);
        if (task >= wa.ntasks) break;
        u64 q = wa.chunk_lo + task * 32ull + (u64)lane;
        const bool live = q < wa.chunk_hi;
        if (!live) q = wa.chunk_hi - 1;
        const u64 g0 = q << wa.K;
        // start vector x(g0) = x0 + the columns set in Gray(g0), and its zeros
        for (int i = 0; i < n; ++i) xs[i * bd] = m.x0[i];
        u64 G = g0 ^ (g0 >> 1);
        while (G) {
            const int j = ctz64(G);
            G &= G - 1;
            for (int k = m.colptr[j]; k < m.colptr[j + 1]; ++k) xs[m.rows[k] * bd] += m.vals[k];
        }
        int zeros = 0;
        for (int i = 0; i < n; ++i) zeros += is_zero_bits(xs[i * bd]) ? 1 : 0;
        ArithF64::Acc acc = ArithF64::acc_zero();
        ArithF64::Blk blk = ArithF64::blk_zero();
        const u64 len = 1ull << wa.K;
        for (u64 l = 0; l < len; ++l) {
            const u64 g = g0 + l;
            if (l) {   // Theorem 1: column ctz(g), + iff bit ctz(g)+1 of g is 0
                const int j = ctz64(g);
                const double s = ((g >> (j + 1)) & 1ull) ? -1.0 : 1.0;
                for (int k = m.colptr[j]; k < m.colptr[j + 1]; ++k) {
                    double *px = xs + m.rows[k] * bd;
                    const double o = *px, v = fma(s, m.vals[k], o);
                    zeros += (is_zero_bits(v) ? 1 : 0) - (is_zero_bits(o) ? 1 : 0);
                    *px = v;
                }
            }
            if (zeros == 0) {   // zero tracking: skip the product while some x_i is 0
                double p = xs[0];
                for (int i = 1; i < n; ++i) p *= xs[i * bd];
                if (g & 1ull) ArithF64::blk_add<-1>(blk, p); else ArithF64::blk_add<1>(blk, p);
                ArithF64::blk_abs(blk, p, abs_shift);
            } else if (live) {
                ++skipped;
            }
            if ((l & 255) == 255) {
                ArithF64::acc_merge(acc, blk);
                blk = ArithF64::blk_zero();
            }
        }
        ArithF64::acc_merge(acc, blk);
        if (!live) acc = ArithF64::acc_zero();
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) acc = ArithF64::acc_add(acc, ArithF64::shfl_down(acc, d));
        if (lane == 0) ArithF64::acc_store(wa.task_out + task * (u64)ArithF64::ACC_WORDS, acc);
    }
    if (wa.skip_counter && skipped) atomicAdd(wa.skip_counter, skipped);
}

}  // namespace pk

namespace perm {

size_t xshared_smem(int n, int img_bytes, int block) { return (size_t)img_bytes + (size_t)n * block * sizeof(double); }

cudaError_t xshared_occupancy(int n, int img_bytes, int block, int *blocks_per_sm) {
    const size_t smem = xshared_smem(n, img_bytes, block);
    cudaError_t e = cudaFuncSetAttribute(pk::k_walk_xshared, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pk::k_walk_xshared, block, smem);
}

cudaError_t xshared_launch(const pk::WalkArgs &wa, const void *img, int img_bytes, int n, int abs_shift, int grid,
                           int block, cudaStream_t st) {
    const size_t smem = xshared_smem(n, img_bytes, block);
    cudaError_t e = cudaFuncSetAttribute(pk::k_walk_xshared, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    pk::k_walk_xshared<<<grid, block, smem, st>>>(wa, static_cast<const unsigned char *>(img), img_bytes, abs_shift);
    return cudaGetLastError();
}

cudaError_t xshared_attr(cudaFuncAttributes *attr) { return cudaFuncGetAttributes(attr, pk::k_walk_xshared); }

}  // namespace perm
