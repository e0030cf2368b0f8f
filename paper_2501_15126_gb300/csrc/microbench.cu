// microbench.cu -- FP64 and INT32 issue-rate probes: the ALU roofline
// denominators of the walk (its time goes to FP64 adds/multiplies on the
// FP64 path and to 32-bit integer multiply-adds on the exact path).
// Each thread runs 8 independent dependency chains so that issue, not
// latency, bounds the rate.
#include <cuda_runtime.h>

#include "perm.h"
#include "plan.hpp"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_fp64_rate(double *out, int iters, double b, double c) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-9 * (t + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[t] = s;
}

__global__ void __launch_bounds__(256) k_imad_rate(unsigned *out, int iters, unsigned m, unsigned c) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned u[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) u[k] = t * 7u + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) u[k] = u[k] * m + c;
    }
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += u[k];
    out[t] = s;
}

}  // namespace

extern "C" perm_status_t perm_issue_rates(void *stream, double *fp64_ops_per_s, double *imad_ops_per_s) {
    if (!fp64_ops_per_s || !imad_ops_per_s) return perm::fail(PERM_ERR_ARG, "NULL output");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return perm::cuda_fail(e, "device query");
    const int block = 256, grid = sms * 8;
    void *buf = nullptr;
    if ((e = cudaMalloc(&buf, (size_t)grid * block * sizeof(double))) != cudaSuccess) return perm::cuda_fail(e, "cudaMalloc");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms_f = 0.f, ms_i = 0.f;
    const int it_f = 400, it_i = 8000;
    k_fp64_rate<<<grid, block, 0, st>>>((double *)buf, 4, 0.999999, 1e-7);   // warm-up
    cudaEventRecord(e0, st);
    k_fp64_rate<<<grid, block, 0, st>>>((double *)buf, it_f, 0.999999, 1e-7);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms_f, e0, e1);
    k_imad_rate<<<grid, block, 0, st>>>((unsigned *)buf, 4, 1664525u, 1013904223u);
    cudaEventRecord(e0, st);
    k_imad_rate<<<grid, block, 0, st>>>((unsigned *)buf, it_i, 1664525u, 1013904223u);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms_i, e0, e1);
    e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) return perm::cuda_fail(e, "issue-rate kernels");
    const double threads = (double)grid * block;
    *fp64_ops_per_s = threads * it_f * kUnroll * kChains / (ms_f * 1e-3);
    *imad_ops_per_s = threads * it_i * kUnroll * kChains / (ms_i * 1e-3);
    return PERM_OK;
}
