// shim.h -- lets the walk code (core.cuh) and a generated kernel's source be
// compiled as plain host C++ and run one lane at a time, for the host
// emulation tests (test infrastructure only).  With one lane the warp-wide
// intrinsics reduce to their single-lane meaning: a vote or an OR over the
// warp is the lane's own value, a shuffle returns the lane's own value.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#define PERM_HOST_EMULATION 1
#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
#define __launch_bounds__(...)
#define __shared__
#define __align__(n) __attribute__((aligned(n)))

using std::fma;
using std::max;
using std::min;

struct perm_dim3 { unsigned x, y, z; };
struct uint4 { unsigned x, y, z, w; };
static perm_dim3 threadIdx = {0, 0, 0}, blockIdx = {0, 0, 0}, blockDim = {32, 1, 1}, gridDim = {1, 1, 1};

template <class T> inline T __shfl_sync(unsigned, T v, int) { return v; }
template <class T> inline T __shfl_down_sync(unsigned, T v, int) { return v; }
inline unsigned __reduce_or_sync(unsigned, unsigned v) { return v; }
inline bool __all_sync(unsigned, bool p) { return p; }
inline void __syncwarp() {}
inline void __syncthreads() {}
inline int __ffsll(long long v) { return __builtin_ffsll(v); }
inline int __ffs(int v) { return __builtin_ffs(v); }
inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v) { unsigned long long o = *p; *p += v; return o; }
inline unsigned long long atomicCAS(unsigned long long *p, unsigned long long c, unsigned long long v) {
    unsigned long long o = *p; if (o == c) *p = v; return o;
}
inline unsigned atomicExch(unsigned *p, unsigned v) { unsigned o = *p; *p = v; return o; }
inline int __double2hiint(double d) { uint64_t u; std::memcpy(&u, &d, 8); return (int)(uint32_t)(u >> 32); }
inline int __double2loint(double d) { uint64_t u; std::memcpy(&u, &d, 8); return (int)(uint32_t)u; }
inline double __hiloint2double(int hi, int lo) {
    const uint64_t u = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo; double d; std::memcpy(&d, &u, 8); return d;
}
inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
inline long long __double_as_longlong(double d) { long long v; std::memcpy(&v, &d, 8); return v; }
inline double __longlong_as_double(long long v) { double d; std::memcpy(&d, &v, 8); return d; }
