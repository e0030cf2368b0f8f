// generic_r128.cu -- generic kernels for exact arithmetic modulo 2^128 (see generic_impl.cuh).
#define PERM_GENERIC_B 5
#include "generic_impl.cuh"

PERM_GENERIC_EXACT_UNIT(r128, 4)
