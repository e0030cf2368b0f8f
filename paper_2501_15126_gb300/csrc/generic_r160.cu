// generic_r160.cu -- generic kernels for exact arithmetic modulo 2^160 (see generic_impl.cuh).
#define PERM_GENERIC_B 5
#include "generic_impl.cuh"

PERM_GENERIC_EXACT_UNIT(r160, 5)
