// generic_r192.cu -- generic kernels for exact arithmetic modulo 2^192 (see generic_impl.cuh).
#define PERM_GENERIC_B 5
#include "generic_impl.cuh"

PERM_GENERIC_EXACT_UNIT(r192, 6)
