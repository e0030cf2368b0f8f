// generic_dd.cu -- generic kernels for double-double arithmetic (see generic_impl.cuh).
#define PERM_GENERIC_B 5
#include "generic_impl.cuh"

PERM_GENERIC_UNIT(dd, pk::ArithDD)
