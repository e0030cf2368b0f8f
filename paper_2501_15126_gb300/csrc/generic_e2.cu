// generic_e2.cu -- generic kernels for one arithmetic (see generic_impl.cuh).
#define PERM_GENERIC_B 5
#include "generic_impl.cuh"

PERM_GENERIC_UNIT(e2, pk::ArithExact<2>)
