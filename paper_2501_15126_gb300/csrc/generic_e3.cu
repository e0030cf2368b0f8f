// generic_e3.cu -- generic kernels for one arithmetic (see generic_impl.cuh).
#define PERM_GENERIC_B 5
#include "generic_impl.cuh"

PERM_GENERIC_UNIT(e3, pk::ArithExact<3>)
