// Layer-wise kernels for HR order m = 2.
#define HRKAN_WIDE_M 2
#include "wide_inst.cuh"
