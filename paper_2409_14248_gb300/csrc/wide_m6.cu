// Layer-wise kernels for HR order m = 6.
#define HRKAN_WIDE_M 6
#include "wide_inst.cuh"
