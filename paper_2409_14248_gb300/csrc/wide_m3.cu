// Layer-wise kernels for HR order m = 3.
#define HRKAN_WIDE_M 3
#include "wide_inst.cuh"
