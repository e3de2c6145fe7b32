// Layer-wise kernels for HR order m = 4.
#define HRKAN_WIDE_M 4
#include "wide_inst.cuh"
