// Layer-wise kernels for HR order m = 5.
#define HRKAN_WIDE_M 5
#include "wide_inst.cuh"
