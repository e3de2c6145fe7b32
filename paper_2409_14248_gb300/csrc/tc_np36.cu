// Tensor-core layer kernels for units padded to 36 elements.
#define HRKAN_TC_NP 36
#include "tc_inst.cuh"
