// Tensor-core layer kernels for units padded to 32 elements.
#define HRKAN_TC_NP 32
#include "tc_inst.cuh"
