// Tensor-core layer kernels for units padded to 64 elements.
#define HRKAN_TC_NP 64
#include "tc_inst.cuh"
