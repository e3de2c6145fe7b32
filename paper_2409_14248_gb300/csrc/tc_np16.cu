// Tensor-core layer kernels for units padded to 16 elements.
#define HRKAN_TC_NP 16
#include "tc_inst.cuh"
