// Tensor-core layer kernels for units padded to 48 elements.
#define HRKAN_TC_NP 48
#include "tc_inst.cuh"
