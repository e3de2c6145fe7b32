// Tensor-core layer kernels for units padded to 40 elements.
#define HRKAN_TC_NP 40
#include "tc_inst.cuh"
