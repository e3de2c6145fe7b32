// Tensor-core layer kernels for units padded to 24 elements.
#define HRKAN_TC_NP 24
#include "tc_inst.cuh"
