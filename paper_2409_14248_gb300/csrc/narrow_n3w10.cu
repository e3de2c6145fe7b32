// Fused kernels for widths [2, 10, 10, 1] (k = 3, m = 4).
#include "narrow_inst.cuh"
HRKAN_NARROW_INSTANCE(narrow_launch_n3w10, 3, 10)
