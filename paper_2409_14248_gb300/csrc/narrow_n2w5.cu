// Fused kernels for widths [2, 5, 1] (k = 3, m = 4).
#include "narrow_inst.cuh"
HRKAN_NARROW_INSTANCE(narrow_launch_n2w5, 2, 5)
