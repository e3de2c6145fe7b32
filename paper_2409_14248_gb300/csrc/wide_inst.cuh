// Instantiates the layer-wise kernels for one HR order HRKAN_WIDE_M (included
// by wide_m*.cu, one translation unit each so that they compile in parallel).
#pragma once

#include "wide_kernels.cuh"

namespace hrkan {
template cudaError_t wide_forward_layer_m<HRKAN_WIDE_M>(const WideLayer&, unsigned, bool, cudaStream_t);
template cudaError_t wide_adjoint_layer_m<HRKAN_WIDE_M>(const WideLayer&, unsigned, cudaStream_t);
template cudaError_t wide_dw_layer_m<HRKAN_WIDE_M>(const WideDw&, unsigned, bool, cudaStream_t);
}  // namespace hrkan
