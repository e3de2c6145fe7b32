// Dispatch of the layer-wise kernels (wide_kernels.cuh) by the HR order m of
// Eq. 2; each order is compiled in its own translation unit (wide_m*.cu).
#include "wide.cuh"

namespace hrkan {

template <int MW>
cudaError_t wide_forward_layer_m(const WideLayer& p, unsigned mask, bool first, cudaStream_t s);
template <int MW>
cudaError_t wide_adjoint_layer_m(const WideLayer& p, unsigned mask, cudaStream_t s);
template <int MW>
cudaError_t wide_dw_layer_m(const WideDw& p, unsigned mask, bool first, cudaStream_t s);

cudaError_t wide_forward_layer(const WideLayer& p, unsigned mask, bool first, cudaStream_t s) {
    switch (p.g.m) {
        case 2: return wide_forward_layer_m<2>(p, mask, first, s);
        case 3: return wide_forward_layer_m<3>(p, mask, first, s);
        case 4: return wide_forward_layer_m<4>(p, mask, first, s);
        case 5: return wide_forward_layer_m<5>(p, mask, first, s);
        case 6: return wide_forward_layer_m<6>(p, mask, first, s);
    }
    return cudaErrorNotSupported;
}

cudaError_t wide_adjoint_layer(const WideLayer& p, unsigned mask, cudaStream_t s) {
    switch (p.g.m) {
        case 2: return wide_adjoint_layer_m<2>(p, mask, s);
        case 3: return wide_adjoint_layer_m<3>(p, mask, s);
        case 4: return wide_adjoint_layer_m<4>(p, mask, s);
        case 5: return wide_adjoint_layer_m<5>(p, mask, s);
        case 6: return wide_adjoint_layer_m<6>(p, mask, s);
    }
    return cudaErrorNotSupported;
}

cudaError_t wide_dw_layer(const WideDw& p, unsigned mask, bool first, cudaStream_t s) {
    switch (p.g.m) {
        case 2: return wide_dw_layer_m<2>(p, mask, first, s);
        case 3: return wide_dw_layer_m<3>(p, mask, first, s);
        case 4: return wide_dw_layer_m<4>(p, mask, first, s);
        case 5: return wide_dw_layer_m<5>(p, mask, first, s);
        case 6: return wide_dw_layer_m<6>(p, mask, first, s);
    }
    return cudaErrorNotSupported;
}

}  // namespace hrkan
