// Table of the fused narrow-network shapes compiled into the library.
#include "internal.h"
#include "narrow.cuh"

namespace hrkan {

cudaError_t narrow_launch_n2w5(int, unsigned, const NarrowParams&, int*, int, bool, cudaStream_t);
cudaError_t narrow_launch_n3w10(int, unsigned, const NarrowParams&, int*, int, bool, cudaStream_t);
cudaError_t narrow_launch_n3w16(int, unsigned, const NarrowParams&, int*, int, bool, cudaStream_t);
cudaError_t narrow_launch_n2w5_batch(int, unsigned, const BatchParams&, int*, int, bool, cudaStream_t);
cudaError_t narrow_launch_n3w10_batch(int, unsigned, const BatchParams&, int*, int, bool, cudaStream_t);
cudaError_t narrow_launch_n3w16_batch(int, unsigned, const BatchParams&, int*, int, bool, cudaStream_t);

int narrow_net_id(int n_layers, int wh) {
    if (n_layers == 2 && wh == 5) return 0;
    if (n_layers == 3 && wh == 10) return 1;
    if (n_layers == 3 && wh == 16) return 2;
    return -1;
}

cudaError_t narrow_launch(int net_id, int mode, unsigned mask, const NarrowParams& p, int* grid, int max_grid,
                          bool launch, cudaStream_t s) {
    switch (net_id) {
        case 0: return narrow_launch_n2w5(mode, mask, p, grid, max_grid, launch, s);
        case 1: return narrow_launch_n3w10(mode, mask, p, grid, max_grid, launch, s);
        case 2: return narrow_launch_n3w16(mode, mask, p, grid, max_grid, launch, s);
    }
    return cudaErrorNotSupported;
}

cudaError_t narrow_batch_launch(int net_id, int mode, unsigned mask, const BatchParams& p, int* grid, int max_grid,
                                bool launch, cudaStream_t s) {
    switch (net_id) {
        case 0: return narrow_launch_n2w5_batch(mode, mask, p, grid, max_grid, launch, s);
        case 1: return narrow_launch_n3w10_batch(mode, mask, p, grid, max_grid, launch, s);
        case 2: return narrow_launch_n3w16_batch(mode, mask, p, grid, max_grid, launch, s);
    }
    return cudaErrorNotSupported;
}

}  // namespace hrkan
