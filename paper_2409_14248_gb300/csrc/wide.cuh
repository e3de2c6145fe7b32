// Launch interface of the layer-wise kernels for wide networks (wide.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hr_device.cuh"

namespace hrkan {

// One layer: I inputs, O outputs, weights W [O][I][n].
struct WideLayer {
    const float* W;
    int I, O;
    const float* z;    // input jets [J][I][N] (first layer: coordinates [D][N])
    float* y;          // forward: output jets [J][O][N]
    const float* gy;   // adjoint: dL/d(output jets) [J][O][N]
    float* gz;         // adjoint: dL/d(input jets) [J][I][N]
    int64_t N;
    Grid g;
    // first layer: the coordinates that jet directions 0 and 1 differentiate
    // along (-1: none); a three-input network runs as passes over direction pairs
    int seed0 = 0, seed1 = 1;
    // adjoint: first point of this launch (point sets above the grid's y limit
    // run as several launches)
    int64_t p0 = 0;
    // many instances (batched path): point block b (WB points) belongs to
    // instance blk_inst[b], whose weights are W + blk_inst[b] * w_stride
    const int* blk_inst = nullptr;
    int64_t w_stride = 0;
};

// Weight gradient of one layer into partial rows [row0, row0 + GP) of a
// [rows][P] buffer, columns [col0, col0 + O*I*n).
struct WideDw {
    const float* z;    // input jets [J][I][N] (first layer: coordinates)
    const float* gy;   // [J][O][N]
    int I, O;
    int64_t N;
    float* partial;
    int64_t P;
    int64_t col0;
    int row0;
    int GP;            // point groups = partial rows written
    Grid g;
    int seed0 = 0, seed1 = 1;   // first layer: as in WideLayer
    // many instances (batched path): GP chunks, chunk c covering points
    // [chunks[c].x, chunks[c].y) (multiples of WB) of instance chunks[c].w and
    // writing partial row chunks[c].z (row0 unused); nullptr: the point tiles
    // gp, gp + GP, ... into row row0 + gp
    const int4* chunks = nullptr;
};

cudaError_t wide_forward_layer(const WideLayer& p, unsigned mask, bool first, cudaStream_t s);
cudaError_t wide_adjoint_layer(const WideLayer& p, unsigned mask, cudaStream_t s);
cudaError_t wide_dw_layer(const WideDw& p, unsigned mask, bool first, cudaStream_t s);

}  // namespace hrkan
