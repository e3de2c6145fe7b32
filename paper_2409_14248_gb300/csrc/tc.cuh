// Tensor-core forward of one hidden layer (tc_kernel.cuh, tc_jets.cu, tc_np*.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hrkan.h"
#include "hr_device.cuh"

namespace hrkan {

// Template precision of the forward kernel for HRKAN_BF16 layers: each
// contraction input x is carried as two bfloat16 values, x = x_hi + x_lo
// (x_hi = bf16(x), x_lo = bf16(x - x_hi)), and every product as
// a_hi w_hi + a_lo w_hi + a_hi w_lo (the a_lo w_lo term dropped), with FP32
// accumulation.  The values of this enum continue hrkan_prec's.
constexpr int TC_BF16X3 = 3;
// W tiles (128-byte rows, TERMS tiles of O rows each) the forward kernel keeps in flight.
constexpr int TC_W_BUFFERS = 8;

struct TcLayer {
    const float* z;   // input jets [J][I][N]
    float* y;         // output jets [J][O][N]
    int I, O;
    int64_t N;
    int ks;           // K slots (one MMA each) over the padded units
    int nbox;         // W tiles of 128 bytes per row (4 slots each)
    int ring;         // A ring slots in TMEM
    int ntiles;       // tiles of 128 points
    Grid g;
    int* status;      // device error word (HRKAN_ETIMEOUT on a timed-out wait)
    // many instances (batched path): tile t (128 points) belongs to instance
    // blk_inst[t / 2] (point blocks of 256), whose W tiles start at row
    // blk_inst[t / 2] * TERMS * O of the tensor map; nullptr: one instance
    const int* blk_inst = nullptr;
    // TMEM columns each CTA allocates (512, or 256 when two CTAs share an SM)
    uint32_t tmem_cols = 512;
};

// Layers the tensor-core kernel handles: 16 <= O <= 64, O % 16 == 0,
// J * O <= 320, n <= 64, masks 0x01 / 0x0F / 0x1F.
bool tc_layer_supported(int prec, int I, int O, int n, unsigned mask);
// Elements of the converted weight buffer of one layer.
int64_t tc_w_elems(int O, int I, int n, int prec);
// Converts W (float32 [O][I][n]) into w_prep (tc_w_elems elements of 2 or 4
// bytes, units padded) and runs the tensor-core contraction: y = jets of the
// layer output.
// Many instances: W holds n_inst layers w_stride floats apart, w_prep
// n_inst * tc_w_elems elements, and blk_inst (device, one entry per 256
// points) names the instance of every point block.
cudaError_t tc_forward_layer(const float* W, void* w_prep, const float* z, float* y, int I, int O, int64_t N,
                             const Grid& g, int prec, unsigned mask, int* status, cudaStream_t s, int n_inst = 1,
                             int64_t w_stride = 0, const int* blk_inst = nullptr);

// Tensor-core weight gradient of one hidden layer (tc_dw.cu): BF16 inputs,
// FP32 accumulation, 16 <= O <= 64 with O % 16 == 0, n <= 64.
bool tc_dw_supported(int prec, int I, int O, int n, unsigned mask);
// gy [J][O][N] float32 -> BF16 [J*O][N rounded up to 64] (zero past N).
cudaError_t tc_gy_to_bf16(const float* gy, void* gy_bf, int J, int O, int64_t N, cudaStream_t s);
// BF16 elements of the gy copy the kernel needs (J * O * N rounded up to 64 points).
int64_t tc_dw_gy_elems(int J, int O, int64_t N);
// dW of the layer (columns [col0, col0 + O*I*n) of rows [row0, row0 + nchunk)
// of partial [rows][P]) from input jets z [J][I][N] and output-jet gradients
// gy [J][O][N]; gy_bf is scratch of tc_dw_gy_elems 2-byte elements.
// first: z is the coordinates [2][N] (layer 0).
// chunks (batched path, device, nchunk entries): chunk c covers points
// [chunks[c].x, chunks[c].y) (multiples of 256) and writes partial row
// chunks[c].z (row0 unused); nullptr: the points split evenly into rows
// row0 .. row0 + nchunk - 1.
// gy_ready: gy_bf already holds the BF16 copy (gy unused), e.g. written so by
// the layer above's adjoint.
cudaError_t tc_dw_layer(const float* z, const float* gy, void* gy_bf, int I, int O, int64_t N, const Grid& g,
                        unsigned mask, bool first, float* partial, int64_t P, int64_t col0, int row0, int nchunk,
                        int* status, cudaStream_t s, const int4* chunks = nullptr, bool gy_ready = false);

// Tensor-core input adjoint of one hidden layer (tc_adj.cu): BF16, masks 0x0F
// and 0x1F, after tc_dw_layer of the same layer and point set (it reuses that
// call's BF16 gy copy).  w_bf: tc_adj_w_elems 2-byte scratch elements.
bool tc_adj_supported(int prec, int I, int O, int n, unsigned mask);
int64_t tc_adj_w_elems(int O, int I, int n);
// Many instances (batched path): W holds n_inst layers w_stride floats apart,
// w_bf n_inst * tc_adj_w_elems elements, and chunk c (device, nchunk entries)
// covers points [chunks[c].x, chunks[c].y) (multiples of 256) of instance
// chunks[c].w.
// gz_bf (optional): write dL/d(input jets) as BF16 [J * I][N rounded up to
// 64] (the tc_dw_layer operand layout, zero past N) instead of FP32 into gz.
cudaError_t tc_adj_layer(const float* W, void* w_bf, const void* gy_bf, const float* z, float* gz, int I, int O,
                         int64_t N, const Grid& g, unsigned mask, int* status, cudaStream_t s, int n_inst = 1,
                         int64_t w_stride = 0, const int4* chunks = nullptr, int nchunk = 0, void* gz_bf = nullptr);

}  // namespace hrkan
