// Internal (C++) interface between the C ABI layer and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hr_device.cuh"

namespace hrkan {

struct NarrowParams;
struct BatchParams;

// ---- fused narrow-network kernels (narrow_*.cu) --------------------------------
// Shapes with a fused kernel: widths [2, WH, 1] or [2, WH, WH, 1], k = 3, m = 4.
// Returns the table id, or -1.
int narrow_net_id(int n_layers, int wh);
// Launch mode (MODE_FWD / MODE_BWD / MODE_TRAIN) for mask on `*grid` blocks.
// If *grid <= 0 it is replaced by the persistent grid (SMs x resident blocks,
// capped at max_grid and at the number of tiles) and nothing is launched when
// `launch` is false.  Returns cudaErrorNotSupported for a mask with no kernel.
cudaError_t narrow_launch(int net_id, int mode, unsigned mask, const NarrowParams& p, int* grid,
                          int max_grid, bool launch, cudaStream_t s);

// Same for the multi-instance kernels (MODE_FWD / MODE_TRAIN) over a work list;
// *grid is capped at max_grid and at the number of items.
cudaError_t narrow_batch_launch(int net_id, int mode, unsigned mask, const BatchParams& p, int* grid, int max_grid,
                                bool launch, cudaStream_t s);

// ---- reductions, Adam, residual (reduce.cu) -------------------------------------
struct ReduceParams {
    const float* partial;   // [G][P]
    int G;
    int64_t P;
    float* dW;              // optional output gradient
    int accumulate;
    int do_adam;
    float* W;
    double* m1;
    double* m2;
    double lr, b1, b2, eps, c1, c2;   // c1 = 1 - b1^t, c2 = 1 - b2^t
    int* t_counter;                   // non-null: t = t_counter[1] (set by the fused kernel), c1/c2 from it
    const double* loss_partial;       // [Gl][2] or null
    int Gl;
    double* loss;                     // [3]
    double alpha;
    int64_t n0, n1;
    int* status;                      // optional device error word: HRKAN_ENONFINITE for a non-finite loss
};
cudaError_t launch_reduce(const ReduceParams& p, cudaStream_t s);

// Per-instance reduction + Adam for the multi-instance step: instance i owns
// partial rows [item_off[i], item_off[i+1]) of [n_items][P].
struct BatchReduceParams {
    const float* partial;
    const int* item_off;       // [n_inst + 1] device
    int n_inst;
    int64_t P;
    float* W;                  // [n_inst][P]
    double* m1;
    double* m2;
    double lr, b1, b2, eps, c1, c2;
    int* t_counter;
    const double* loss_partial;  // [n_items][2] (rows of instance i: [item_off[i], item_off[i+1]))
    const int* loss_off;         // optional [n_inst + 1]: the loss-partial rows of instance i are
                                 // [loss_off[i], loss_off[i+1]) instead
    const float* counts;         // [n_inst][2] interior / boundary point counts
    double* loss;                // [n_inst][3]
    float* dW;                   // optional [n_inst][P]
    double alpha;
    int* status;                 // optional device error word: HRKAN_ENONFINITE for a non-finite loss
};
cudaError_t launch_batch_reduce(const BatchReduceParams& p, cudaStream_t s);

struct ResidualParams {
    PdeParams pde;
    unsigned mask;
    const float* x;        // [2][N]
    const float* jets;     // [J][N]
    int64_t N;
    float* dL;             // [J][N] or null
    const float* u_bnd;
    const float* g_bnd;
    int64_t Nb;
    float* dLb;            // [Nb] or null
    float scale0, scale1;
    double* loss_partial;  // [grid][2]
    int* t_counter;        // optional device step counter: t_counter[1] = t_counter[0] + 1
};
// Enqueue the residual kernel on `grid` blocks (grid must be <= the rows of loss_partial).
cudaError_t launch_residual(const ResidualParams& p, int grid, cudaStream_t s);
// The Poisson residual in three coordinates (kind 3): x [3][N], jets the seven rows of
// mask 0x7F (u, u_x, u_y, u_z, u_xx, u_yy, u_zz), the third frequency in pde.lam.
cudaError_t launch_residual3(const ResidualParams& p, int grid, cudaStream_t s);
bool residual_mask_supported(unsigned mask);

// ---- layer-wise multi-instance path (lbatch.cu) ------------------------------------
// Points of every instance sit in whole blocks of LB_BLOCK points (the layer
// kernels' point block, two tensor-core tiles), padded with copies of the
// instance's last point.
constexpr int LB_BLOCK = 256;
struct BatchInst;
struct LbResidualParams {
    PdeParams pde;                 // kind, lam, nu, alpha (a, b, src per instance)
    unsigned mask;
    const BatchInst* inst;         // [n_inst]: a, b, src, scale0 = 2 alpha / n_int, scale1 = 2 / n_bnd
    const float* x;                // padded interior coordinates [2][Ni]
    const float* jets;             // [J][Ni]
    int64_t Ni;
    float* dL;                     // [J][Ni] (written; zero at padding points)
    const float* u_bnd;            // [Nb]
    const float* g_bnd;            // padded boundary targets [Nb]
    int64_t Nb;
    float* dLb;                    // [Nb] (written; zero at padding points)
    int nbi, nbb;                  // interior / boundary point blocks
    const int* blk_inst_int;       // [nbi] instance of each block
    const int* blk_valid_int;      // [nbi] real points in each block
    const int* blk_inst_bnd;       // [nbb]
    const int* blk_valid_bnd;      // [nbb]
    const int* lrow_int;           // [nbi] loss-partial row of each block
    const int* lrow_bnd;           // [nbb]
    double* loss_partial;          // [rows][2] (interior, boundary sums of squares)
    int* t_counter;                // optional device step counter: t_counter[1] = t_counter[0] + 1
};
// dst[r][p] = src[r][pt_src[p]], r < rows, p < n_dst (source rows n_src apart).
cudaError_t lb_gather(const float* src, int64_t n_src, const int* pt_src, float* dst, int64_t n_dst, int rows,
                      cudaStream_t s);
// dst[r][pt_src[p]] = src[r][p] for the real points p < n_src of the padded layout.
cudaError_t lb_scatter(const float* src, int64_t n_src, const int* pt_src, const int* blk_valid, float* dst,
                       int64_t n_dst, int rows, cudaStream_t s);
// Residual and loss partials of both point sets, one block per point block (masks 0x0F, 0x1F, 0x2F).
cudaError_t lb_residual(const LbResidualParams& p, cudaStream_t s);
// The output layer (O = 1) of one point set: forward, residual (or boundary
// misfit), loss partials, input adjoint and weight gradient in one launch,
// one block per weight-gradient chunk.
struct LbTailParams {
    const float* W;                // instance 0's output layer [1][I][n]; instance i at W + i * w_stride
    int64_t w_stride;
    int I;                         // the layer's inputs
    Grid g;
    const float* z;                // its input jets [J][I][N] (the tape)
    float* gz;                     // dL/d(input jets) [J][I][N] (written; zero at padding points)
    uint16_t* gz_bf;               // non-null: gz goes out as BF16 [J * I][N] here instead (N is a
                                   // multiple of 256: the layer below's tensor-core operand layout)
    int64_t N;                     // padded points of the set
    const float* x;                // interior set: padded coordinates [2][N]
    const float* g_bnd;            // boundary set: padded targets [N]
    PdeParams pde;                 // kind, lam, nu, alpha (a, b, src per instance)
    const BatchInst* inst;
    const int* blk_valid;          // real points of each point block
    const int* lrow;               // loss-partial row of each point block
    const int4* chunks;            // points [x, y) of instance w, gradient partial row z
    float* partial;                // [rows][P]: the layer's columns [col0, col0 + I*n) of row z
    int64_t P, col0;
    double* loss_partial;          // [rows][2]
    int* t_counter;                // optional device step counter: t_counter[1] = t_counter[0] + 1
};
// mask: the interior jet mask (0x0F, 0x1F, 0x2F); bnd: the boundary set (value row only).
cudaError_t lb_tail(const LbTailParams& p, unsigned mask, bool bnd, int nchunk, cudaStream_t s);

// out[c] = fixed-order sum of rows [0, rows) of src (row stride `stride`), c < cols.
cudaError_t sum_rows(const float* src, int rows, int64_t stride, int64_t cols, float* out, cudaStream_t s);

// Sets the thread's last-error message and returns code.
int set_last_error(int code, const char* msg);

}  // namespace hrkan
