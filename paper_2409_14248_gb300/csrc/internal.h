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
    const double* loss_partial;  // [n_items][2]
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
bool residual_mask_supported(unsigned mask);

// out[c] = fixed-order sum of rows [0, rows) of src (row stride `stride`), c < cols.
cudaError_t sum_rows(const float* src, int rows, int64_t stride, int64_t cols, float* out, cudaStream_t s);

// Sets the thread's last-error message and returns code.
int set_last_error(int code, const char* msg);

}  // namespace hrkan
