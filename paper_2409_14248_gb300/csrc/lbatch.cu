// Kernels of the layer-wise multi-instance path (many independent networks of
// one shape trained together, the batched form of the training experiments of
// Section 4).  Every instance's points sit in a block-padded layout: instance
// i owns whole blocks of LB_BLOCK points, the last one filled up with copies of
// the instance's last point, so that every block (and every 128-point tensor-
// core tile) belongs to one instance and the layer kernels find its weights
// from a per-block table.  Padding points get a zero loss gradient, so they add
// exactly nothing to any weight gradient (every reverse step is linear in it).
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "narrow.cuh"

namespace hrkan {

namespace {

// dst[r][p] = src[r][pt_src[p]] for rows r < rows, padded points p < n_dst.
__global__ void lb_gather_kernel(const float* __restrict__ src, int64_t n_src, const int* __restrict__ pt_src,
                                 float* __restrict__ dst, int64_t n_dst, int rows) {
    const int64_t total = int64_t(rows) * n_dst;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = t / n_dst, p = t % n_dst;
        dst[t] = src[r * n_src + pt_src[p]];
    }
}

// dst[r][pt_src[p]] = src[r][p] for the real (non-padding) points p.
__global__ void lb_scatter_kernel(const float* __restrict__ src, int64_t n_src, const int* __restrict__ pt_src,
                                  const int* __restrict__ blk_valid, float* __restrict__ dst, int64_t n_dst, int rows) {
    const int64_t total = int64_t(rows) * n_src;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = t / n_src, p = t % n_src;
        if (int(p % LB_BLOCK) < blk_valid[p / LB_BLOCK]) dst[r * n_dst + pt_src[p]] = src[t];
    }
}

// One block per point block: blocks [0, nbi) of the interior set, then
// [nbi, nbi + nbb) of the boundary set.  The instance's Poisson frequencies
// and loss scales come from its BatchInst; kind, lam, nu and alpha are shared.
template <unsigned MASK>
__global__ void __launch_bounds__(LB_BLOCK) lb_residual_kernel(LbResidualParams p) {
    using JT = Jet<MASK>;
    constexpr int J = JT::J;
    const int blk = blockIdx.x, tid = threadIdx.x;
    if (p.t_counter && blk == 0 && tid == 0) p.t_counter[1] = p.t_counter[0] + 1;
    double l = 0.0;
    int row, col;
    if (blk < p.nbi) {
        const int inst = p.blk_inst_int[blk];
        const bool valid = tid < p.blk_valid_int[blk];
        const int64_t pt = int64_t(blk) * LB_BLOCK + tid, N = p.Ni;
        const BatchInst bi = p.inst[inst];
        PdeParams pde = p.pde;
        pde.a = bi.a;
        pde.b = bi.b;
        pde.src = bi.src;
        float u[J], gu[J];
#pragma unroll
        for (int r = 0; r < J; ++r) u[r] = p.jets[r * N + pt];
        const float r = pde_residual<MASK>(pde, p.x[pt], p.x[N + pt], u);
        if (valid) {
            l = double(r) * double(r);
            pde_residual_grad<MASK>(pde, r, u, bi.scale0, gu);
        } else {
#pragma unroll
            for (int q = 0; q < J; ++q) gu[q] = 0.0f;
        }
#pragma unroll
        for (int q = 0; q < J; ++q) p.dL[q * N + pt] = gu[q];
        row = p.lrow_int[blk];
        col = 0;
    } else {
        const int b = blk - p.nbi;
        const int inst = p.blk_inst_bnd[b];
        const bool valid = tid < p.blk_valid_bnd[b];
        const int64_t pt = int64_t(b) * LB_BLOCK + tid;
        const float d = p.u_bnd[pt] - p.g_bnd[pt];
        if (valid) l = double(d) * double(d);
        p.dLb[pt] = valid ? p.inst[inst].scale1 * d : 0.0f;
        row = p.lrow_bnd[b];
        col = 1;
    }
    __shared__ double red[LB_BLOCK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((tid & 31) == 0) red[tid >> 5] = l;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int t = 0; t < LB_BLOCK / 32; ++t) a += red[t];   // fixed order
        p.loss_partial[2 * int64_t(row) + col] = a;
        p.loss_partial[2 * int64_t(row) + 1 - col] = 0.0;
    }
}

int grid_for(int64_t total) { return int(std::min<int64_t>(std::max<int64_t>((total + 255) / 256, 1), 8192)); }

}  // namespace

cudaError_t lb_gather(const float* src, int64_t n_src, const int* pt_src, float* dst, int64_t n_dst, int rows,
                      cudaStream_t s) {
    if (n_dst == 0) return cudaSuccess;
    lb_gather_kernel<<<grid_for(int64_t(rows) * n_dst), 256, 0, s>>>(src, n_src, pt_src, dst, n_dst, rows);
    return cudaGetLastError();
}

cudaError_t lb_scatter(const float* src, int64_t n_src, const int* pt_src, const int* blk_valid, float* dst,
                       int64_t n_dst, int rows, cudaStream_t s) {
    if (n_src == 0) return cudaSuccess;
    lb_scatter_kernel<<<grid_for(int64_t(rows) * n_src), 256, 0, s>>>(src, n_src, pt_src, blk_valid, dst, n_dst,
                                                                       rows);
    return cudaGetLastError();
}

cudaError_t lb_residual(const LbResidualParams& p, cudaStream_t s) {
    const int grid = p.nbi + p.nbb;
    if (grid == 0) return cudaSuccess;
    switch (p.mask) {
        case 0x0Fu: lb_residual_kernel<0x0Fu><<<grid, LB_BLOCK, 0, s>>>(p); break;
        case 0x1Fu: lb_residual_kernel<0x1Fu><<<grid, LB_BLOCK, 0, s>>>(p); break;
        case 0x2Fu: lb_residual_kernel<0x2Fu><<<grid, LB_BLOCK, 0, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hrkan
