// Cross-block reductions, the Adam step and the stand-alone residual kernel.
//
// reduce_kernel sums per-block weight-gradient partials [G][P] in a fixed
// order (so the result does not depend on scheduling), optionally writes the
// gradient and optionally applies Adam with float64 moments; block 0 also
// finishes the loss (Eq. 4 / Eq. 8) from per-block float64 partials with a
// fixed-order pairwise float64 tree.
#include <algorithm>

#include "../../include/hrkan.h"
#include "internal.h"

namespace hrkan {

constexpr int RED_LANES = 32;   // parameters per block
constexpr int RED_WARPS = 16;   // partial rows split across warps


// Fixed-order pairwise float64 fold of rows [r0, r1) of the loss partials
// [row][2] by all threads of the block (blockDim = 32 x RED_WARPS).  The
// partials are sums of squares, all non-negative, so the pairwise tree (depth
// ~log2 of the row count) bounds the relative error by ~depth * 2^-53 without a
// compensation term, and keeps the float64 dependency chain short (float64
// latency dominates this step on GB300).  Thread (0,0) receives the totals.
__device__ __forceinline__ void fold_loss_rows(const double* lp, int r0, int r1, double& t0, double& t1) {
    __shared__ double sh[2][RED_WARPS];
    const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane, nt = 32 * RED_WARPS;
    double a = 0.0, b = 0.0;
    for (int g = r0 + tid; g < r1; g += nt) {
        a += lp[2 * int64_t(g)];
        b += lp[2 * int64_t(g) + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { sh[0][w] = a; sh[1][w] = b; }
    __syncthreads();
    if (w == 0) {
        a = lane < RED_WARPS ? sh[0][lane] : 0.0;
        b = lane < RED_WARPS ? sh[1][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
    t0 = a;
    t1 = b;
}

__global__ void __launch_bounds__(RED_LANES * RED_WARPS) reduce_kernel(ReduceParams p) {
    __shared__ float part[RED_WARPS][RED_LANES];
    __shared__ float corr[2];
    const int lane = threadIdx.x, w = threadIdx.y;
    const int64_t i = int64_t(blockIdx.x) * RED_LANES + lane;
    if (p.do_adam && w == 0 && lane == 0) {
        // bias corrections 1 - b^t (float64 pow once per block)
        double c1 = p.c1, c2 = p.c2;
        if (p.t_counter) {
            const int t = p.t_counter[1];
            c1 = 1.0 - pow(p.b1, double(t));
            c2 = 1.0 - pow(p.b2, double(t));
        }
        corr[0] = float(1.0 / c1);
        corr[1] = float(1.0 / sqrt(c2));
    }
    if (i < p.P) {
        float acc = 0.0f;
        // rows w, w + 16, ...: 4 independent loads in flight per step
        int g = w;
        for (; g + 3 * RED_WARPS < p.G; g += 4 * RED_WARPS) {
            float a0 = p.partial[int64_t(g) * p.P + i];
            float a1 = p.partial[int64_t(g + RED_WARPS) * p.P + i];
            float a2 = p.partial[int64_t(g + 2 * RED_WARPS) * p.P + i];
            float a3 = p.partial[int64_t(g + 3 * RED_WARPS) * p.P + i];
            acc += a0; acc += a1; acc += a2; acc += a3;
        }
        for (; g < p.G; g += RED_WARPS) acc += p.partial[int64_t(g) * p.P + i];
        part[w][lane] = acc;
    }
    __syncthreads();
    if (w == 0 && i < p.P) {
        float gsum = 0.0f;
#pragma unroll
        for (int t = 0; t < RED_WARPS; ++t) gsum += part[t][lane];
        if (p.dW) p.dW[i] = p.accumulate ? p.dW[i] + gsum : gsum;
        if (p.do_adam) {
            // float64 moments (fused multiply-adds only); the step itself in float32:
            // W <- W - lr * (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps)
            const double gd = gsum;
            const double m1 = fma(p.b1, p.m1[i], (1.0 - p.b1) * gd);
            const double m2 = fma(p.b2, p.m2[i], (1.0 - p.b2) * gd * gd);
            p.m1[i] = m1;
            p.m2[i] = m2;
            const float mh = float(m1) * corr[0];
            const float vh = sqrtf(float(m2)) * corr[1];
            p.W[i] = p.W[i] - float(p.lr) * mh / (vh + float(p.eps));
        }
    }
    // commit the step counter; this kernel reads only t_counter[1]
    if (p.t_counter && blockIdx.x == 0 && w == 0 && lane == 0) p.t_counter[0] = p.t_counter[1];
    if (blockIdx.x == 0 && p.loss_partial) {   // block-uniform: the fold synchronises the block
        double s0, s1;
        fold_loss_rows(p.loss_partial, 0, p.Gl, s0, s1);
        if (w == 0 && lane == 0) {
            const double lp = p.n0 > 0 ? s0 / double(p.n0) : 0.0;
            const double lb = p.n1 > 0 ? s1 / double(p.n1) : 0.0;
            p.loss[0] = p.alpha * lp + lb;
            p.loss[1] = lp;
            p.loss[2] = lb;
            // a non-finite loss (NaN or infinite inputs, a diverged run) is recorded for hrkan_sync_status
            if (p.status && !isfinite(p.alpha * lp + lb)) atomicCAS(p.status, 0, int(HRKAN_ENONFINITE));
        }
    }
}

cudaError_t launch_reduce(const ReduceParams& p, cudaStream_t s) {
    int64_t blocks = (p.P + RED_LANES - 1) / RED_LANES;
    if (blocks < 1) blocks = 1;
    reduce_kernel<<<dim3((unsigned)blocks), dim3(RED_LANES, RED_WARPS), 0, s>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- residual

constexpr int RES_BLOCK = 256;

template <unsigned MASK>
__global__ void __launch_bounds__(RES_BLOCK) residual_kernel(ResidualParams p) {
    using JT = Jet<MASK>;
    if (p.t_counter && blockIdx.x == 0 && threadIdx.x == 0) p.t_counter[1] = p.t_counter[0] + 1;
    double l0 = 0.0, l1 = 0.0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t pt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; pt < p.N; pt += stride) {
        float u[JT::J], gu[JT::J];
#pragma unroll
        for (int r = 0; r < JT::J; ++r) u[r] = p.jets[r * p.N + pt];
        float r = pde_residual<MASK>(p.pde, p.x[pt], p.x[p.N + pt], u);
        l0 += double(r) * double(r);
        if (p.dL) {
            pde_residual_grad<MASK>(p.pde, r, u, p.scale0, gu);
#pragma unroll
            for (int q = 0; q < JT::J; ++q) p.dL[q * p.N + pt] = gu[q];
        }
    }
    for (int64_t pt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; pt < p.Nb; pt += stride) {
        float d = p.u_bnd[pt] - p.g_bnd[pt];
        l1 += double(d) * double(d);
        if (p.dLb) p.dLb[pt] = p.scale1 * d;
    }
    __shared__ double red[2][RES_BLOCK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l0 += __shfl_down_sync(0xffffffffu, l0, o);
        l1 += __shfl_down_sync(0xffffffffu, l1, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = l0; red[1][threadIdx.x >> 5] = l1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int t = 0; t < RES_BLOCK / 32; ++t) { a += red[0][t]; b += red[1][t]; }
        p.loss_partial[2 * blockIdx.x] = a;
        p.loss_partial[2 * blockIdx.x + 1] = b;
    }
}

// Three coordinates, r = u_xx + u_yy + u_zz + (a^2 + b^2 + c^2) pi^2 sin(a pi x) sin(b pi y)
// sin(c pi z) (pde.src holds the factor, pde.lam holds c); dL/d(u_xx, u_yy, u_zz) = scale0 r,
// nothing for the lower rows.  Boundary misfit and the block's loss partials as residual_kernel.
__global__ void __launch_bounds__(RES_BLOCK) residual3_kernel(ResidualParams p) {
    if (p.t_counter && blockIdx.x == 0 && threadIdx.x == 0) p.t_counter[1] = p.t_counter[0] + 1;
    double l0 = 0.0, l1 = 0.0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x, N = p.N;
    for (int64_t pt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; pt < N; pt += stride) {
        const float f = p.pde.src * sinpif(p.pde.a * p.x[pt]) * sinpif(p.pde.b * p.x[N + pt]) *
                        sinpif(p.pde.lam * p.x[2 * N + pt]);
        const float r = p.jets[4 * N + pt] + p.jets[5 * N + pt] + p.jets[6 * N + pt] + f;
        l0 += double(r) * double(r);
        if (p.dL) {
#pragma unroll
            for (int q = 0; q < 4; ++q) p.dL[q * N + pt] = 0.0f;
#pragma unroll
            for (int q = 4; q < 7; ++q) p.dL[q * N + pt] = p.scale0 * r;
        }
    }
    for (int64_t pt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; pt < p.Nb; pt += stride) {
        float d = p.u_bnd[pt] - p.g_bnd[pt];
        l1 += double(d) * double(d);
        if (p.dLb) p.dLb[pt] = p.scale1 * d;
    }
    __shared__ double red[2][RES_BLOCK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l0 += __shfl_down_sync(0xffffffffu, l0, o);
        l1 += __shfl_down_sync(0xffffffffu, l1, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = l0; red[1][threadIdx.x >> 5] = l1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int t = 0; t < RES_BLOCK / 32; ++t) { a += red[0][t]; b += red[1][t]; }
        p.loss_partial[2 * blockIdx.x] = a;
        p.loss_partial[2 * blockIdx.x + 1] = b;
    }
}

cudaError_t launch_residual3(const ResidualParams& p, int grid, cudaStream_t s) {
    if (p.mask != 0x7Fu) return cudaErrorInvalidValue;
    residual3_kernel<<<grid, RES_BLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

bool residual_mask_supported(unsigned mask) { return mask == 0x0Fu || mask == 0x1Fu || mask == 0x2Fu; }

cudaError_t launch_residual(const ResidualParams& p, int grid, cudaStream_t s) {
    switch (p.mask) {
        case 0x0Fu: residual_kernel<0x0Fu><<<grid, RES_BLOCK, 0, s>>>(p); break;
        case 0x1Fu: residual_kernel<0x1Fu><<<grid, RES_BLOCK, 0, s>>>(p); break;
        case 0x2Fu: residual_kernel<0x2Fu><<<grid, RES_BLOCK, 0, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hrkan

// ------------------------------------------------------- many instances

namespace hrkan {

// grid (ceil(P / 512), n_inst): block (x, i) sums instance i's partial rows for
// 512 weights, one per thread, in a fixed order (per residue class of the row
// index mod 16, then the classes in order; an instance has a few to a few
// hundred rows), applies Adam, and block (0, i) finishes the instance's loss.
__global__ void __launch_bounds__(RED_LANES * RED_WARPS) batch_reduce_kernel(BatchReduceParams p) {
    __shared__ float corr[2];
    const int lane = threadIdx.x, w = threadIdx.y;
    const int inst = blockIdx.y;
    // one weight per thread, RED_LANES * RED_WARPS weights per block
    const int64_t k = int64_t(blockIdx.x) * (RED_LANES * RED_WARPS) + w * RED_LANES + lane;
    const int r0 = p.item_off[inst], r1 = p.item_off[inst + 1];
    if (w == 0 && lane == 0) {
        double c1 = p.c1, c2 = p.c2;
        if (p.t_counter) {
            const int t = p.t_counter[1];
            c1 = 1.0 - pow(p.b1, double(t));
            c2 = 1.0 - pow(p.b2, double(t));
        }
        corr[0] = float(1.0 / c1);
        corr[1] = float(1.0 / sqrt(c2));
    }
    __syncthreads();
    if (k < p.P) {
        // fixed order: a partial sum per residue class of the row index (mod RED_WARPS),
        // then the classes in order
        float gsum = 0.0f;
        for (int t = 0; t < RED_WARPS; ++t) {
            float acc = 0.0f;
            for (int g = r0 + t; g < r1; g += RED_WARPS) acc += p.partial[int64_t(g) * p.P + k];
            gsum += acc;
        }
        const int64_t i = int64_t(inst) * p.P + k;
        if (p.dW) p.dW[i] = gsum;
        const double gd = gsum;
        const double m1 = fma(p.b1, p.m1[i], (1.0 - p.b1) * gd);
        const double m2 = fma(p.b2, p.m2[i], (1.0 - p.b2) * gd * gd);
        p.m1[i] = m1;
        p.m2[i] = m2;
        const float mh = float(m1) * corr[0];
        const float vh = sqrtf(float(m2)) * corr[1];
        p.W[i] = p.W[i] - float(p.lr) * mh / (vh + float(p.eps));
    }
    if (p.t_counter && blockIdx.x == 0 && inst == 0 && w == 0 && lane == 0) p.t_counter[0] = p.t_counter[1];
    if (blockIdx.x == 0) {   // block-uniform
        double s0, s1;
        if (p.loss_off) fold_loss_rows(p.loss_partial, p.loss_off[inst], p.loss_off[inst + 1], s0, s1);
        else fold_loss_rows(p.loss_partial, r0, r1, s0, s1);
        if (w == 0 && lane == 0) {
            const double n0 = p.counts[2 * inst], n1 = p.counts[2 * inst + 1];
            const double lp = n0 > 0 ? s0 / n0 : 0.0;
            const double lb = n1 > 0 ? s1 / n1 : 0.0;
            p.loss[3 * inst] = p.alpha * lp + lb;
            p.loss[3 * inst + 1] = lp;
            p.loss[3 * inst + 2] = lb;
            if (p.status && !isfinite(p.alpha * lp + lb)) atomicCAS(p.status, 0, int(HRKAN_ENONFINITE));
        }
    }
}

cudaError_t launch_batch_reduce(const BatchReduceParams& p, cudaStream_t s) {
    int64_t bx = (p.P + RED_LANES * RED_WARPS - 1) / (RED_LANES * RED_WARPS);
    batch_reduce_kernel<<<dim3((unsigned)bx, (unsigned)p.n_inst), dim3(RED_LANES, RED_WARPS), 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace hrkan

namespace hrkan {
namespace {
// out[c] = sum over rows r (in order) of src[r * stride + c].
__global__ void sum_rows_kernel(const float* __restrict__ src, int rows, int64_t stride, int64_t cols,
                                float* __restrict__ out) {
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < cols; c += int64_t(gridDim.x) * blockDim.x) {
        float a = 0.0f;
        for (int r = 0; r < rows; ++r) a += src[int64_t(r) * stride + c];
        out[c] = a;
    }
}
}  // namespace

cudaError_t sum_rows(const float* src, int rows, int64_t stride, int64_t cols, float* out, cudaStream_t s) {
    if (cols <= 0) return cudaSuccess;
    const int grid = int(std::min<int64_t>((cols + 255) / 256, 4096));
    sum_rows_kernel<<<grid, 256, 0, s>>>(src, rows, stride, cols, out);
    return cudaGetLastError();
}
}  // namespace hrkan
