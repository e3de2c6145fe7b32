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

#include <cuda_bf16.h>

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

// ------------------------------------------------------------------ output layer
// The last layer (O = 1) of every instance, its residual and its reverse in
// one pass per point block: forward u jets from the layer's input jets z
// (the tape), the residual (interior set) or the boundary misfit, the loss
// partial of the block, then per input unit the input adjoint gz (written)
// and the weight-gradient contributions.  Those are summed without atomics:
// within a warp, lanes whose unit value falls in the same grid cell share the
// four weight addresses, so the warp walks its distinct cells in lane order,
// sums each cell's lanes with a butterfly and lets one lane add the sums into
// the warp's own copy of the layer's gradient; the copies are summed in a
// fixed order at the end (deterministic).  One block per weight-gradient
// chunk of one instance (partial row chunks[c].z, the layer's columns).
namespace hrkan {
namespace {

constexpr int TAIL_WARPS = LB_BLOCK / 32;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sum of NV values per lane (NV = 16 or 32) by recursive halving: at
// each level the lanes whose mask bit is set keep the upper half of their
// values and send the lower half to their partner (and the other way round),
// so NV - 1 shuffles leave every lane with the full sum of one index (its
// `idx`); for NV = 16 the lane pairs (l, l ^ 1) hold the same index.  The
// order of the additions is fixed.
template <int NV>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NV], int lane, int& idx) {
    static_assert(NV == 16 || NV == 32, "16 or 32 values");
    int off = 0;
#pragma unroll
    for (int lvl = 0; (NV >> (lvl + 1)) >= 1; ++lvl) {
        const int h = NV >> (lvl + 1), m = 16 >> lvl;
        const bool hi = (lane & m) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const float send = hi ? v[k] : v[k + h];
            const float keep = hi ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
        if (hi) off += h;
    }
    if constexpr (NV == 16) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    idx = off;
    return v[0];
}

template <int MW, unsigned MASK, bool BND, int NV>
__global__ void __launch_bounds__(LB_BLOCK) lb_tail_kernel(LbTailParams p) {
    using JT = Jet<MASK>;
    constexpr int J = JT::J, KP = 4;
    extern __shared__ __align__(16) float sm[];
    const int I = p.I, n = p.g.n, In = I * n;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 ch = p.chunks[blockIdx.x];
    const int inst = ch.w;
    float* w = sm;                       // [I][n] the instance's output-layer weights
    float* dws = sm + ((In + 3) & ~3);   // [TAIL_WARPS][I][n]
    const float* Wi = p.W + int64_t(inst) * p.w_stride;
    for (int t = tid; t < In; t += LB_BLOCK) w[t] = Wi[t];
    for (int t = tid; t < TAIL_WARPS * In; t += LB_BLOCK) dws[t] = 0.0f;
    if (p.t_counter && blockIdx.x == 0 && tid == 0) p.t_counter[1] = p.t_counter[0] + 1;
    __syncthreads();
    float* dwm = dws + warp * In;
    const BatchInst bi = p.inst[inst];
    PdeParams pde = p.pde;
    pde.a = bi.a;
    pde.b = bi.b;
    pde.src = bi.src;
    const int64_t N = p.N;
    for (int64_t b0 = ch.x; b0 < ch.y; b0 += LB_BLOCK) {
        const int blk = int(b0 / LB_BLOCK);
        const int64_t pt = b0 + tid;
        const bool valid = tid < p.blk_valid[blk];
        // forward: u jets
        float u[J];
#pragma unroll
        for (int r = 0; r < J; ++r) u[r] = 0.0f;
        // the next unit's jets are loaded while this one is evaluated
        float zn[J];
#pragma unroll
        for (int r = 0; r < J; ++r) zn[r] = p.z[int64_t(r) * I * N + pt];
#pragma unroll 1
        for (int j = 0; j < I; ++j) {
            float z[J];
#pragma unroll
            for (int r = 0; r < J; ++r) z[r] = zn[r];
            if (j + 1 < I) {
#pragma unroll
                for (int r = 0; r < J; ++r) zn[r] = p.z[(int64_t(r) * I + j + 1) * N + pt];
            }
            Active<3, MW, JT::NDER_ROWS> b;
            b.eval(z[0], p.g);
            float a[J][KP];
            JT::template rows_b<KP>(z, b, a);
#pragma unroll
            for (int q = 0; q < KP; ++q) {
                const float wq = w[j * n + b.idx(q, n)];
#pragma unroll
                for (int r = 0; r < J; ++r) u[r] = fmaf(wq, a[r][q], u[r]);
            }
        }
        // residual / boundary misfit and dL/du
        float gu[J];
        double l = 0.0;
        if constexpr (BND) {
            const float d = u[0] - p.g_bnd[pt];
            if (valid) l = double(d) * double(d);
            gu[0] = valid ? bi.scale1 * d : 0.0f;
        } else {
            const float rr = pde_residual<MASK>(pde, p.x[pt], p.x[N + pt], u);
            if (valid) {
                l = double(rr) * double(rr);
                pde_residual_grad<MASK>(pde, rr, u, bi.scale0, gu);
            } else {
#pragma unroll
                for (int q = 0; q < J; ++q) gu[q] = 0.0f;
            }
        }
        {
            __shared__ double red[TAIL_WARPS];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
            if (lane == 0) red[warp] = l;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int t = 0; t < TAIL_WARPS; ++t) s += red[t];   // fixed order
                const int row = p.lrow[blk];
                p.loss_partial[2 * int64_t(row) + (BND ? 1 : 0)] = s;
                p.loss_partial[2 * int64_t(row) + (BND ? 0 : 1)] = 0.0;
            }
            __syncthreads();
        }
        // reverse: input adjoint and weight gradient, unit by unit
#pragma unroll
        for (int r = 0; r < J; ++r) zn[r] = p.z[int64_t(r) * I * N + pt];
#pragma unroll 1
        for (int j = 0; j < I; ++j) {
            float z[J];
#pragma unroll
            for (int r = 0; r < J; ++r) z[r] = zn[r];
            if (j + 1 < I) {
#pragma unroll
                for (int r = 0; r < J; ++r) zn[r] = p.z[(int64_t(r) * I + j + 1) * N + pt];
            }
            Active<3, MW, JT::NDER_ADJ> b;
            b.eval(z[0], p.g);
            float a[J][KP], dA[J][KP], gw[KP];
            JT::template rows_b<KP>(z, b, a);
#pragma unroll
            for (int q = 0; q < KP; ++q) {
                const float wq = w[j * n + b.idx(q, n)];
                float s = 0.0f;
#pragma unroll
                for (int r = 0; r < J; ++r) {
                    s = fmaf(gu[r], a[r][q], s);
                    dA[r][q] = gu[r] * wq;
                }
                gw[q] = s;
            }
            float gz[J];
            JT::template adjoint_b<KP>(z, b, dA, gz);
            if (p.gz_bf) {   // the BF16 operand layout of the layer below's tensor-core kernels
#pragma unroll
                for (int r = 0; r < J; ++r)
                    p.gz_bf[(int64_t(r) * I + j) * N + pt] = __bfloat16_as_ushort(__float2bfloat16_rn(gz[r]));
            } else {
#pragma unroll
                for (int r = 0; r < J; ++r) p.gz[(int64_t(r) * I + j) * N + pt] = gz[r];
            }
            const int c = b.c;
            if constexpr (NV > 0) {
                // n <= NV: every lane spreads its window over NV slots (slot i holds
                // gw[i - c] for c <= i < c + 4), one reduce-scatter sums all slots
                float g_rot[KP];
                const int rot = c & 3;   // c mod 4, also for c < 0
#pragma unroll
                for (int r = 0; r < KP; ++r) {
                    const int q = (r - rot) & 3;
                    g_rot[r] = q == 0 ? gw[0] : q == 1 ? gw[1] : q == 2 ? gw[2] : gw[3];
                }
                float v[NV];
#pragma unroll
                for (int i = 0; i < NV; ++i) v[i] = unsigned(i - c) < 4u ? g_rot[i & 3] : 0.0f;
                int idx;
                const float sum = warp_reduce_scatter<NV>(v, lane, idx);
                if ((NV == 32 || (lane & 1) == 0) && idx < n) dwm[j * n + idx] += sum;
            } else {
                // the warp's distinct cells in lane order, one butterfly sum per cell and basis
                unsigned todo = 0xffffffffu;
                while (todo) {
                    const int leader = __ffs(todo) - 1;
                    const int cl = __shfl_sync(0xffffffffu, c, leader);
                    const bool in = c == cl;
                    const unsigned m = __ballot_sync(0xffffffffu, in);
#pragma unroll
                    for (int q = 0; q < KP; ++q) {
                        const float v = warp_sum(in ? gw[q] : 0.0f);
                        const int i = cl + q;
                        if (lane == 0 && unsigned(i) < unsigned(n)) dwm[j * n + i] += v;
                    }
                    todo &= ~m;
                }
            }
        }
    }
    __syncthreads();
    float* out = p.partial + int64_t(ch.z) * p.P + p.col0;
    for (int t = tid; t < In; t += LB_BLOCK) {
        float s = 0.0f;
        for (int k = 0; k < TAIL_WARPS; ++k) s += dws[k * In + t];   // fixed order
        out[t] = s;
    }
}

template <int MW, int NV, class Go>
cudaError_t tail_mask(Go& go, unsigned mask, bool bnd) {
    if (bnd) return go(lb_tail_kernel<MW, 0x01u, true, NV>);
    switch (mask) {
        case 0x0Fu: return go(lb_tail_kernel<MW, 0x0Fu, false, NV>);
        case 0x1Fu: return go(lb_tail_kernel<MW, 0x1Fu, false, NV>);
        case 0x2Fu: return go(lb_tail_kernel<MW, 0x2Fu, false, NV>);
    }
    return cudaErrorNotSupported;
}

template <int MW>
cudaError_t tail_m(const LbTailParams& p, unsigned mask, bool bnd, int nchunk, cudaStream_t s) {
    const size_t smem = sizeof(float) * (((size_t(p.I) * p.g.n + 3) & ~size_t(3)) + size_t(TAIL_WARPS) * p.I * p.g.n);
    auto go = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (e != cudaSuccess) { cudaGetLastError(); return e; }
        }
        kern<<<nchunk, LB_BLOCK, smem, s>>>(p);
        return cudaGetLastError();
    };
    // the weight-gradient sum: a reduce-scatter over 16 or 32 slots when the
    // layer's n bases fit, else the walk over the warp's distinct cells
    const int n = p.g.n;
    if (n <= 16) return tail_mask<MW, 16>(go, mask, bnd);
    if (n <= 32) return tail_mask<MW, 32>(go, mask, bnd);
    return tail_mask<MW, 0>(go, mask, bnd);
}

}  // namespace

cudaError_t lb_tail(const LbTailParams& p, unsigned mask, bool bnd, int nchunk, cudaStream_t s) {
    if (nchunk == 0) return cudaSuccess;
    switch (p.g.m) {
        case 2: return tail_m<2>(p, mask, bnd, nchunk, s);
        case 3: return tail_m<3>(p, mask, bnd, nchunk, s);
        case 4: return tail_m<4>(p, mask, bnd, nchunk, s);
        case 5: return tail_m<5>(p, mask, bnd, nchunk, s);
        case 6: return tail_m<6>(p, mask, bnd, nchunk, s);
    }
    return cudaErrorNotSupported;
}

}  // namespace hrkan
