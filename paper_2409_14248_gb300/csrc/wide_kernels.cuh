// Layer-wise kernels for wide HRKANs (hidden widths up to 64, any number of
// layers): the KAN layer of Sections 1-3 with Eq. 2 bases, its input-jet
// forward, the input adjoint through v''' (v'''' for third-derivative rows) and
// the weight gradient.  Jet masks: 0x01, 0x0F, 0x1F (the PDE rows), 0x2F, 0x7F
// (with third derivatives), 0x87, 0xFF (with the mixed derivative u_x0x1),
// 0x12F (u, u_x, u_y, u_xx, u_xxx, u_xxxx) and 0x52F (and u_xxxxx): fourth and
// fifth derivatives along x_0 (Section 3 picks m = 6 for a fifth derivative).
//
// Jets live in HBM between layers as [J][units][N] float32 (one row per jet
// component and unit, points contiguous), so every per-point access of a warp
// is one coalesced 128-byte line.  Only the k+1 active bases of each unit are
// evaluated and contracted (Eq. 2 has compact support):
//   forward      y[r][o] = sum_j sum_q W[o][j][c_j+q] A_r[j][q]
//   adjoint      dA[j][r][q] = sum_o gy[r][o] W[o][j][c_j+q], then through v'''
//   weight grad  dW[o][j][c_j+q] += sum_r gy[r][o] A_r[j][q]  (summed over points)
#pragma once

#include <algorithm>

#include "internal.h"
#include "narrow.cuh"
#include "wide.cuh"

namespace hrkan {

constexpr int WB = 256;      // threads (= points) per block of the point-parallel kernels
constexpr int KW = 3;        // k
constexpr int KPW = KW + 1;
// The HR order m (Eq. 2) is the template parameter MW of every kernel below.

// Jets of input unit j of a layer: from the tape, or (first layer) the
// coordinate x_j itself with derivative 1 along the jet direction that
// differentiates along it (seed0 / seed1) and no other derivative.
template <unsigned MASK, bool FIRST>
__device__ __forceinline__ void load_unit_jets(const float* __restrict__ z, int I, int j, int64_t N, int64_t p,
                                               float* zj, int seed0 = 0, int seed1 = 1) {
    using JT = Jet<MASK>;
    if constexpr (FIRST) {
        zj[0] = z[j * N + p];
        if constexpr (JT::F0) zj[JT::RF0] = (j == seed0) ? 1.0f : 0.0f;
        if constexpr (JT::F1) zj[JT::RF1] = (j == seed1) ? 1.0f : 0.0f;
        if constexpr (JT::S0) zj[JT::RS0] = 0.0f;
        if constexpr (JT::S1) zj[JT::RS1] = 0.0f;
        if constexpr (JT::T0) zj[JT::RT0] = 0.0f;
        if constexpr (JT::T1) zj[JT::RT1] = 0.0f;
        if constexpr (JT::X01) zj[JT::RX] = 0.0f;
        if constexpr (JT::P0) zj[JT::RP0] = 0.0f;
        if constexpr (JT::P1) zj[JT::RP1] = 0.0f;
        if constexpr (JT::Q0) zj[JT::RQ0] = 0.0f;
        if constexpr (JT::Q1) zj[JT::RQ1] = 0.0f;
    } else {
#pragma unroll
        for (int r = 0; r < JT::J; ++r) zj[r] = z[(int64_t(r) * I + j) * N + p];
    }
}

// ------------------------------------------------------------------ forward
// grid (ceil(N / WB), ceil(O / OT)); the block's weights W[o0 .. o0+OT) sit in
// shared memory as [j][i][OT] so an active basis reads its OT outputs as float4.
template <int MW, unsigned MASK, int OT, bool FIRST>
__global__ void __launch_bounds__(WB) wide_fwd_kernel(WideLayer p) {
    using JT = Jet<MASK>;
    constexpr int J = JT::J;
    extern __shared__ __align__(16) float wt[];
    const int I = p.I, O = p.O, n = p.g.n;
    const int o0 = blockIdx.y * OT;
    const float* W = p.blk_inst ? p.W + int64_t(p.blk_inst[blockIdx.x]) * p.w_stride : p.W;
    for (int t = threadIdx.x; t < I * n * OT; t += blockDim.x) {
        const int oo = t % OT, ji = t / OT;
        wt[t] = (o0 + oo < O) ? W[int64_t(o0 + oo) * I * n + ji] : 0.0f;
    }
    __syncthreads();
    const int64_t N = p.N;
    const int64_t pt = int64_t(blockIdx.x) * WB + threadIdx.x;
    if (pt >= N) return;
    float acc[OT][J];
#pragma unroll
    for (int o = 0; o < OT; ++o)
#pragma unroll
        for (int r = 0; r < J; ++r) acc[o][r] = 0.0f;
#pragma unroll 1
    for (int j = 0; j < I; ++j) {
        float z[J];
        load_unit_jets<MASK, FIRST>(p.z, I, j, N, pt, z, p.seed0, p.seed1);
        Active<KW, MW, JT::NDER_ROWS> b;
        b.eval(z[0], p.g);
        float a[J][KPW];
        JT::template rows_b<KPW>(z, b, a);
#pragma unroll
        for (int q = 0; q < KPW; ++q) {
            const float* wr = wt + (j * n + b.idx(q, n)) * OT;
            if constexpr (OT % 4 == 0) {
#pragma unroll
                for (int o4 = 0; o4 < OT / 4; ++o4) {
                    const float4 w4 = reinterpret_cast<const float4*>(wr)[o4];
                    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
#pragma unroll
                        for (int r = 0; r < J; ++r) acc[o4 * 4 + e][r] = fmaf(wv[e], a[r][q], acc[o4 * 4 + e][r]);
                }
            } else {
#pragma unroll
                for (int o = 0; o < OT; ++o)
#pragma unroll
                    for (int r = 0; r < J; ++r) acc[o][r] = fmaf(wr[o], a[r][q], acc[o][r]);
            }
        }
    }
#pragma unroll
    for (int o = 0; o < OT; ++o)
        if (o0 + o < O)
#pragma unroll
            for (int r = 0; r < J; ++r) p.y[(int64_t(r) * O + o0 + o) * N + pt] = acc[o][r];
}

// ------------------------------------------------------------ input adjoint
// grid (ceil(I / IT), point blocks): the input-chunk index runs fastest so the
// blocks sharing a point tile run together and reuse its gy lines from L2.  A
// grid's y extent is at most 65535, so a launch covers at most 65535 * WB
// points starting at p.p0 and larger sets take several launches.
// Shared memory holds W[all o][chunk][all i] as [jj][o][i] (basis fastest:
// lanes with different cells hit different banks).
template <int MW, unsigned MASK, int IT>
__global__ void __launch_bounds__(WB) wide_adjoint_kernel(WideLayer p) {
    using JT = Jet<MASK>;
    constexpr int J = JT::J;
    extern __shared__ __align__(16) float ws[];
    const int I = p.I, O = p.O, n = p.g.n;
    const int j0 = blockIdx.x * IT;
    const float* W = p.blk_inst ? p.W + int64_t(p.blk_inst[p.p0 / WB + blockIdx.y]) * p.w_stride : p.W;
    for (int t = threadIdx.x; t < IT * O * n; t += blockDim.x) {
        const int i = t % n, rest = t / n, o = rest % O, jj = rest / O;
        ws[t] = (j0 + jj < I) ? W[(int64_t(o) * I + j0 + jj) * n + i] : 0.0f;
    }
    __syncthreads();
    const int64_t N = p.N;
    const int64_t pt = p.p0 + int64_t(blockIdx.y) * WB + threadIdx.x;
    if (pt >= N) return;
    float z[IT][J];
    int cb[IT];
#pragma unroll
    for (int jj = 0; jj < IT; ++jj) {
        const int j = (j0 + jj < I) ? j0 + jj : I - 1;
        load_unit_jets<MASK, false>(p.z, I, j, N, pt, z[jj]);
        Active<KW, MW, 2> b;
        b.eval(z[jj][0], p.g);
        cb[jj] = b.c;
    }
    float dA[IT][J][KPW];
#pragma unroll
    for (int jj = 0; jj < IT; ++jj)
#pragma unroll
        for (int r = 0; r < J; ++r)
#pragma unroll
            for (int q = 0; q < KPW; ++q) dA[jj][r][q] = 0.0f;
    // gy of output o + GPF is loaded while output o is contracted (hides the load latency)
    constexpr int GPF = 4;
    float gq[GPF][J];
#pragma unroll
    for (int u = 0; u < GPF; ++u)
#pragma unroll
        for (int r = 0; r < J; ++r) gq[u][r] = u < O ? p.gy[(int64_t(r) * O + u) * N + pt] : 0.0f;
#pragma unroll 1
    for (int ob = 0; ob < O; ob += GPF) {
#pragma unroll
      for (int u = 0; u < GPF; ++u) {
        const int o = ob + u;
        if (o >= O) break;
        float g[J];
#pragma unroll
        for (int r = 0; r < J; ++r) g[r] = gq[u][r];
        if (o + GPF < O) {
#pragma unroll
            for (int r = 0; r < J; ++r) gq[u][r] = p.gy[(int64_t(r) * O + o + GPF) * N + pt];
        }
#pragma unroll
        for (int jj = 0; jj < IT; ++jj) {
            const float* wr = ws + (jj * O + o) * n;
#pragma unroll
            for (int q = 0; q < KPW; ++q) {
                int i = cb[jj] + q;
                i = i < 0 ? 0 : (i >= n ? n - 1 : i);
                const float w = wr[i];
#pragma unroll
                for (int r = 0; r < J; ++r) dA[jj][r][q] = fmaf(g[r], w, dA[jj][r][q]);
            }
        }
      }
    }
#pragma unroll
    for (int jj = 0; jj < IT; ++jj) {
        if (j0 + jj >= I) break;
        Active<KW, MW, JT::NDER_ADJ> b;
        b.eval(z[jj][0], p.g);
        // bases that do not exist contribute nothing (their dA used a clamped weight)
        float gz[J];
        JT::template adjoint_b<KPW>(z[jj], b, dA[jj], gz);
#pragma unroll
        for (int r = 0; r < J; ++r) p.gz[(int64_t(r) * I + j0 + jj) * N + pt] = gz[r];
    }
}

// ------------------------------------------------------------ weight gradient
// grid NJC x GP (chunk fastest).  Block (jc, gp) owns the gradient of input
// units [jc*JC, +JC) and walks point tiles gp, gp + GP, ... : it stages the
// tile's gy [PB][J][O] and basis rows [PB][JC][J][4] (+ cells) in shared
// memory, then each thread exclusively owns whole (unit, output) rows of the
// gradient (with fewer rows than threads, a copy of a row and every S-th point),
// so the accumulation needs no atomics and is deterministic.  At the end the
// block writes its rows into partial row gp (columns of its units).
template <int MW, unsigned MASK, int JC, int PB, bool FIRST>
__global__ void __launch_bounds__(WB) wide_dw_kernel(WideDw p) {
    using JT = Jet<MASK>;
    constexpr int J = JT::J;
    extern __shared__ __align__(16) float sm[];
    const int I = p.I, O = p.O, n = p.g.n;
    const int NP = n | 1;                       // odd row stride: lanes with consecutive o hit distinct banks
    const int njc = (I + JC - 1) / JC;
    const int jc = blockIdx.x % njc, gp = blockIdx.x / njc;
    const int j0 = jc * JC;
    const int nj = min(JC, I - j0);
    // outputs [o0, o0 + Ob) of this block (blockIdx.y slices the outputs when the
    // unit chunks alone give too few blocks, e.g. the 2-input first layer)
    const int OS = (O + gridDim.y - 1) / gridDim.y;
    const int o0 = blockIdx.y * OS, Ob = min(OS, O - o0);
    // R owned rows; with fewer rows than threads, S threads share a row, each
    // accumulating every S-th point of a tile into its own copy (summed at the end)
    const int R = nj * Ob, S = max(1, int(blockDim.x) / max(R, 1));
    const int cap = max(JC * O, WB);                  // rows of gradient storage
    const int sz_dw = (cap * NP + 3) & ~3, sz_gy = (PB * J * O + 3) & ~3;
    float* dws = sm;                                  // [S][R][NP]
    float* gys = dws + sz_dw;                         // [PB][J][O]
    float* as = gys + sz_gy;                          // [PB][JC][J][4] (16-byte aligned)
    int* cs = reinterpret_cast<int*>(as + PB * JC * J * KPW);   // [PB][JC]
    for (int t = threadIdx.x; t < S * R * NP; t += blockDim.x) dws[t] = 0.0f;
    const int64_t N = p.N;
    const int64_t tiles = (N + PB - 1) / PB;
    // the tiles of this block's chunk (batched path), else every GP-th tile
    const int64_t t_first = p.chunks ? int64_t(p.chunks[gp].x) / PB : gp;
    const int64_t t_end = p.chunks ? std::min<int64_t>((int64_t(p.chunks[gp].y) + PB - 1) / PB, tiles) : tiles;
    const int64_t t_step = p.chunks ? 1 : p.GP;
    for (int64_t tile = t_first; tile < t_end; tile += t_step) {
        const int64_t base = tile * PB;
        __syncthreads();
        // stage gy: element (pp, r, o) = gy[r][o][base + pp]
        for (int t = threadIdx.x; t < PB * J * Ob; t += blockDim.x) {
            const int pp = t % PB, ro = t / PB;   // ro = r * Ob + o
            const int r = ro / Ob, o = ro % Ob;
            const int64_t pt = base + pp;
            gys[pp * J * Ob + ro] = (pt < N) ? p.gy[(int64_t(r) * O + o0 + o) * N + pt] : 0.0f;
        }
        // stage basis rows of the chunk's units
        for (int t = threadIdx.x; t < PB * JC; t += blockDim.x) {
            const int pp = t % PB, jj = t / PB;
            const int64_t pt = base + pp;
            int c = -(1 << 20);   // no basis: all four slots out of range
            float a[J][KPW];
            if (pt < N && jj < nj) {
                float z[J];
                load_unit_jets<MASK, FIRST>(p.z, I, j0 + jj, N, pt, z, p.seed0, p.seed1);
                Active<KW, MW, JT::NDER_ROWS> b;
                b.eval(z[0], p.g);
                JT::template rows_b<KPW>(z, b, a);
                c = b.c;
            } else {
#pragma unroll
                for (int r = 0; r < J; ++r)
#pragma unroll
                    for (int q = 0; q < KPW; ++q) a[r][q] = 0.0f;
            }
            float* dst = as + (pp * JC + jj) * J * KPW;
#pragma unroll
            for (int r = 0; r < J; ++r)
                reinterpret_cast<float4*>(dst)[r] = make_float4(a[r][0], a[r][1], a[r][2], a[r][3]);
            cs[pp * JC + jj] = c;
        }
        __syncthreads();
        // owners: row (jj, o) of the gradient, copy `sub`
        for (int k = threadIdx.x; k < R * S; k += blockDim.x) {
            const int rk = k % R, sub = k / R;
            const int o = rk % Ob, jj = rk / Ob;
            float* row = dws + (sub * R + rk) * NP;
#pragma unroll 4
            for (int pp = sub; pp < PB; pp += S) {
                const int c = cs[pp * JC + jj];
                const float* ar = as + (pp * JC + jj) * J * KPW;
                const float* gr = gys + pp * J * Ob + o;
                float gq[KPW] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int r = 0; r < J; ++r) {
                    const float gv = gr[r * Ob];
                    const float4 a4 = reinterpret_cast<const float4*>(ar)[r];
                    gq[0] = fmaf(gv, a4.x, gq[0]);
                    gq[1] = fmaf(gv, a4.y, gq[1]);
                    gq[2] = fmaf(gv, a4.z, gq[2]);
                    gq[3] = fmaf(gv, a4.w, gq[3]);
                }
#pragma unroll
                for (int q = 0; q < KPW; ++q)
                    if ((unsigned)(c + q) < (unsigned)n) row[c + q] += gq[q];
            }
        }
    }
    __syncthreads();
    float* out = p.partial + int64_t(p.chunks ? p.chunks[gp].z : p.row0 + gp) * p.P + p.col0;
    for (int t = threadIdx.x; t < nj * Ob * n; t += blockDim.x) {
        const int i = t % n, rest = t / n, o = rest % Ob, jj = rest / Ob;
        float v = 0.0f;
        for (int sub = 0; sub < S; ++sub) v += dws[(sub * R + jj * Ob + o) * NP + i];   // fixed order
        out[(int64_t(o0 + o) * I + j0 + jj) * n + i] = v;
    }
}

// ------------------------------------------------------------------ launch

inline cudaError_t smem_optin(const void* kern, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

template <int MW, unsigned MASK>
static cudaError_t fwd_mask(const WideLayer& p, bool first, cudaStream_t s) {
    const int n = p.g.n;
    const unsigned gx = unsigned((p.N + WB - 1) / WB);
    auto go = [&](auto kern, int ot) -> cudaError_t {
        const size_t sm = size_t(p.I) * n * ot * sizeof(float);
        cudaError_t e = smem_optin((const void*)kern, sm);
        if (e != cudaSuccess) return e;
        kern<<<dim3(gx, unsigned((p.O + ot - 1) / ot)), WB, sm, s>>>(p);
        return cudaGetLastError();
    };
    if (p.O == 1) return first ? go(wide_fwd_kernel<MW, MASK, 1, true>, 1) : go(wide_fwd_kernel<MW, MASK, 1, false>, 1);
    // eight outputs per block: fewer accumulators and more resident warps pay
    // for evaluating a point's bases once per eight outputs (measured: the
    // batching workload's 2 -> 16 layer 0.47 ms per step against 0.68 with 16
    // outputs per block and 0.56 with 4; its 16 -> 16 layer ~2.0 against ~3.0;
    // the FP32 step of [2,64,64,64,1] 39.1 ms against 42.2)
    return first ? go(wide_fwd_kernel<MW, MASK, 8, true>, 8) : go(wide_fwd_kernel<MW, MASK, 8, false>, 8);
}

template <int MW, unsigned MASK>
static cudaError_t adj_mask(const WideLayer& p, cudaStream_t s) {
    constexpr int IT = 2;   // measured best of 2 / 4 / 8 (registers vs gy reuse)
    const size_t sm = size_t(IT) * p.O * p.g.n * sizeof(float);
    auto kern = wide_adjoint_kernel<MW, MASK, IT>;
    cudaError_t e = smem_optin((const void*)kern, sm);
    if (e != cudaSuccess) return e;
    constexpr int64_t kMaxBlocksY = 65535;
    const int64_t blocks = (p.N + WB - 1) / WB;
    for (int64_t b0 = 0; b0 < blocks; b0 += kMaxBlocksY) {
        WideLayer q = p;
        q.p0 = b0 * WB;
        const unsigned by = unsigned(std::min<int64_t>(kMaxBlocksY, blocks - b0));
        kern<<<dim3(unsigned((p.I + IT - 1) / IT), by), WB, sm, s>>>(q);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <unsigned MASK, int JC, int PB, bool FIRST>
static size_t dw_smem(int O, int n) {
    constexpr int J = Jet<MASK>::J;
    return sizeof(float) * (((std::max<size_t>(size_t(JC) * O, WB) * (n | 1) + 3) & ~size_t(3)) +
                            ((size_t(PB) * J * O + 3) & ~size_t(3)) +
                            size_t(PB) * JC * J * KPW) +
           sizeof(int) * size_t(PB) * JC;
}

template <int MW, unsigned MASK>
static cudaError_t dw_mask(const WideDw& p, bool first, cudaStream_t s) {
    constexpr int PB = 32;
    auto go = [&](auto kern, int jc, size_t sm) -> cudaError_t {
        cudaError_t e = smem_optin((const void*)kern, sm);
        if (e != cudaSuccess) return e;
        const int njc = (p.I + jc - 1) / jc;
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        // slice the outputs until there are about two blocks per SM (at least 8 outputs a slice)
        const int want = (2 * nsm + njc * p.GP - 1) / (njc * p.GP);
        const int nos = std::max(1, std::min(want, p.O / 8));
        kern<<<dim3(unsigned(njc * p.GP), unsigned(nos)), WB, sm, s>>>(p);
        return cudaGetLastError();
    };
    if (first) return go(wide_dw_kernel<MW, MASK, 2, PB, true>, 2, dw_smem<MASK, 2, PB, true>(p.O, p.g.n));
    return go(wide_dw_kernel<MW, MASK, 8, PB, false>, 8, dw_smem<MASK, 8, PB, false>(p.O, p.g.n));
}

template <int MW>
cudaError_t wide_forward_layer_m(const WideLayer& p, unsigned mask, bool first, cudaStream_t s) {
    if (p.N == 0) return cudaSuccess;
    switch (mask) {
        case 0x01u: return fwd_mask<MW, 0x01u>(p, first, s);
        case 0x0Fu: return fwd_mask<MW, 0x0Fu>(p, first, s);
        case 0x1Fu: return fwd_mask<MW, 0x1Fu>(p, first, s);
        case 0x2Fu: return fwd_mask<MW, 0x2Fu>(p, first, s);
        case 0x7Fu: return fwd_mask<MW, 0x7Fu>(p, first, s);
        case 0x87u: return fwd_mask<MW, 0x87u>(p, first, s);
        case 0xFFu: return fwd_mask<MW, 0xFFu>(p, first, s);
        case 0x12Fu: return fwd_mask<MW, 0x12Fu>(p, first, s);
        case 0x52Fu: return fwd_mask<MW, 0x52Fu>(p, first, s);
    }
    return cudaErrorNotSupported;
}

template <int MW>
cudaError_t wide_adjoint_layer_m(const WideLayer& p, unsigned mask, cudaStream_t s) {
    if (p.N == 0) return cudaSuccess;
    switch (mask) {
        case 0x01u: return adj_mask<MW, 0x01u>(p, s);
        case 0x0Fu: return adj_mask<MW, 0x0Fu>(p, s);
        case 0x1Fu: return adj_mask<MW, 0x1Fu>(p, s);
        case 0x2Fu: return adj_mask<MW, 0x2Fu>(p, s);
        case 0x7Fu: return adj_mask<MW, 0x7Fu>(p, s);
        case 0x87u: return adj_mask<MW, 0x87u>(p, s);
        case 0xFFu: return adj_mask<MW, 0xFFu>(p, s);
        case 0x12Fu: return adj_mask<MW, 0x12Fu>(p, s);
        case 0x52Fu: return adj_mask<MW, 0x52Fu>(p, s);
    }
    return cudaErrorNotSupported;
}

template <int MW>
cudaError_t wide_dw_layer_m(const WideDw& p, unsigned mask, bool first, cudaStream_t s) {
    switch (mask) {
        case 0x01u: return dw_mask<MW, 0x01u>(p, first, s);
        case 0x0Fu: return dw_mask<MW, 0x0Fu>(p, first, s);
        case 0x1Fu: return dw_mask<MW, 0x1Fu>(p, first, s);
        case 0x2Fu: return dw_mask<MW, 0x2Fu>(p, first, s);
        case 0x7Fu: return dw_mask<MW, 0x7Fu>(p, first, s);
        case 0x87u: return dw_mask<MW, 0x87u>(p, first, s);
        case 0xFFu: return dw_mask<MW, 0xFFu>(p, first, s);
        case 0x12Fu: return dw_mask<MW, 0x12Fu>(p, first, s);
        case 0x52Fu: return dw_mask<MW, 0x52Fu>(p, first, s);
    }
    return cudaErrorNotSupported;
}

}  // namespace hrkan
