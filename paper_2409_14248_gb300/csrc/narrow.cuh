// Fused whole-network kernels for narrow HRKANs: widths [2, WH, 1] (NL = 2)
// or [2, WH, WH, 1] (NL = 3) with WH <= 16.
//
// One thread owns one collocation point for the whole network: the forward
// jets (Section 3 bases through the KAN layer matrix operation), the PDE
// residual (Eq. 3-4 / Eq. 6-8) and the backward all stay in registers; only
// the k+1 active bases of each unit are evaluated (the others are exactly
// zero, Eq. 2 has compact support).  The weights of all layers (<= 16 KB) sit
// in shared memory, the hidden layer transposed to [j][i][o] so that one
// active basis reads its WH output weights as float4 vectors.  The weight
// gradient accumulates in shared memory and leaves the block once, as a
// per-block partial that a second kernel sums in a fixed order.
//
// Storage per thread: the hidden->hidden layer input jets z1 are never kept;
// both passes recompute a unit of z1 from the coordinate bases right before
// using it, so the register footprint is the last hidden layer's jets plus
// the coordinate bases.
#pragma once

#include "hr_device.cuh"

namespace hrkan {

enum { MODE_FWD = 0, MODE_BWD = 1, MODE_TRAIN = 2 };

constexpr int NARROW_BLOCK = 128;

template <int NL_, int WH_, int K_, int M_>
struct NarrowNet {
    static constexpr int NL = NL_, WH = WH_, K = K_, M = M_, KP = K_ + 1;
    static constexpr int WHP = (WH_ + 3) & ~3;   // padded row of the transposed hidden layer
    // Copies of the shared weight gradient, one per group of lanes (lane % COPIES).
    // Hidden activations of a PINN often sit in one or two grid cells, so the
    // lanes of a warp would otherwise add into the same address at once.
    static constexpr int COPIES = 4;
    // resident blocks per SM the register budget is sized for
    static constexpr int MINB = WH_ >= 16 ? 3 : 4;
    static_assert(NL == 2 || NL == 3, "narrow nets have one or two hidden layers");

    // shared-memory layout in floats (n = number of bases)
    __host__ __device__ static int off_w0() { return 0; }                       // [WH][2][n]
    __host__ __device__ static int off_w1(int n) { return 2 * WH * n; }         // [WH][n][WHP] (NL == 3)
    __host__ __device__ static int off_wl(int n) {                              // [WH][n]
        return 2 * WH * n + (NL == 3 ? WH * n * WHP : 0);
    }
    __host__ __device__ static int smem_floats(int n) { return (off_wl(n) + WH * n + 3) & ~3; }
};

// Global W (natural [o][j][i] per layer, concatenated) -> shared layout.
template <class Net>
__device__ void narrow_load_w(const float* __restrict__ W, float* s, int n) {
    constexpr int WH = Net::WH, WHP = Net::WHP;
    const int p0 = 2 * WH * n;
    for (int t = threadIdx.x; t < p0; t += blockDim.x) s[t] = W[t];
    int off = p0;
    if constexpr (Net::NL == 3) {
        const int p1 = WH * WH * n;
        float* w1 = s + Net::off_w1(n);
        for (int t = threadIdx.x; t < p1; t += blockDim.x) {
            int o = t / (WH * n), rem = t - o * WH * n;   // rem = j*n + i
            w1[rem * WHP + o] = W[off + t];
        }
        for (int t = threadIdx.x; t < WH * n; t += blockDim.x)   // zero the padding columns
            for (int o = WH; o < WHP; ++o) w1[t * WHP + o] = 0.0f;
        off += p1;
    }
    float* wl = s + Net::off_wl(n);
    for (int t = threadIdx.x; t < WH * n; t += blockDim.x) wl[t] = W[off + t];
}

// Shared dW (same layout) -> global partial row (natural layout).
template <class Net>
__device__ void narrow_store_dw(const float* s, float* __restrict__ out, int n) {
    constexpr int WH = Net::WH, WHP = Net::WHP;
    const int p0 = 2 * WH * n;
    for (int t = threadIdx.x; t < p0; t += blockDim.x) out[t] = s[t];
    int off = p0;
    if constexpr (Net::NL == 3) {
        const int p1 = WH * WH * n;
        const float* w1 = s + Net::off_w1(n);
        for (int t = threadIdx.x; t < p1; t += blockDim.x) {
            int o = t / (WH * n), rem = t - o * WH * n;
            out[off + t] = w1[rem * WHP + o];
        }
        off += p1;
    }
    const float* wl = s + Net::off_wl(n);
    for (int t = threadIdx.x; t < WH * n; t += blockDim.x) out[off + t] = wl[t];
}

// The shared weight gradient holds Net::COPIES interleaved copies of the
// layout above: logical element e of copy c lives at base[e * COPIES + c],
// and a lane adds into copy lane % COPIES.
template <class Net>
struct DwAcc {
    float* base;
    int cp;
    __device__ __forceinline__ void add(int e, float v) const { atomicAdd(base + e * Net::COPIES + cp, v); }
};

// Coordinate bases of one point (first layer inputs).
template <class Net>
struct CoordBases {
    Active<Net::K, Net::M, 2> b[2];
};

// z1[j] jets = first-layer output unit j: sum_d sum_q W0[j][d][c_d+q] * rows of x_d.
template <class Net, unsigned MASK>
__device__ __forceinline__ void layer0_unit(int j, const CoordBases<Net>& xb, const float* w0, int n,
                                            float* z) {
    using JT = Jet<MASK>;
#pragma unroll
    for (int r = 0; r < JT::J; ++r) z[r] = 0.0f;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const float* wr = w0 + (j * 2 + d) * n;
#pragma unroll
        for (int q = 0; q < Net::KP; ++q) {
            float w = wr[xb.b[d].idx(q, n)];
            z[0] = fmaf(w, xb.b[d].v[q], z[0]);
            if (d == 0) {
                if constexpr (JT::F0) z[JT::RF0] = fmaf(w, xb.b[d].d1[q], z[JT::RF0]);
                if constexpr (JT::S0) z[JT::RS0] = fmaf(w, xb.b[d].d2[q], z[JT::RS0]);
            } else {
                if constexpr (JT::F1) z[JT::RF1] = fmaf(w, xb.b[d].d1[q], z[JT::RF1]);
                if constexpr (JT::S1) z[JT::RS1] = fmaf(w, xb.b[d].d2[q], z[JT::RS1]);
            }
        }
    }
}

// dW0[j][d][c_d+q] += sum_r gz[r] * rows of x_d  (first-layer weight gradient for output unit j)
template <class Net, unsigned MASK>
__device__ __forceinline__ void layer0_unit_dw(int j, const CoordBases<Net>& xb, const float* gz,
                                               const DwAcc<Net>& dw, int n) {
    using JT = Jet<MASK>;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const int dr = Net::off_w0() + (j * 2 + d) * n;
#pragma unroll
        for (int q = 0; q < Net::KP; ++q) {
            float g = gz[0] * xb.b[d].v[q];
            if (d == 0) {
                if constexpr (JT::F0) g = fmaf(gz[JT::RF0], xb.b[d].d1[q], g);
                if constexpr (JT::S0) g = fmaf(gz[JT::RS0], xb.b[d].d2[q], g);
            } else {
                if constexpr (JT::F1) g = fmaf(gz[JT::RF1], xb.b[d].d1[q], g);
                if constexpr (JT::S1) g = fmaf(gz[JT::RS1], xb.b[d].d2[q], g);
            }
            int i = xb.b[d].c + q;
            if ((unsigned)i < (unsigned)n) dw.add(dr + i, g);
        }
    }
}

// Forward of one point: returns the last hidden layer jets h[WH][J] and output jets u[J].
template <class Net, unsigned MASK>
__device__ __forceinline__ void narrow_forward(const CoordBases<Net>& xb, const float* s, int n,
                                               const Grid& g, float (*h)[Jet<MASK>::J], float* u) {
    using JT = Jet<MASK>;
    constexpr int WH = Net::WH, J = JT::J, KP = Net::KP;
    const float* w0 = s + Net::off_w0();
    if constexpr (Net::NL == 2) {
#pragma unroll
        for (int j = 0; j < WH; ++j) layer0_unit<Net, MASK>(j, xb, w0, n, h[j]);
    } else {
        const float* w1 = s + Net::off_w1(n);
#pragma unroll
        for (int o = 0; o < WH; ++o)
#pragma unroll
            for (int r = 0; r < J; ++r) h[o][r] = 0.0f;
#pragma unroll 1
        for (int j = 0; j < WH; ++j) {
            float z[J];
            layer0_unit<Net, MASK>(j, xb, w0, n, z);
            Active<Net::K, Net::M, 2> b;
            b.eval(z[0], g);
            float a[J][KP];
            JT::template rows<KP>(z, b.v, b.d1, b.d2, a);
#pragma unroll
            for (int q = 0; q < KP; ++q) {
                const float4* wr = reinterpret_cast<const float4*>(w1 + (j * n + b.idx(q, n)) * Net::WHP);
#pragma unroll
                for (int o4 = 0; o4 < Net::WHP / 4; ++o4) {
                    float4 w4 = wr[o4];
                    float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int o = o4 * 4 + e;
                        if (o < WH) {
#pragma unroll
                            for (int r = 0; r < J; ++r) h[o][r] = fmaf(wv[e], a[r][q], h[o][r]);
                        }
                    }
                }
            }
        }
    }
    // output layer (O = 1)
    const float* wl = s + Net::off_wl(n);
#pragma unroll
    for (int r = 0; r < J; ++r) u[r] = 0.0f;
#pragma unroll
    for (int j = 0; j < WH; ++j) {
        Active<Net::K, Net::M, 2> b;
        b.eval(h[j][0], g);
        float a[J][KP];
        JT::template rows<KP>(h[j], b.v, b.d1, b.d2, a);
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            float w = wl[j * n + b.idx(q, n)];
#pragma unroll
            for (int r = 0; r < J; ++r) u[r] = fmaf(w, a[r][q], u[r]);
        }
    }
}

// Backward of one point given gu = dL/d(output jets); h[][] (last hidden jets
// from narrow_forward) is consumed.  Adds to the shared dW.
template <class Net, unsigned MASK>
__device__ __forceinline__ void narrow_backward(const CoordBases<Net>& xb, const float* s, const DwAcc<Net>& dw,
                                                int n, const Grid& g, float (*h)[Jet<MASK>::J],
                                                const float* gu) {
    using JT = Jet<MASK>;
    constexpr int WH = Net::WH, J = JT::J, KP = Net::KP;
    // output layer: dW_L and dL/dh
    const float* wl = s + Net::off_wl(n);
    const int dwl = Net::off_wl(n);
#pragma unroll
    for (int j = 0; j < WH; ++j) {
        Active<Net::K, Net::M, 3> b;
        b.eval(h[j][0], g);
        float a[J][KP], dA[J][KP];
        JT::template rows<KP>(h[j], b.v, b.d1, b.d2, a);
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            int i = b.c + q;
            float w = wl[j * n + b.idx(q, n)];
            float gw = 0.0f;
#pragma unroll
            for (int r = 0; r < J; ++r) {
                gw = fmaf(gu[r], a[r][q], gw);
                dA[r][q] = gu[r] * w;
            }
            if ((unsigned)i < (unsigned)n) dw.add(dwl + j * n + i, gw);
        }
        float gz[J];
        JT::template rows_adjoint<KP>(h[j], b.d1, b.d2, b.d3, dA, gz);
#pragma unroll
        for (int r = 0; r < J; ++r) h[j][r] = gz[r];   // h now holds dL/dh
    }
    if constexpr (Net::NL == 2) {
#pragma unroll
        for (int j = 0; j < WH; ++j) layer0_unit_dw<Net, MASK>(j, xb, h[j], dw, n);
    } else {
        const float* w0 = s + Net::off_w0();
        const float* w1 = s + Net::off_w1(n);
        const int dw1 = Net::off_w1(n);
        // Lanes that share a gradient copy (lane, lane+COPIES, ...) start at
        // different units, so at any instant they add into different rows.
        const int rot = ((int(threadIdx.x) & 31) / Net::COPIES) * WH / (32 / Net::COPIES);
#pragma unroll 1
        for (int jj = 0; jj < WH; ++jj) {
            const int j = (jj + rot < WH) ? jj + rot : jj + rot - WH;
            float z[J];
            layer0_unit<Net, MASK>(j, xb, w0, n, z);
            Active<Net::K, Net::M, 3> b;
            b.eval(z[0], g);
            float a[J][KP], dA[J][KP];
            JT::template rows<KP>(z, b.v, b.d1, b.d2, a);
#pragma unroll
            for (int q = 0; q < KP; ++q) {
                int i = b.c + q;
                bool ok = (unsigned)i < (unsigned)n;
                int row = (j * n + b.idx(q, n)) * Net::WHP;
                const float4* wr = reinterpret_cast<const float4*>(w1 + row);
#pragma unroll
                for (int r = 0; r < J; ++r) dA[r][q] = 0.0f;
#pragma unroll
                for (int o4 = 0; o4 < Net::WHP / 4; ++o4) {
                    float4 w4 = wr[o4];
                    float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int o = o4 * 4 + e;
                        if (o < WH) {
                            float gw = 0.0f;
#pragma unroll
                            for (int r = 0; r < J; ++r) {
                                gw = fmaf(h[o][r], a[r][q], gw);
                                dA[r][q] = fmaf(h[o][r], wv[e], dA[r][q]);
                            }
                            if (ok) dw.add(dw1 + row + o, gw);
                        }
                    }
                }
            }
            float gz[J];
            JT::template rows_adjoint<KP>(z, b.d1, b.d2, b.d3, dA, gz);
            layer0_unit_dw<Net, MASK>(j, xb, gz, dw, n);
        }
    }
}

// Everything a fused launch needs.
struct NarrowParams {
    const float* W;
    // point set 0 (interior in training; the only set in FWD/BWD)
    const float* x0;
    int64_t n0;
    float* jets;            // FWD: [J][n0]
    const float* dL;        // BWD: [J][n0]
    // point set 1 (boundary, TRAIN only)
    const float* x1;
    const float* g1;
    int64_t n1;
    float* partial;         // [gridDim.x][P]
    double* loss_partial;   // [gridDim.x][2]
    PdeParams pde;
    float scale0;           // 2 alpha / N_int
    float scale1;           // 2 / N_bnd
    Grid grid;
    int64_t P;
    int* t_counter;         // TRAIN: optional device step counter, t_counter[1] = t_counter[0] + 1
};

template <class Net>
__device__ __forceinline__ void narrow_block_loss(double a0, double a1, double* out) {
    __shared__ double red[2][NARROW_BLOCK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, o);
        a1 += __shfl_down_sync(0xffffffffu, a1, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = a0; red[1][w] = a1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int t = 0; t < NARROW_BLOCK / 32; ++t) { s0 += red[0][t]; s1 += red[1][t]; }
        out[0] = s0;
        out[1] = s1;
    }
}

template <class Net, unsigned MASK>
__global__ void __launch_bounds__(NARROW_BLOCK) narrow_fwd_kernel(NarrowParams p) {
    using JT = Jet<MASK>;
    extern __shared__ __align__(16) float smem[];
    const int n = p.grid.n;
    narrow_load_w<Net>(p.W, smem, n);
    __syncthreads();
    const int64_t N = p.n0;
    for (int64_t pt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; pt < N;
         pt += int64_t(gridDim.x) * blockDim.x) {
        CoordBases<Net> xb;
        xb.b[0].eval(p.x0[pt], p.grid);
        xb.b[1].eval(p.x0[N + pt], p.grid);
        float h[Net::WH][JT::J], u[JT::J];
        narrow_forward<Net, MASK>(xb, smem, n, p.grid, h, u);
#pragma unroll
        for (int r = 0; r < JT::J; ++r) p.jets[r * N + pt] = u[r];
    }
}

// MODE_BWD: one point set, gu read from dL.  MODE_TRAIN: interior (MASK)
// then boundary (value only) tiles, gu from the residual.
template <class Net, unsigned MASK, int MODE>
__global__ void __launch_bounds__(NARROW_BLOCK, Net::MINB) narrow_grad_kernel(NarrowParams p) {
    extern __shared__ __align__(16) float smem[];
    if (MODE == MODE_TRAIN && p.t_counter && blockIdx.x == 0 && threadIdx.x == 0)
        p.t_counter[1] = p.t_counter[0] + 1;
    const int n = p.grid.n;
    const int sf = Net::smem_floats(n);
    float* s = smem;
    float* ds = smem + sf;
    narrow_load_w<Net>(p.W, s, n);
    for (int t = threadIdx.x; t < sf * Net::COPIES; t += blockDim.x) ds[t] = 0.0f;
    __syncthreads();
    const DwAcc<Net> dwacc{ds, int(threadIdx.x) & (Net::COPIES - 1)};

    const int64_t T0 = (p.n0 + NARROW_BLOCK - 1) / NARROW_BLOCK;
    const int64_t T1 = (MODE == MODE_TRAIN) ? (p.n1 + NARROW_BLOCK - 1) / NARROW_BLOCK : 0;
    double lsum0 = 0.0, lsum1 = 0.0;
    for (int64_t tile = blockIdx.x; tile < T0 + T1; tile += gridDim.x) {
        if (tile < T0) {
            using JT = Jet<MASK>;
            const int64_t pt = tile * NARROW_BLOCK + threadIdx.x;
            if (pt < p.n0) {
                const int64_t N = p.n0;
                float x0 = p.x0[pt], x1 = p.x0[N + pt];
                CoordBases<Net> xb;
                xb.b[0].eval(x0, p.grid);
                xb.b[1].eval(x1, p.grid);
                float h[Net::WH][JT::J], u[JT::J], gu[JT::J];
                narrow_forward<Net, MASK>(xb, s, n, p.grid, h, u);
                if constexpr (MODE == MODE_TRAIN) {
                    float r = pde_residual<MASK>(p.pde, x0, x1, u);
                    lsum0 += double(r) * double(r);
                    pde_residual_grad<MASK>(p.pde, r, u, p.scale0, gu);
                } else {
#pragma unroll
                    for (int q = 0; q < JT::J; ++q) gu[q] = p.dL[q * N + pt];
                }
                narrow_backward<Net, MASK>(xb, s, dwacc, n, p.grid, h, gu);
            }
        } else if constexpr (MODE == MODE_TRAIN) {
            const int64_t pt = (tile - T0) * NARROW_BLOCK + threadIdx.x;
            if (pt < p.n1) {
                const int64_t N = p.n1;
                CoordBases<Net> xb;
                xb.b[0].eval(p.x1[pt], p.grid);
                xb.b[1].eval(p.x1[N + pt], p.grid);
                float h[Net::WH][1], u[1], gu[1];
                narrow_forward<Net, 1u>(xb, s, n, p.grid, h, u);
                float d = u[0] - p.g1[pt];
                lsum1 += double(d) * double(d);
                gu[0] = p.scale1 * d;
                narrow_backward<Net, 1u>(xb, s, dwacc, n, p.grid, h, gu);
            }
        }
    }
    if constexpr (MODE == MODE_TRAIN) narrow_block_loss<Net>(lsum0, lsum1, p.loss_partial + 2 * blockIdx.x);
    __syncthreads();
    // fold the copies into the (no longer needed) weight region, then store
    for (int t = threadIdx.x; t < sf; t += blockDim.x) {
        float a = 0.0f;
#pragma unroll
        for (int c = 0; c < Net::COPIES; ++c) a += ds[t * Net::COPIES + c];
        s[t] = a;
    }
    __syncthreads();
    narrow_store_dw<Net>(s, p.partial + int64_t(blockIdx.x) * p.P, n);
}

}  // namespace hrkan

// ---------------------------------------------------------------------------
// Many independent networks of one narrow shape in one persistent launch.
//
// The host cuts every instance's interior and boundary points into items of a
// few tiles; block b walks items b, b + grid, ...  Per item the block loads
// that instance's weights into shared memory, accumulates the item's weight
// gradient in the shared copies, and writes one partial row (and one loss
// partial) per item.  A second kernel sums each instance's rows in a fixed
// order and applies Adam per instance.
namespace hrkan {

struct BatchItem {
    int inst;          // instance
    int set;           // 0 = interior (residual), 1 = boundary / initial (value)
    int64_t begin;     // point range [begin, end) in the concatenated set
    int64_t end;
};

struct BatchInst {
    float a, b, src;   // Poisson frequencies and (a^2+b^2) pi^2
    float scale0;      // 2 alpha / N_int of the instance
    float scale1;      // 2 / N_bnd of the instance
};

struct BatchParams {
    const float* W;            // [inst][P]
    int64_t P;
    const float* x0;           // interior [2][n0]
    int64_t n0;
    const float* x1;           // boundary [2][n1]
    const float* g1;
    int64_t n1;
    float* jets;               // forward only: [J][n0]
    const BatchItem* items;
    int n_items;
    const BatchInst* inst;
    PdeParams pde;             // kind, lam, nu, alpha (shared by the instances)
    float* partial;            // [n_items][P]
    double* loss_partial;      // [n_items][2]
    Grid grid;
    int* t_counter;
};

template <class Net, unsigned MASK>
__global__ void __launch_bounds__(NARROW_BLOCK, Net::MINB) narrow_batch_kernel(BatchParams p) {
    extern __shared__ __align__(16) float smem[];
    if (p.t_counter && blockIdx.x == 0 && threadIdx.x == 0) p.t_counter[1] = p.t_counter[0] + 1;
    const int n = p.grid.n;
    const int sf = Net::smem_floats(n);
    float* s = smem;
    float* ds = smem + sf;
    const DwAcc<Net> dwacc{ds, int(threadIdx.x) & (Net::COPIES - 1)};
    for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
        const BatchItem item = p.items[it];
        const BatchInst bi = p.inst[item.inst];
        narrow_load_w<Net>(p.W + int64_t(item.inst) * p.P, s, n);
        for (int t = threadIdx.x; t < sf * Net::COPIES; t += blockDim.x) ds[t] = 0.0f;
        __syncthreads();
        PdeParams pde = p.pde;
        pde.a = bi.a;
        pde.b = bi.b;
        pde.src = bi.src;
        double lsum = 0.0;
        for (int64_t base = item.begin; base < item.end; base += NARROW_BLOCK) {
            const int64_t pt = base + threadIdx.x;
            if (pt >= item.end) continue;
            if (item.set == 0) {
                using JT = Jet<MASK>;
                const int64_t N = p.n0;
                const float x0 = p.x0[pt], x1 = p.x0[N + pt];
                CoordBases<Net> xb;
                xb.b[0].eval(x0, p.grid);
                xb.b[1].eval(x1, p.grid);
                float h[Net::WH][JT::J], u[JT::J], gu[JT::J];
                narrow_forward<Net, MASK>(xb, s, n, p.grid, h, u);
                const float r = pde_residual<MASK>(pde, x0, x1, u);
                lsum += double(r) * double(r);
                pde_residual_grad<MASK>(pde, r, u, bi.scale0, gu);
                narrow_backward<Net, MASK>(xb, s, dwacc, n, p.grid, h, gu);
            } else {
                const int64_t N = p.n1;
                CoordBases<Net> xb;
                xb.b[0].eval(p.x1[pt], p.grid);
                xb.b[1].eval(p.x1[N + pt], p.grid);
                float h[Net::WH][1], u[1], gu[1];
                narrow_forward<Net, 1u>(xb, s, n, p.grid, h, u);
                const float d = u[0] - p.g1[pt];
                lsum += double(d) * double(d);
                gu[0] = bi.scale1 * d;
                narrow_backward<Net, 1u>(xb, s, dwacc, n, p.grid, h, gu);
            }
        }
        narrow_block_loss<Net>(item.set == 0 ? lsum : 0.0, item.set == 0 ? 0.0 : lsum,
                               p.loss_partial + 2 * int64_t(it));
        __syncthreads();
        for (int t = threadIdx.x; t < sf; t += blockDim.x) {
            float a = 0.0f;
#pragma unroll
            for (int c = 0; c < Net::COPIES; ++c) a += ds[t * Net::COPIES + c];
            s[t] = a;
        }
        __syncthreads();
        narrow_store_dw<Net>(s, p.partial + int64_t(it) * p.P, n);
        __syncthreads();
    }
}

// Forward jets of many instances: items carry the instance of each point range.
template <class Net, unsigned MASK>
__global__ void __launch_bounds__(NARROW_BLOCK) narrow_batch_fwd_kernel(BatchParams p) {
    using JT = Jet<MASK>;
    extern __shared__ __align__(16) float smem[];
    const int n = p.grid.n;
    for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
        const BatchItem item = p.items[it];
        narrow_load_w<Net>(p.W + int64_t(item.inst) * p.P, smem, n);
        __syncthreads();
        const int64_t N = p.n0;
        for (int64_t pt = item.begin + threadIdx.x; pt < item.end; pt += NARROW_BLOCK) {
            CoordBases<Net> xb;
            xb.b[0].eval(p.x0[pt], p.grid);
            xb.b[1].eval(p.x0[N + pt], p.grid);
            float h[Net::WH][JT::J], u[JT::J];
            narrow_forward<Net, MASK>(xb, smem, n, p.grid, h, u);
#pragma unroll
            for (int r = 0; r < JT::J; ++r) p.jets[r * N + pt] = u[r];
        }
        __syncthreads();
    }
}

}  // namespace hrkan
