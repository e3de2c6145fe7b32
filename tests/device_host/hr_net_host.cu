// Host harness: a whole network's input jets in float32, composed from the
// device formulas of csrc/hr_device.cuh (Active, Jet::rows_b) in the order the
// layer-wise forward kernel accumulates them (per output and row: over input
// units, then over the k+1 active bases, one fmaf each).  A CPU test compares
// the result with the FP64 oracle, which shows the float32 error level of the
// formulas through several layers, including the jet rows no kernel has been
// instantiated for yet.
//
// usage: hr_net_host <in> <out> [bwd]
//   in:  int32 m, mask, n_widths, widths[n_widths], G, N, seed0, seed1;
//        float32 lo, hi, W[params] ([layer][O][I][G+3]), x[widths[0]][N], and
//        with bwd gy[J][N].  The first layer's derivative rows differentiate
//        along inputs seed0 and seed1 (-1: along none), as the kernels seed
//        them: three-input networks run as a pass along (x, y) and one along z.
//   out: float32 jets[J][N] (rows in mask-bit order), or with bwd float64 dW[params]
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_2409_14248_gb300/csrc/hr_device.cuh"

using namespace hrkan;

static const int K = 3, KP = K + 1, MAXW = 64;

template <int M, unsigned MASK>
static void net_forward(const std::vector<int>& widths, const Grid& g, const float* W, const float* x, long N,
                        int seed0, int seed1, float* out) {
    using JT = Jet<MASK>;
    constexpr int J = JT::J;
    const int L = int(widths.size()) - 1, n = g.n;
    std::vector<float> z(size_t(J) * MAXW), y(size_t(J) * MAXW);
    for (long p = 0; p < N; ++p) {
        // first layer: the coordinates, with derivative 1 along the seeded directions
        const int I0 = widths[0];
        for (int r = 0; r < J; ++r)
            for (int j = 0; j < I0; ++j) z[r * MAXW + j] = 0.0f;
        for (int j = 0; j < I0; ++j) z[j] = x[j * N + p];
        if constexpr (JT::F0) if (seed0 >= 0) z[JT::RF0 * MAXW + seed0] = 1.0f;
        if constexpr (JT::F1) if (seed1 >= 0) z[JT::RF1 * MAXW + seed1] = 1.0f;
        const float* Wl = W;
        for (int l = 0; l < L; ++l) {
            const int I = widths[l], O = widths[l + 1];
            float acc[MAXW][J];
            for (int o = 0; o < O; ++o)
                for (int r = 0; r < J; ++r) acc[o][r] = 0.0f;
            for (int j = 0; j < I; ++j) {
                float zj[J];
                for (int r = 0; r < J; ++r) zj[r] = z[r * MAXW + j];
                Active<K, M, JT::NDER_ROWS> b;
                b.eval(zj[0], g);
                float a[J][KP];
                JT::template rows_b<KP>(zj, b, a);
                for (int q = 0; q < KP; ++q) {
                    const int i = b.idx(q, n);
                    for (int o = 0; o < O; ++o) {
                        const float w = Wl[(long(o) * I + j) * n + i];
                        for (int r = 0; r < J; ++r) acc[o][r] = fmaf(w, a[r][q], acc[o][r]);
                    }
                }
            }
            for (int r = 0; r < J; ++r)
                for (int o = 0; o < O; ++o) y[r * MAXW + o] = acc[o][r];
            z.swap(y);
            Wl += long(O) * I * n;
        }
        for (int r = 0; r < J; ++r) out[r * N + p] = z[r * MAXW];
    }
}

// Weight gradient for output-jet gradients gy[J][N]: per point, the forward
// with its layer inputs kept, then from the last layer down dW += gy^T A (the
// rows of rows_b) and dA = gy W, taken to the layer's input jets by adjoint_b.
// Per point everything is float32 (fmaf); the sum over points is float64, so
// the result shows the formulas' error rather than a summation order's.
template <int M, unsigned MASK>
static void net_backward(const std::vector<int>& widths, const Grid& g, const float* W, const float* x, long N,
                         int seed0, int seed1, const float* gy, double* dW) {
    using JT = Jet<MASK>;
    constexpr int J = JT::J;
    const int L = int(widths.size()) - 1, n = g.n;
    std::vector<long> off(L + 1, 0);
    for (int l = 0; l < L; ++l) off[l + 1] = off[l] + long(widths[l]) * widths[l + 1] * n;
    for (long i = 0; i < off[L]; ++i) dW[i] = 0.0;
    std::vector<float> tape(size_t(L) * J * MAXW), gcur(size_t(J) * MAXW), gnext(size_t(J) * MAXW);
    for (long p = 0; p < N; ++p) {
        float* z0 = tape.data();
        for (int r = 0; r < J; ++r)
            for (int j = 0; j < MAXW; ++j) z0[r * MAXW + j] = 0.0f;
        for (int j = 0; j < widths[0]; ++j) z0[j] = x[j * N + p];
        if constexpr (JT::F0) if (seed0 >= 0) z0[JT::RF0 * MAXW + seed0] = 1.0f;
        if constexpr (JT::F1) if (seed1 >= 0) z0[JT::RF1 * MAXW + seed1] = 1.0f;
        for (int l = 0; l + 1 < L; ++l) {      // inputs of layers 1 .. L-1
            const int I = widths[l], O = widths[l + 1];
            const float* z = tape.data() + size_t(l) * J * MAXW;
            float* y = tape.data() + size_t(l + 1) * J * MAXW;
            float acc[MAXW][J];
            for (int o = 0; o < O; ++o)
                for (int r = 0; r < J; ++r) acc[o][r] = 0.0f;
            for (int j = 0; j < I; ++j) {
                float zj[J];
                for (int r = 0; r < J; ++r) zj[r] = z[r * MAXW + j];
                Active<K, M, JT::NDER_ROWS> b;
                b.eval(zj[0], g);
                float a[J][KP];
                JT::template rows_b<KP>(zj, b, a);
                for (int q = 0; q < KP; ++q)
                    for (int o = 0; o < O; ++o) {
                        const float w = W[off[l] + (long(o) * I + j) * n + b.idx(q, n)];
                        for (int r = 0; r < J; ++r) acc[o][r] = fmaf(w, a[r][q], acc[o][r]);
                    }
            }
            for (int r = 0; r < J; ++r)
                for (int o = 0; o < O; ++o) y[r * MAXW + o] = acc[o][r];
        }
        for (int r = 0; r < J; ++r) gcur[r * MAXW] = gy[r * N + p];
        for (int l = L - 1; l >= 0; --l) {
            const int I = widths[l], O = widths[l + 1];
            const float* z = tape.data() + size_t(l) * J * MAXW;
            for (int j = 0; j < I; ++j) {
                float zj[J];
                for (int r = 0; r < J; ++r) zj[r] = z[r * MAXW + j];
                Active<K, M, JT::NDER_ADJ> b;
                b.eval(zj[0], g);
                float a[J][KP], dA[J][KP];
                JT::template rows_b<KP>(zj, b, a);
                for (int q = 0; q < KP; ++q) {
                    const int i = b.idx(q, n);
                    for (int r = 0; r < J; ++r) dA[r][q] = 0.0f;
                    for (int o = 0; o < O; ++o) {
                        const long wi = off[l] + (long(o) * I + j) * n + i;
                        float gw = 0.0f;
                        for (int r = 0; r < J; ++r) {
                            gw = fmaf(gcur[r * MAXW + o], a[r][q], gw);
                            dA[r][q] = fmaf(gcur[r * MAXW + o], W[wi], dA[r][q]);
                        }
                        dW[wi] += double(gw);
                    }
                }
                if (l > 0) {
                    float gz[J];
                    JT::template adjoint_b<KP>(zj, b, dA, gz);
                    for (int r = 0; r < J; ++r) gnext[r * MAXW + j] = gz[r];
                }
            }
            gcur.swap(gnext);
        }
    }
}

template <int M>
static bool by_mask_bwd(unsigned mask, const std::vector<int>& w, const Grid& g, const float* W, const float* x,
                        long N, int s0, int s1, const float* gy, double* dW) {
    switch (mask) {
        case 0x0Fu: net_backward<M, 0x0Fu>(w, g, W, x, N, s0, s1, gy, dW); return true;
        case 0x1Fu: net_backward<M, 0x1Fu>(w, g, W, x, N, s0, s1, gy, dW); return true;
        case 0x2Fu: net_backward<M, 0x2Fu>(w, g, W, x, N, s0, s1, gy, dW); return true;
        case 0xFFu: net_backward<M, 0xFFu>(w, g, W, x, N, s0, s1, gy, dW); return true;
        case 0x12Fu: net_backward<M, 0x12Fu>(w, g, W, x, N, s0, s1, gy, dW); return true;
        case 0x52Fu: net_backward<M, 0x52Fu>(w, g, W, x, N, s0, s1, gy, dW); return true;
        case 0xFFFu: net_backward<M, 0xFFFu>(w, g, W, x, N, s0, s1, gy, dW); return true;
    }
    return false;
}

template <int M>
static bool by_mask(unsigned mask, const std::vector<int>& w, const Grid& g, const float* W, const float* x, long N,
                    int s0, int s1, float* out) {
    switch (mask) {
        case 0x0Fu: net_forward<M, 0x0Fu>(w, g, W, x, N, s0, s1, out); return true;
        case 0x1Fu: net_forward<M, 0x1Fu>(w, g, W, x, N, s0, s1, out); return true;
        case 0x2Fu: net_forward<M, 0x2Fu>(w, g, W, x, N, s0, s1, out); return true;
        case 0xFFu: net_forward<M, 0xFFu>(w, g, W, x, N, s0, s1, out); return true;
        case 0x12Fu: net_forward<M, 0x12Fu>(w, g, W, x, N, s0, s1, out); return true;
        case 0x52Fu: net_forward<M, 0x52Fu>(w, g, W, x, N, s0, s1, out); return true;
        case 0xFFFu: net_forward<M, 0xFFFu>(w, g, W, x, N, s0, s1, out); return true;
    }
    return false;
}

static bool rd(FILE* f, void* p, size_t bytes) { return fread(p, 1, bytes, f) == bytes; }

int main(int argc, char** argv) {
    if (argc != 3 && argc != 4) return 2;
    const bool bwd = argc == 4;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 3;
    int m = 0, nw = 0, G = 0, N = 0;
    unsigned mask = 0;
    if (!rd(f, &m, 4) || !rd(f, &mask, 4) || !rd(f, &nw, 4) || nw < 2 || nw > 16) return 4;
    std::vector<int> widths(nw);
    int seed0 = 0, seed1 = 1;
    if (!rd(f, widths.data(), 4 * size_t(nw)) || !rd(f, &G, 4) || !rd(f, &N, 4) || G < 1 || N < 1) return 4;
    if (!rd(f, &seed0, 4) || !rd(f, &seed1, 4)) return 4;
    if (widths[0] < 2 || widths[0] > 3 || widths[nw - 1] != 1) return 4;
    if (seed0 < -1 || seed0 >= widths[0] || seed1 < -1 || seed1 >= widths[0]) return 4;
    for (int w : widths)
        if (w < 1 || w > MAXW) return 4;
    float lo = 0.0f, hi = 0.0f;
    if (!rd(f, &lo, 4) || !rd(f, &hi, 4)) return 4;
    const int n = G + K;
    long P = 0;
    for (int l = 0; l + 1 < nw; ++l) P += long(widths[l]) * widths[l + 1] * n;
    std::vector<float> W(P), x(size_t(widths[0]) * N);
    if (!rd(f, W.data(), 4 * size_t(P)) || !rd(f, x.data(), 4 * x.size())) return 4;
    int J = 0;
    for (int b = 0; b < 12; ++b) J += (mask >> b) & 1;
    std::vector<float> gy(bwd ? size_t(J) * N : 0);
    if (bwd && !rd(f, gy.data(), 4 * gy.size())) return 4;
    fclose(f);
    Grid g;   // as the library's handle sets it up
    const double hh = (double(hi) - double(lo)) / G;
    g.lo = lo;
    g.h = float(hh);
    g.inv_h = float(1.0 / hh);
    g.inv_a = float(2.0 / ((K + 1) * hh));
    g.m = m;
    g.n = n;
    if (bwd) {
        std::vector<double> dW(P);
        bool ok = false;
        switch (m) {
            case 4: ok = by_mask_bwd<4>(mask, widths, g, W.data(), x.data(), N, seed0, seed1, gy.data(), dW.data()); break;
            case 6: ok = by_mask_bwd<6>(mask, widths, g, W.data(), x.data(), N, seed0, seed1, gy.data(), dW.data()); break;
        }
        if (!ok) return 5;
        FILE* o = fopen(argv[2], "wb");
        if (!o || fwrite(dW.data(), 8, dW.size(), o) != dW.size()) return 6;
        fclose(o);
        return 0;
    }
    std::vector<float> out(size_t(J) * N);
    bool ok = false;
    switch (m) {
        case 4: ok = by_mask<4>(mask, widths, g, W.data(), x.data(), N, seed0, seed1, out.data()); break;
        case 6: ok = by_mask<6>(mask, widths, g, W.data(), x.data(), N, seed0, seed1, out.data()); break;
    }
    if (!ok) return 5;
    FILE* o = fopen(argv[2], "wb");
    if (!o || fwrite(out.data(), 4, out.size(), o) != out.size()) return 6;
    fclose(o);
    return 0;
}
