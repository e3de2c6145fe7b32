// Host harness for the device basis and jet-row formulas (csrc/hr_device.cuh):
// prints the kernels' own float32 values for a fixed set of inputs so that a
// CPU test can compare them with the FP64 oracle.  Output lines:
//   B m z c v0..v3 d1_0..d1_3 d2_.. d3_.. d4_.. d5_.. d6_..  (Active<3, m, 6>)
//   R mask m z c <J rows x 4 entries> <J adjoint values>  (Jet rows and their reverse)
//   P kind mask x0 x1 u r <J values of gu>               (pde_residual, pde_residual_grad)
//   W mask m z c <J adjoint values>                      (the reverse row by row, row_adjoint)
// Inputs of the R lines: jets z[r] = zr[r] (z[0] = the value), dA[r][q] =
// gy[r] * w[c + q] with w[i] = wv(i) (a rank-1 gradient, as a one-output layer has).
#include <cstdio>

#include "../../paper_2409_14248_gb300/csrc/hr_device.cuh"

using namespace hrkan;

static const int G = 6, K = 3;
static const float ZS[] = {-1.3f, -1.0f, -0.95f, -2.0f / 3.0f, -0.5f, -0.31f, -0.1f, 0.0f, 0.07f,
                           1.0f / 3.0f, 0.42f, 0.8f, 0.999f, 1.0f, 1.2f};
// z[0] replaced per line
static const float ZR[12] = {0.0f, 0.7f, -1.3f, 0.45f, -0.8f, 2.1f, -0.6f, 0.35f, -1.7f, 0.9f, 2.4f, -0.55f};
static const float GY[12] = {0.9f, -0.4f, 1.7f, 0.25f, -1.1f, 0.6f, 1.3f, -0.75f, 0.5f, -0.95f, 0.3f, 1.15f};
static float wv(int i) { return 0.5f - 0.17f * float(i) + 0.03f * float(i * i); }

static Grid grid(int m) {
    Grid g;
    g.lo = -1.0f;
    g.h = 2.0f / G;
    g.inv_h = G / 2.0f;
    g.inv_a = 2.0f / ((K + 1) * g.h);
    g.n = G + K;
    g.m = m;
    return g;
}

template <int M>
static void basis() {
    const Grid g = grid(M);
    for (float z : ZS) {
        Active<K, M, 6> a;
        a.eval(z, g);
        printf("B %d %.9g %d", M, (double)z, a.c);
        const float* arr[7] = {a.v, a.d1, a.d2, a.d3, a.d4, a.d5, a.d6};
        for (auto* p : arr)
            for (int q = 0; q <= K; ++q) printf(" %.9g", (double)p[q]);
        printf("\n");
    }
}

template <unsigned MASK, int M>
static void rows() {
    using JT = Jet<MASK>;
    const Grid g = grid(M);
    for (float z0 : ZS) {
        Active<K, M, 6> a;
        a.eval(z0, g);
        float z[12], gz[12], A[12][K + 1], dA[12][K + 1];
        int r = 0;
        for (int b = 0; b < 12; ++b)
            if (MASK & (1u << b)) z[r++] = (b == 0) ? z0 : ZR[b];
        for (int rr = 0; rr < JT::J; ++rr)
            for (int q = 0; q <= K; ++q) {
                const int i = a.c + q;
                dA[rr][q] = (i >= 0 && i < g.n) ? GY[rr] * wv(i) : 0.0f;
            }
        JT::template rows_b<K + 1>(z, a, A);
        JT::template adjoint_b<K + 1>(z, a, dA, gz);
        printf("R %u %d %.9g %d", MASK, M, (double)z0, a.c);
        for (int rr = 0; rr < JT::J; ++rr)
            for (int q = 0; q <= K; ++q) printf(" %.9g", (double)A[rr][q]);
        for (int rr = 0; rr < JT::J; ++rr) printf(" %.9g", (double)gz[rr]);
        printf("\n");
    }
}

// The reverse of the R lines' rows taken one row of dA at a time (Jet::row_adjoint,
// as the tensor-core adjoint applies it), same inputs.
template <unsigned MASK, int M>
static void rows_rowwise() {
    using JT = Jet<MASK>;
    const Grid g = grid(M);
    for (float z0 : ZS) {
        Active<K, M, 6> a;
        a.eval(z0, g);
        float z[12], gz[12];
        int r = 0;
        for (int b = 0; b < 12; ++b)
            if (MASK & (1u << b)) z[r++] = (b == 0) ? z0 : ZR[b];
        for (int rr = 0; rr < JT::J; ++rr) gz[rr] = 0.0f;
        for (int rr = 0; rr < JT::J; ++rr) {
            float dA[K + 1];
            for (int q = 0; q <= K; ++q) {
                const int i = a.c + q;
                dA[q] = (i >= 0 && i < g.n) ? GY[rr] * wv(i) : 0.0f;
            }
            JT::template row_adjoint<K + 1>(rr, z, a.d1, a.d2, a.d3, dA, gz);
        }
        printf("W %u %d %.9g %d", MASK, M, (double)z0, a.c);
        for (int rr = 0; rr < JT::J; ++rr) printf(" %.9g", (double)gz[rr]);
        printf("\n");
    }
}

// Residual r of one interior point and gu = dL/d(jets) for L = alpha r^2
// (scale 2 alpha: one point), with the point's jets taken from ZR and a
// varying value row.  Problem constants as make_pde in csrc/capi.cu sets them.
static const double PI = 3.14159265358979323846;
static PdeParams problem(int kind) {
    PdeParams P{};
    P.kind = kind;
    P.a = 2.0f;
    P.b = 3.0f;
    P.src = float((2.0 * 2.0 + 3.0 * 3.0) * PI * PI);
    P.lam = kind == 1 ? 1.0f : 6.0f;
    P.nu = kind == 1 ? float(0.01 / PI) : 1.0f;
    P.alpha = 0.5f;
    return P;
}

template <unsigned MASK>
static void residual(int kind) {
    using JT = Jet<MASK>;
    const PdeParams P = problem(kind);
    static const float X0[] = {-0.9f, -0.37f, 0.0f, 0.21f, 0.64f};
    static const float X1[] = {0.15f, -0.8f, 0.5f, 0.93f, -0.05f};
    for (int t = 0; t < 5; ++t) {
        float u[12], gu[12];
        int r = 0;
        for (int b = 0; b < 12; ++b)
            if (MASK & (1u << b)) u[r++] = (b == 0) ? 0.3f * float(t) - 0.55f : ZR[b];
        const float res = pde_residual<MASK>(P, X0[t], X1[t], u);
        pde_residual_grad<MASK>(P, res, u, 2.0f * P.alpha, gu);
        printf("P %d %u %.9g %.9g %.9g %.9g", kind, MASK, (double)X0[t], (double)X1[t], (double)u[0], (double)res);
        for (int rr = 0; rr < JT::J; ++rr) printf(" %.9g", (double)gu[rr]);
        printf("\n");
    }
}

int main() {
    basis<2>(); basis<3>(); basis<4>(); basis<5>(); basis<6>();
    rows<0x1Fu, 4>(); rows<0x0Fu, 4>(); rows<0xFFu, 4>(); rows<0xFFu, 6>(); rows<0x2Fu, 3>();
    rows<0x12Fu, 5>(); rows<0x52Fu, 6>(); rows<0x3FFu, 4>(); rows<0xFFFu, 6>();
    residual<0x1Fu>(0); residual<0xFFu>(0); residual<0x0Fu>(1); residual<0xFFu>(1); residual<0x2Fu>(2);
    residual<0x7Fu>(2);
    rows_rowwise<0x1Fu, 4>(); rows_rowwise<0x0Fu, 4>(); rows_rowwise<0x07u, 3>(); rows_rowwise<0x01u, 4>();
    return 0;
}
