// Device building blocks of the HRKAN hot path: the HR basis with its first
// six derivatives on the k+1 active supports (Section 3, Eq. 2), and the
// jet-row structure that the PDE residuals need (Eq. 3: the Laplacian; Eq. 6:
// u_t, u_x, u_xx).  The basis evaluation, the row formulas and the residuals
// are also callable on the host, where a test compares them with the FP64 oracle.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hrkan {

// Geometry of the uniform grid shared by every layer.
struct Grid {
    float lo;      // grid_lo
    float h;       // (grid_hi - grid_lo) / G
    float inv_h;   // G / (grid_hi - grid_lo)
    float inv_a;   // 1 / half-width of a support = 2 / ((k+1) h)
    int n;         // number of bases G + k
    int m;         // HR order of Eq. 2
};

// Active bases of one input value.
//
// Basis i lives on [s_i, e_i] = [lo + (i-k)h, lo + (i+1)h].  With
// t = (z - lo)/h and c = floor(t), the bases touching z are i = c + q,
// q = 0..K.  The offset inside the cell is taken from the knot,
// f = (z - (lo + c h))/h, not as t - c: for |z| much smaller than the grid
// range, t carries an absolute error of one ulp of t, far above the ulp of z.  Writing u = (z - mid_i)/a for the position inside the support
// (a = (K+1)h/2 the half-width), Eq. 2 becomes v = (1 - u^2)^M because
// c_m = a^{-2m}, and u = (2(t - c) + K - 1 - 2q)/(K + 1) for basis c + q.
// With Q = 1 - u^2 the derivatives with respect to z are
//   v'   = -2M u Q^{M-1} / a
//   v''  = (-2M Q^{M-1} + 4M(M-1) u^2 Q^{M-2}) / a^2
//   v''' = (12M(M-1) u Q^{M-2} - 8M(M-1)(M-2) u^3 Q^{M-3}) / a^3
//   v''''= (12M(M-1) Q^{M-2} - 48M(M-1)(M-2) u^2 Q^{M-3} + 16M(M-1)(M-2)(M-3) u^4 Q^{M-4}) / a^4
// and in general, because Q is quadratic in u (Faa di Bruno's formula with
// Q' = -2u, Q'' = -2 and (M)_j = M(M-1)...(M-j+1), zero for j > M),
//   d^r/du^r Q^M = sum_{j <= r/2} r!/(j!(r-2j)!) (-1)^j (M)_{r-j} (-2u)^{r-2j} Q^{M-r+j},
// which gives the fifth and sixth derivatives
//   v^(5) = (-120(M)_3 u Q^{M-3} + 160(M)_4 u^3 Q^{M-4} - 32(M)_5 u^5 Q^{M-5}) / a^5
//   v^(6) = (-120(M)_3 Q^{M-3} + 720(M)_4 u^2 Q^{M-4} - 480(M)_5 u^4 Q^{M-5} + 64(M)_6 u^6 Q^{M-6}) / a^6
// A basis index outside [0, n) gets all-zero values and a clamped index.
template <int E>
__host__ __device__ __forceinline__ float qpow(float Q) {
    float r = 1.0f;
#pragma unroll
    for (int e = 0; e < E; ++e) r *= Q;
    return r;
}

// (M)_j = M (M-1) ... (M-j+1), zero once j > M.
__host__ __device__ constexpr float falling(int M, int j) {
    float r = 1.0f;
    for (int t = 0; t < j; ++t) r *= float(M - t);
    return r;
}

template <int K, int M, int NDER>
struct Active {
    int c;               // first active basis index (may be < 0 or > n-1-K)
    float v[K + 1];      // v_{c+q}(z)
    float d1[K + 1];     // v'
    float d2[K + 1];     // v''
    float d3[K + 1];     // v''' (only when NDER >= 3)
    float d4[K + 1];     // v'''' (only when NDER >= 4)
    float d5[K + 1];     // v^(5) (only when NDER >= 5)
    float d6[K + 1];     // v^(6) (only when NDER >= 6)

    __host__ __device__ __forceinline__ int idx(int q, int n) const {
        int i = c + q;
        return (i < 0) ? 0 : (i >= n ? n - 1 : i);
    }

    __host__ __device__ __forceinline__ void eval(float z, const Grid& g) {
        static_assert(M >= 2, "the jets need M >= 2");
        float t = (z - g.lo) * g.inv_h;
        // Beyond +-2^30 cells nothing is active; keep floorf's result in int range.
        t = fminf(fmaxf(t, -1.0e9f), 1.0e9f);
        float fc = floorf(t);
        c = (int)fc;
        float f = (z - fmaf(fc, g.h, g.lo)) * g.inv_h;
        const float s = 2.0f / (K + 1);
#pragma unroll
        for (int q = 0; q < K + 1; ++q) {
            float u = (f + 0.5f * (K - 1 - 2 * q)) * s;
            float Q = fmaxf(1.0f - u * u, 0.0f);
            // powers Q^{M-3} .. Q^{M}
            float Qm3 = 1.0f;
#pragma unroll
            for (int e = 0; e < M - 3; ++e) Qm3 *= Q;
            float Qm2 = (M >= 3) ? Qm3 * Q : 1.0f;
            float Qm1 = Qm2 * Q;
            float Qm = Qm1 * Q;
            bool ok = (unsigned)(c + q) < (unsigned)g.n;
            float a1 = g.inv_a;
            v[q] = ok ? Qm : 0.0f;
            d1[q] = ok ? (-2.0f * M) * u * Qm1 * a1 : 0.0f;
            float u2 = u * u;
            d2[q] = ok ? ((-2.0f * M) * Qm1 + (4.0f * M * (M - 1)) * u2 * Qm2) * (a1 * a1) : 0.0f;
            if constexpr (NDER >= 3) {
                float t3 = (12.0f * M * (M - 1)) * u * Qm2;
                if constexpr (M >= 3) t3 -= (8.0f * M * (M - 1) * (M - 2)) * u2 * u * Qm3;
                d3[q] = ok ? t3 * (a1 * a1 * a1) : 0.0f;
            }
            if constexpr (NDER >= 4) {
                float t4 = (12.0f * M * (M - 1)) * Qm2;
                if constexpr (M >= 3) t4 -= (48.0f * M * (M - 1) * (M - 2)) * u2 * Qm3;
                if constexpr (M >= 4) {
                    float Qm4 = 1.0f;
#pragma unroll
                    for (int e = 0; e < M - 4; ++e) Qm4 *= Q;
                    t4 += (16.0f * M * (M - 1) * (M - 2) * (M - 3)) * u2 * u2 * Qm4;
                }
                d4[q] = ok ? t4 * ((a1 * a1) * (a1 * a1)) : 0.0f;
            }
            if constexpr (NDER >= 5) {
                float t5 = 0.0f;
                if constexpr (M >= 3) t5 -= (120.0f * falling(M, 3)) * u * qpow<M - 3>(Q);
                if constexpr (M >= 4) t5 += (160.0f * falling(M, 4)) * u2 * u * qpow<M - 4>(Q);
                if constexpr (M >= 5) t5 -= (32.0f * falling(M, 5)) * (u2 * u2) * u * qpow<M - 5>(Q);
                d5[q] = ok ? t5 * ((a1 * a1) * (a1 * a1) * a1) : 0.0f;
            }
            if constexpr (NDER >= 6) {
                float t6 = 0.0f;
                if constexpr (M >= 3) t6 -= (120.0f * falling(M, 3)) * qpow<M - 3>(Q);
                if constexpr (M >= 4) t6 += (720.0f * falling(M, 4)) * u2 * qpow<M - 4>(Q);
                if constexpr (M >= 5) t6 -= (480.0f * falling(M, 5)) * (u2 * u2) * qpow<M - 5>(Q);
                if constexpr (M >= 6) t6 += (64.0f * falling(M, 6)) * (u2 * u2) * u2 * qpow<M - 6>(Q);
                d6[q] = ok ? t6 * ((a1 * a1) * (a1 * a1) * (a1 * a1)) : 0.0f;
            }
        }
    }
};

// Jet-row structure selected by a mask over D = 2 input dimensions:
// bit 0 = value, bit 1+d = first derivative along d, bit 3+d = second
// derivative along d (which needs the first along d), bit 5+d = third
// derivative along d (which needs the first and second), bit 7 = the mixed
// derivative u_x0x1 (which needs both first derivatives), bit 8+d = fourth
// derivative along d (which needs the third), bit 10+d = fifth derivative
// along d (which needs the fourth).  Rows are in bit order.
template <unsigned MASK>
struct Jet {
    static constexpr bool F0 = (MASK >> 1) & 1, F1 = (MASK >> 2) & 1;
    static constexpr bool S0 = (MASK >> 3) & 1, S1 = (MASK >> 4) & 1;
    static constexpr bool T0 = (MASK >> 5) & 1, T1 = (MASK >> 6) & 1;
    static constexpr bool X01 = (MASK >> 7) & 1;
    static constexpr bool P0 = (MASK >> 8) & 1, P1 = (MASK >> 9) & 1;     // fourth derivatives
    static constexpr bool Q0 = (MASK >> 10) & 1, Q1 = (MASK >> 11) & 1;   // fifth derivatives
    static_assert(MASK & 1, "the value row is always present");
    static_assert((MASK >> 12) == 0, "two inputs have twelve jet bits");
    static_assert(!S0 || F0, "u_x0x0 needs u_x0");
    static_assert(!S1 || F1, "u_x1x1 needs u_x1");
    static_assert(!T0 || S0, "u_x0x0x0 needs u_x0x0");
    static_assert(!T1 || S1, "u_x1x1x1 needs u_x1x1");
    static_assert(!X01 || (F0 && F1), "u_x0x1 needs u_x0 and u_x1");
    static_assert(!P0 || T0, "the fourth derivative along x0 needs the third");
    static_assert(!P1 || T1, "the fourth derivative along x1 needs the third");
    static_assert(!Q0 || P0, "the fifth derivative along x0 needs the fourth");
    static_assert(!Q1 || P1, "the fifth derivative along x1 needs the fourth");
    static constexpr int NF = int(F0) + int(F1);
    static constexpr int NS = int(S0) + int(S1);
    static constexpr int NT = int(T0) + int(T1);
    static constexpr int NP = int(P0) + int(P1);
    static constexpr int NQ = int(Q0) + int(Q1);
    static constexpr int J = 1 + NF + NS + NT + int(X01) + NP + NQ;
    static constexpr int RF0 = 1, RF1 = 1 + int(F0);
    static constexpr int RS0 = 1 + NF, RS1 = 1 + NF + int(S0);
    static constexpr int RT0 = 1 + NF + NS, RT1 = 1 + NF + NS + int(T0);
    static constexpr int RX = 1 + NF + NS + NT;
    static constexpr int RP0 = RX + int(X01), RP1 = RP0 + int(P0);
    static constexpr int RQ0 = RP0 + NP, RQ1 = RQ0 + int(Q0);
    // rows beyond the PDE masks' value / first / second derivatives
    static constexpr bool GENERAL = NT > 0 || X01 || NP > 0;
    // the fourth / fifth derivative rows
    static constexpr bool HIGH = NP > 0;
    // basis derivatives the rows need, and their reverse (one more)
    static constexpr int NDER_ROWS = NQ ? 5 : NP ? 4 : NT ? 3 : 2;
    static constexpr int NDER_ADJ = NDER_ROWS + 1;

    // Rows of the basis matrix A for one input unit with jets z[J] and the
    // active basis values (v, v', v'') of its value z[0]:
    //   value row  v
    //   d-row      v' z_d
    //   dd-row     v'' z_d^2 + v' z_dd
    template <int KP>
    __host__ __device__ __forceinline__ static void rows(const float* z, const float* v, const float* d1,
                                                const float* d2, float (*a)[KP]) {
        static_assert(!GENERAL, "third-derivative or mixed rows: use rows_b");
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            a[0][q] = v[q];
            if constexpr (F0) a[RF0][q] = d1[q] * z[RF0];
            if constexpr (F1) a[RF1][q] = d1[q] * z[RF1];
            if constexpr (S0) a[RS0][q] = fmaf(d2[q] * z[RF0], z[RF0], d1[q] * z[RS0]);
            if constexpr (S1) a[RS1][q] = fmaf(d2[q] * z[RF1], z[RF1], d1[q] * z[RS1]);
        }
    }

    // Reverse of rows(): given dA[r][q] = dL/dA (rows of one input unit) and
    // the active basis values including v''', accumulate dL/dz[J] for the
    // unit's jets:
    //   dz      += sum_q dA0 v' + dAd v'' z_d + dAdd (v''' z_d^2 + v'' z_dd)
    //   dz_d    += sum_q dAd v' + dAdd 2 v'' z_d
    //   dz_dd   += sum_q dAdd v'
    template <int KP>
    __host__ __device__ __forceinline__ static void rows_adjoint(const float* z, const float* d1,
                                                        const float* d2, const float* d3,
                                                        const float (*dA)[KP], float* gz) {
        static_assert(!GENERAL, "third-derivative or mixed rows: use adjoint_b");
#pragma unroll
        for (int r = 0; r < J; ++r) gz[r] = 0.0f;
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            float g0 = dA[0][q] * d1[q];
            if constexpr (F0) {
                g0 = fmaf(dA[RF0][q] * d2[q], z[RF0], g0);
                gz[RF0] = fmaf(dA[RF0][q], d1[q], gz[RF0]);
            }
            if constexpr (F1) {
                g0 = fmaf(dA[RF1][q] * d2[q], z[RF1], g0);
                gz[RF1] = fmaf(dA[RF1][q], d1[q], gz[RF1]);
            }
            if constexpr (S0) {
                g0 = fmaf(dA[RS0][q], fmaf(d3[q] * z[RF0], z[RF0], d2[q] * z[RS0]), g0);
                gz[RF0] = fmaf(dA[RS0][q] * 2.0f * d2[q], z[RF0], gz[RF0]);
                gz[RS0] = fmaf(dA[RS0][q], d1[q], gz[RS0]);
            }
            if constexpr (S1) {
                g0 = fmaf(dA[RS1][q], fmaf(d3[q] * z[RF1], z[RF1], d2[q] * z[RS1]), g0);
                gz[RF1] = fmaf(dA[RS1][q] * 2.0f * d2[q], z[RF1], gz[RF1]);
                gz[RS1] = fmaf(dA[RS1][q], d1[q], gz[RS1]);
            }
            gz[0] += g0;
        }
    }

    // rows_adjoint() taken one row of dA at a time: the map is linear in dA, so
    // row r's terms (a[q] = dA[r][q]) can be added to gz as soon as that row is
    // known, and no row needs to be kept.  Summed over r = 0..J-1 it gives
    // rows_adjoint() up to the order of the float additions.
    template <int KP>
    __host__ __device__ __forceinline__ static void row_adjoint(int r, const float* z, const float* d1,
                                                       const float* d2, const float* d3, const float* a,
                                                       float* gz) {
        static_assert(!GENERAL, "value, first and second derivative rows only");
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            if (r == 0) gz[0] = fmaf(a[q], d1[q], gz[0]);
            if constexpr (F0)
                if (r == RF0) {
                    gz[0] = fmaf(a[q] * d2[q], z[RF0], gz[0]);
                    gz[RF0] = fmaf(a[q], d1[q], gz[RF0]);
                }
            if constexpr (F1)
                if (r == RF1) {
                    gz[0] = fmaf(a[q] * d2[q], z[RF1], gz[0]);
                    gz[RF1] = fmaf(a[q], d1[q], gz[RF1]);
                }
            if constexpr (S0)
                if (r == RS0) {
                    gz[0] = fmaf(a[q], fmaf(d3[q] * z[RF0], z[RF0], d2[q] * z[RS0]), gz[0]);
                    gz[RF0] = fmaf(a[q] * 2.0f * d2[q], z[RF0], gz[RF0]);
                    gz[RS0] = fmaf(a[q], d1[q], gz[RS0]);
                }
            if constexpr (S1)
                if (r == RS1) {
                    gz[0] = fmaf(a[q], fmaf(d3[q] * z[RF1], z[RF1], d2[q] * z[RS1]), gz[0]);
                    gz[RF1] = fmaf(a[q] * 2.0f * d2[q], z[RF1], gz[RF1]);
                    gz[RS1] = fmaf(a[q], d1[q], gz[RS1]);
                }
        }
    }

    // rows() plus the third-derivative rows (needs v''') and the mixed row:
    //   ddd-row    v''' z_d^3 + 3 v'' z_d z_dd + v' z_ddd
    //   01-row     v'' z_0 z_1 + v' z_01
    template <int KP>
    __host__ __device__ __forceinline__ static void rows3(const float* z, const float* v, const float* d1,
                                                 const float* d2, const float* d3, float (*a)[KP]) {
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            a[0][q] = v[q];
            if constexpr (F0) a[RF0][q] = d1[q] * z[RF0];
            if constexpr (F1) a[RF1][q] = d1[q] * z[RF1];
            if constexpr (S0) a[RS0][q] = fmaf(d2[q] * z[RF0], z[RF0], d1[q] * z[RS0]);
            if constexpr (S1) a[RS1][q] = fmaf(d2[q] * z[RF1], z[RF1], d1[q] * z[RS1]);
            if constexpr (T0)
                a[RT0][q] = fmaf(d3[q] * z[RF0] * z[RF0], z[RF0],
                                 fmaf(3.0f * d2[q] * z[RF0], z[RS0], d1[q] * z[RT0]));
            if constexpr (T1)
                a[RT1][q] = fmaf(d3[q] * z[RF1] * z[RF1], z[RF1],
                                 fmaf(3.0f * d2[q] * z[RF1], z[RS1], d1[q] * z[RT1]));
            if constexpr (X01) a[RX][q] = fmaf(d2[q] * z[RF0], z[RF1], d1[q] * z[RX]);
        }
    }

    // rows_adjoint() plus the reverse of the third-derivative rows (needs v'''')
    // and of the mixed row:
    //   dz      += dAddd (v'''' z_d^3 + 3 v''' z_d z_dd + v'' z_ddd) + dA01 (v''' z_0 z_1 + v'' z_01)
    //   dz_d    += dAddd (3 v''' z_d^2 + 3 v'' z_dd) + dA01 v'' z_(1-d)
    //   dz_dd   += dAddd 3 v'' z_d
    //   dz_ddd  += dAddd v'
    //   dz_01   += dA01 v'
    template <int KP>
    __host__ __device__ __forceinline__ static void rows_adjoint3(const float* z, const float* d1, const float* d2,
                                                         const float* d3, const float* d4,
                                                         const float (*dA)[KP], float* gz) {
#pragma unroll
        for (int r = 0; r < J; ++r) gz[r] = 0.0f;
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            float g0 = dA[0][q] * d1[q];
            if constexpr (F0) {
                g0 = fmaf(dA[RF0][q] * d2[q], z[RF0], g0);
                gz[RF0] = fmaf(dA[RF0][q], d1[q], gz[RF0]);
            }
            if constexpr (F1) {
                g0 = fmaf(dA[RF1][q] * d2[q], z[RF1], g0);
                gz[RF1] = fmaf(dA[RF1][q], d1[q], gz[RF1]);
            }
            if constexpr (S0) {
                g0 = fmaf(dA[RS0][q], fmaf(d3[q] * z[RF0], z[RF0], d2[q] * z[RS0]), g0);
                gz[RF0] = fmaf(dA[RS0][q] * 2.0f * d2[q], z[RF0], gz[RF0]);
                gz[RS0] = fmaf(dA[RS0][q], d1[q], gz[RS0]);
            }
            if constexpr (S1) {
                g0 = fmaf(dA[RS1][q], fmaf(d3[q] * z[RF1], z[RF1], d2[q] * z[RS1]), g0);
                gz[RF1] = fmaf(dA[RS1][q] * 2.0f * d2[q], z[RF1], gz[RF1]);
                gz[RS1] = fmaf(dA[RS1][q], d1[q], gz[RS1]);
            }
            if constexpr (T0) {
                const float g = dA[RT0][q], zd = z[RF0], zdd = z[RS0], zddd = z[RT0];
                g0 = fmaf(g, fmaf(d4[q] * zd * zd, zd, fmaf(3.0f * d3[q] * zd, zdd, d2[q] * zddd)), g0);
                gz[RF0] = fmaf(g, fmaf(3.0f * d3[q] * zd, zd, 3.0f * d2[q] * zdd), gz[RF0]);
                gz[RS0] = fmaf(g * 3.0f * d2[q], zd, gz[RS0]);
                gz[RT0] = fmaf(g, d1[q], gz[RT0]);
            }
            if constexpr (T1) {
                const float g = dA[RT1][q], zd = z[RF1], zdd = z[RS1], zddd = z[RT1];
                g0 = fmaf(g, fmaf(d4[q] * zd * zd, zd, fmaf(3.0f * d3[q] * zd, zdd, d2[q] * zddd)), g0);
                gz[RF1] = fmaf(g, fmaf(3.0f * d3[q] * zd, zd, 3.0f * d2[q] * zdd), gz[RF1]);
                gz[RS1] = fmaf(g * 3.0f * d2[q], zd, gz[RS1]);
                gz[RT1] = fmaf(g, d1[q], gz[RT1]);
            }
            if constexpr (X01) {
                const float g = dA[RX][q];
                g0 = fmaf(g, fmaf(d3[q] * z[RF0], z[RF1], d2[q] * z[RX]), g0);
                gz[RF0] = fmaf(g * d2[q], z[RF1], gz[RF0]);
                gz[RF1] = fmaf(g * d2[q], z[RF0], gz[RF1]);
                gz[RX] = fmaf(g, d1[q], gz[RX]);
            }
            gz[0] += g0;
        }
    }

    // Fourth and fifth derivatives of v(z(x)) along one input from the
    // derivatives f1..f5 of v at z and the jets g1..g5 of z along that input
    // (Faa di Bruno's formula):
    //   4-row  f4 g1^4 + 6 f3 g1^2 g2 + f2 (3 g2^2 + 4 g1 g3) + f1 g4
    //   5-row  f5 g1^5 + 10 f4 g1^3 g2 + f3 (15 g1 g2^2 + 10 g1^2 g3)
    //          + f2 (10 g2 g3 + 5 g1 g4) + f1 g5
    // d/dz of a row is the same polynomial with every f_r moved to f_{r+1}.
    __host__ __device__ __forceinline__ static float row4(float f1, float f2, float f3, float f4, float g1,
                                                          float g2, float g3, float g4) {
        const float g11 = g1 * g1;
        float r = fmaf(f4 * g11, g11, 6.0f * f3 * g11 * g2);
        r = fmaf(f2, fmaf(3.0f * g2, g2, 4.0f * g1 * g3), r);
        return fmaf(f1, g4, r);
    }
    __host__ __device__ __forceinline__ static float row5(float f1, float f2, float f3, float f4, float f5,
                                                          float g1, float g2, float g3, float g4, float g5) {
        const float g11 = g1 * g1;
        float r = fmaf(f5 * g11 * g11, g1, 10.0f * f4 * g11 * g1 * g2);
        r = fmaf(f3, fmaf(15.0f * g1 * g2, g2, 10.0f * g11 * g3), r);
        r = fmaf(f2, fmaf(10.0f * g2, g3, 5.0f * g1 * g4), r);
        return fmaf(f1, g5, r);
    }

    // The fourth / fifth derivative rows of rows3's layout (bits 8..11).
    template <int KP, class B>
    __host__ __device__ __forceinline__ static void rows_high(const float* z, const B& b, float (*a)[KP]) {
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            if constexpr (P0) a[RP0][q] = row4(b.d1[q], b.d2[q], b.d3[q], b.d4[q], z[RF0], z[RS0], z[RT0], z[RP0]);
            if constexpr (P1) a[RP1][q] = row4(b.d1[q], b.d2[q], b.d3[q], b.d4[q], z[RF1], z[RS1], z[RT1], z[RP1]);
            if constexpr (Q0)
                a[RQ0][q] = row5(b.d1[q], b.d2[q], b.d3[q], b.d4[q], b.d5[q], z[RF0], z[RS0], z[RT0], z[RP0], z[RQ0]);
            if constexpr (Q1)
                a[RQ1][q] = row5(b.d1[q], b.d2[q], b.d3[q], b.d4[q], b.d5[q], z[RF1], z[RS1], z[RT1], z[RP1], z[RQ1]);
        }
    }

    // Reverse of one input direction's 4-row (weight g4r = dL/dA) and 5-row
    // (g5r; 0 without one) into the gradients of z and its jets g1..g5:
    //   4-row: dg1 4 f4 g1^3 + 12 f3 g1 g2 + 4 f2 g3, dg2 6 f3 g1^2 + 6 f2 g2,
    //          dg3 4 f2 g1, dg4 f1
    //   5-row: dg1 5 f5 g1^4 + 30 f4 g1^2 g2 + f3 (15 g2^2 + 20 g1 g3) + 5 f2 g4,
    //          dg2 10 f4 g1^3 + 30 f3 g1 g2 + 10 f2 g3, dg3 10 f3 g1^2 + 10 f2 g2,
    //          dg4 5 f2 g1, dg5 f1
    template <bool FIFTH>
    __host__ __device__ __forceinline__ static void high_adjoint(const float* f, float g4r, float g5r,
                                                                 const float* g, float& gz0, float* gg) {
        const float g1 = g[1], g2 = g[2], g3 = g[3], g4 = g[4], g11 = g1 * g1;
        gz0 = fmaf(g4r, row4(f[2], f[3], f[4], f[5], g1, g2, g3, g4), gz0);
        gg[1] = fmaf(g4r, fmaf(4.0f * f[4] * g11, g1, fmaf(12.0f * f[3] * g1, g2, 4.0f * f[2] * g3)), gg[1]);
        gg[2] = fmaf(g4r, fmaf(6.0f * f[3], g11, 6.0f * f[2] * g2), gg[2]);
        gg[3] = fmaf(g4r * 4.0f * f[2], g1, gg[3]);
        gg[4] = fmaf(g4r, f[1], gg[4]);
        if constexpr (FIFTH) {
            const float g5 = g[5];
            gz0 = fmaf(g5r, row5(f[2], f[3], f[4], f[5], f[6], g1, g2, g3, g4, g5), gz0);
            float t = fmaf(5.0f * f[5] * g11, g11, 30.0f * f[4] * g11 * g2);
            t = fmaf(f[3], fmaf(15.0f * g2, g2, 20.0f * g1 * g3), t);
            gg[1] = fmaf(g5r, fmaf(5.0f * f[2], g4, t), gg[1]);
            gg[2] = fmaf(g5r, fmaf(10.0f * f[4] * g11, g1, fmaf(30.0f * f[3] * g1, g2, 10.0f * f[2] * g3)), gg[2]);
            gg[3] = fmaf(g5r, fmaf(10.0f * f[3], g11, 10.0f * f[2] * g2), gg[3]);
            gg[4] = fmaf(g5r * 5.0f * f[2], g1, gg[4]);
            gg[5] = fmaf(g5r, f[1], gg[5]);
        }
    }

    // Reverse of rows_high(), added to gz (rows_adjoint3 zeroes and fills the rest first).
    template <int KP, class B>
    __host__ __device__ __forceinline__ static void adjoint_high(const float* z, const B& b, const float (*dA)[KP],
                                                                 float* gz) {
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            const float f[7] = {b.v[q], b.d1[q], b.d2[q], b.d3[q], b.d4[q],
                                NDER_ADJ >= 5 ? b.d5[q] : 0.0f, NDER_ADJ >= 6 ? b.d6[q] : 0.0f};
            if constexpr (P0) {
                const float g[6] = {0.0f, z[RF0], z[RS0], z[RT0], z[RP0], Q0 ? z[RQ0] : 0.0f};
                float gg[6] = {0.0f, gz[RF0], gz[RS0], gz[RT0], gz[RP0], Q0 ? gz[RQ0] : 0.0f};
                high_adjoint<Q0>(f, dA[RP0][q], Q0 ? dA[RQ0][q] : 0.0f, g, gz[0], gg);
                gz[RF0] = gg[1]; gz[RS0] = gg[2]; gz[RT0] = gg[3]; gz[RP0] = gg[4];
                if constexpr (Q0) gz[RQ0] = gg[5];
            }
            if constexpr (P1) {
                const float g[6] = {0.0f, z[RF1], z[RS1], z[RT1], z[RP1], Q1 ? z[RQ1] : 0.0f};
                float gg[6] = {0.0f, gz[RF1], gz[RS1], gz[RT1], gz[RP1], Q1 ? gz[RQ1] : 0.0f};
                high_adjoint<Q1>(f, dA[RP1][q], Q1 ? dA[RQ1][q] : 0.0f, g, gz[0], gg);
                gz[RF1] = gg[1]; gz[RS1] = gg[2]; gz[RT1] = gg[3]; gz[RP1] = gg[4];
                if constexpr (Q1) gz[RQ1] = gg[5];
            }
        }
    }

    // The rows / their reverse for a basis evaluation b (Active<K, M, NDER_ROWS> /
    // Active<K, M, NDER_ADJ>): the PDE masks keep the second-order formulas.
    template <int KP, class B>
    __host__ __device__ __forceinline__ static void rows_b(const float* z, const B& b, float (*a)[KP]) {
        if constexpr (!GENERAL) rows<KP>(z, b.v, b.d1, b.d2, a);
        else rows3<KP>(z, b.v, b.d1, b.d2, b.d3, a);
        if constexpr (HIGH) rows_high<KP>(z, b, a);
    }
    template <int KP, class B>
    __host__ __device__ __forceinline__ static void adjoint_b(const float* z, const B& b, const float (*dA)[KP], float* gz) {
        if constexpr (!GENERAL) rows_adjoint<KP>(z, b.d1, b.d2, b.d3, dA, gz);
        else rows_adjoint3<KP>(z, b.d1, b.d2, b.d3, b.d4, dA, gz);
        if constexpr (HIGH) adjoint_high<KP>(z, b, dA, gz);
    }
};

// Residual of one interior point and dL/d(jets) (Eq. 4, Eq. 8):
//   Poisson: r = u_xx + u_yy + (a^2+b^2) pi^2 sin(a pi x) sin(b pi y)
//   Burgers: r = u_t + lam u u_x - nu u_xx
//   KdV:     r = u_t + lam u u_x + nu u_xxx (a third-order equation, mask 0x2F)
// gu[r] = dL/d jet row r for L = alpha mean(r^2): scale = 2 alpha / N_int.
struct PdeParams {
    int kind;
    float a, b, src;   // src = (a^2 + b^2) pi^2
    float lam, nu;
    float alpha;
};

template <unsigned MASK>
__host__ __device__ __forceinline__ float pde_residual(const PdeParams& P, float x0, float x1, const float* u) {
    using JT = Jet<MASK>;
    if (P.kind == 0) {
        if constexpr (JT::S0 && JT::S1) {
            float f = P.src * sinpif(P.a * x0) * sinpif(P.b * x1);
            return u[JT::RS0] + u[JT::RS1] + f;
        }
        return 0.0f;
    } else if (P.kind == 1) {
        if constexpr (JT::F0 && JT::F1 && JT::S0) {
            return u[JT::RF1] + P.lam * u[0] * u[JT::RF0] - P.nu * u[JT::RS0];
        }
        return 0.0f;
    } else {
        if constexpr (JT::F0 && JT::F1 && JT::T0) {
            return u[JT::RF1] + P.lam * u[0] * u[JT::RF0] + P.nu * u[JT::RT0];
        }
        return 0.0f;
    }
}

template <unsigned MASK>
__host__ __device__ __forceinline__ void pde_residual_grad(const PdeParams& P, float r, const float* u,
                                                  float scale, float* gu) {
    using JT = Jet<MASK>;
#pragma unroll
    for (int q = 0; q < JT::J; ++q) gu[q] = 0.0f;
    float g = scale * r;
    if (P.kind == 0) {
        if constexpr (JT::S0 && JT::S1) { gu[JT::RS0] = g; gu[JT::RS1] = g; }
    } else if (P.kind == 1) {
        if constexpr (JT::F0 && JT::F1 && JT::S0) {
            gu[JT::RF1] = g;
            gu[0] = g * P.lam * u[JT::RF0];
            gu[JT::RF0] = g * P.lam * u[0];
            gu[JT::RS0] = -g * P.nu;
        }
    } else {
        if constexpr (JT::F0 && JT::F1 && JT::T0) {
            gu[JT::RF1] = g;
            gu[0] = g * P.lam * u[JT::RF0];
            gu[JT::RF0] = g * P.lam * u[0];
            gu[JT::RT0] = g * P.nu;
        }
    }
}

// Masks for which a residual exists: Poisson u_xx, u_yy; Burgers u, u_x, u_t,
// u_xx; KdV u, u_x, u_t, u_xxx.
__host__ __device__ constexpr bool mask_has_rows(unsigned mask, int kind) {
    return kind == 0   ? ((mask & 0x18u) == 0x18u)
           : kind == 1 ? ((mask & 0x0Fu) == 0x0Fu)
           : kind == 2 ? ((mask & 0x27u) == 0x27u)
                       : ((mask & 0x70u) == 0x70u);   // three inputs: u_xx, u_yy, u_zz
}

// The interior jet mask the training step uses for a problem kind.
// (three inputs, kind 3: every row up to the second derivatives, 0x7F)
__host__ __device__ constexpr unsigned pde_mask(int kind) {
    return kind == 0 ? 0x1Fu : kind == 1 ? 0x0Fu : kind == 2 ? 0x2Fu : 0x7Fu;
}

}  // namespace hrkan
