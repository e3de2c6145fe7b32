// Device building blocks of the HRKAN hot path: the HR basis with its first
// four derivatives on the k+1 active supports (Section 3, Eq. 2), and the
// jet-row structure that the PDE residuals need (Eq. 3: the Laplacian; Eq. 6:
// u_t, u_x, u_xx).  The basis evaluation and the row formulas are also
// callable on the host, where a test compares them with the FP64 oracle.
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
// A basis index outside [0, n) gets all-zero values and a clamped index.
template <int K, int M, int NDER>
struct Active {
    int c;               // first active basis index (may be < 0 or > n-1-K)
    float v[K + 1];      // v_{c+q}(z)
    float d1[K + 1];     // v'
    float d2[K + 1];     // v''
    float d3[K + 1];     // v''' (only when NDER >= 3)
    float d4[K + 1];     // v'''' (only when NDER >= 4)

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
        }
    }
};

// Jet-row structure selected by a mask over D = 2 input dimensions:
// bit 0 = value, bit 1+d = first derivative along d, bit 3+d = second
// derivative along d (which needs the first along d), bit 5+d = third
// derivative along d (which needs the first and second), bit 7 = the mixed
// derivative u_x0x1 (which needs both first derivatives).  Rows are in bit order.
template <unsigned MASK>
struct Jet {
    static constexpr bool F0 = (MASK >> 1) & 1, F1 = (MASK >> 2) & 1;
    static constexpr bool S0 = (MASK >> 3) & 1, S1 = (MASK >> 4) & 1;
    static constexpr bool T0 = (MASK >> 5) & 1, T1 = (MASK >> 6) & 1;
    static constexpr bool X01 = (MASK >> 7) & 1;
    static_assert(MASK & 1, "the value row is always present");
    static_assert(!S0 || F0, "u_x0x0 needs u_x0");
    static_assert(!S1 || F1, "u_x1x1 needs u_x1");
    static_assert(!T0 || S0, "u_x0x0x0 needs u_x0x0");
    static_assert(!T1 || S1, "u_x1x1x1 needs u_x1x1");
    static_assert(!X01 || (F0 && F1), "u_x0x1 needs u_x0 and u_x1");
    static constexpr int NF = int(F0) + int(F1);
    static constexpr int NS = int(S0) + int(S1);
    static constexpr int NT = int(T0) + int(T1);
    static constexpr int J = 1 + NF + NS + NT + int(X01);
    static constexpr int RF0 = 1, RF1 = 1 + int(F0);
    static constexpr int RS0 = 1 + NF, RS1 = 1 + NF + int(S0);
    static constexpr int RT0 = 1 + NF + NS, RT1 = 1 + NF + NS + int(T0);
    static constexpr int RX = 1 + NF + NS + NT;
    // rows beyond the PDE masks' value / first / second derivatives
    static constexpr bool GENERAL = NT > 0 || X01;
    // basis derivatives the rows need, and their reverse (one more)
    static constexpr int NDER_ROWS = NT ? 3 : 2;
    static constexpr int NDER_ADJ = NT ? 4 : 3;

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

    // The rows / their reverse for a basis evaluation b (Active<K, M, NDER_ROWS> /
    // Active<K, M, NDER_ADJ>): the PDE masks keep the second-order formulas.
    template <int KP, class B>
    __host__ __device__ __forceinline__ static void rows_b(const float* z, const B& b, float (*a)[KP]) {
        if constexpr (!GENERAL) rows<KP>(z, b.v, b.d1, b.d2, a);
        else rows3<KP>(z, b.v, b.d1, b.d2, b.d3, a);
    }
    template <int KP, class B>
    __host__ __device__ __forceinline__ static void adjoint_b(const float* z, const B& b, const float (*dA)[KP], float* gz) {
        if constexpr (!GENERAL) rows_adjoint<KP>(z, b.d1, b.d2, b.d3, dA, gz);
        else rows_adjoint3<KP>(z, b.d1, b.d2, b.d3, b.d4, dA, gz);
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
__device__ __forceinline__ float pde_residual(const PdeParams& P, float x0, float x1, const float* u) {
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
__device__ __forceinline__ void pde_residual_grad(const PdeParams& P, float r, const float* u,
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
    return kind == 0 ? ((mask & 0x18u) == 0x18u) : kind == 1 ? ((mask & 0x0Fu) == 0x0Fu) : ((mask & 0x27u) == 0x27u);
}

// The interior jet mask the training step uses for a problem kind.
__host__ __device__ constexpr unsigned pde_mask(int kind) { return kind == 0 ? 0x1Fu : kind == 1 ? 0x0Fu : 0x2Fu; }

}  // namespace hrkan
