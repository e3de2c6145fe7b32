// Tensor-core (tcgen05 / TMEM / TMA) contraction of the stacked jet rows with
// the layer weights, for the hidden layers of wide networks (Sections 1-3:
// the KAN layer as a matrix operation; Eq. 2 bases).
//
//   Y_r[p, o] = sum_k A_r[p, k] W[o, k],   r = 0..J-1 jet rows
//
// K runs over the layer's input units, each padded to NP elements (basis i of
// unit j at k = j*NP + (i mod 4)*NP/4 + i/4; W and A are zero for i >= n).  Per point and unit only the
// k+1 = 4 bases c..c+3 are non-zero, so A is built on the fly, never stored.
//
// One persistent CTA per SM walks tiles of 128 points (the MMA's M); every jet
// row has an FP32 accumulator of 128 x O in TMEM (N = O).  Warp roles:
//   warps 0-3  producers: thread = point = TMEM lane (with PARTS > 1, warps
//              w, w+4, ... share the lanes of quarter w and split the units).  For
//              each slot of 16 BF16 (8 TF32) K elements they write the point's A
//              words of every jet row into a ring of slots in TMEM
//              (tcgen05.st), then run the tile's epilogue (tcgen05.ld -> y);
//   next warp  one thread issues, per slot, J tcgen05.mma (A from TMEM, B = W
//              from shared memory) and commits them to the slot's "empty" barrier;
//   last warp  one thread streams W tiles of 128 bytes per row into a ring of
//              shared-memory buffers with TMA (128-byte swizzle, K-major).
// The placement of the 4 non-zeros is the cost that matters: with NP fixed at
// compile time, the unit and word offset of every word of a slot are constants
// of an unrolled period of slots; the bases of a unit are stored by residue
// mod 4 (four quarters), so every word holds at most one non-zero and a word of
// one jet row costs one select.
//
// Every mbarrier wait is bounded (~1 s) and also gives up when another role has
// given up: the CTA then records HRKAN_ETIMEOUT in a device status word, waits
// (bounded) for its own copies and MMAs, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "tc.cuh"

namespace hrkan {
namespace tck {

constexpr int TILE_M = 128;
constexpr int NB = TC_W_BUFFERS;  // W tiles (4 slots each) in flight
constexpr int RS_MAX = 8;        // A ring slots
constexpr int PARTS = 1;                  // producer warps per TMEM lane quarter
constexpr int PRODUCER_WARPS = 4 * PARTS;
constexpr int THREADS = 32 * PRODUCER_WARPS + 64;   // producer warps, the MMA warp, the TMA warp
constexpr long long WAIT_CYCLES = 2000000000LL;   // ~1 s at 2 GHz
constexpr int ERR_TIMEOUT = -5;                   // HRKAN_ETIMEOUT

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity.  Gives up (false) after `limit`
// cycles, raising *abort, or as soon as *abort is raised by another thread.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          long long limit = WAIT_CYCLES) {
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > limit) {
            *abort = 1;
            return false;
        }
    }
    return true;
}
// The handle's device status block is int[4]: [0] the error word the kernels
// set, [2..3] the limit of their waits in clock cycles (int64; 0 = WAIT_CYCLES).
// A small limit makes the waits give up early (fault-injection tests); the
// drains on the way out keep WAIT_CYCLES.
__device__ __forceinline__ long long wait_limit(const int* status) {
    const long long w = *reinterpret_cast<const volatile long long*>(status + 2);
    return w > 0 ? w : WAIT_CYCLES;
}

// Bounded wait that ignores *abort (draining own work on the way out).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > WAIT_CYCLES) return;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFF) >> 4);      // start address
    d |= uint64_t(1) << 16;                     // leading byte offset (unused for swizzled K-major)
    d |= uint64_t(1024 >> 4) << 32;             // stride byte offset: next 8-row group
    d |= uint64_t(1) << 46;                     // descriptor version
    d |= uint64_t(2) << 61;                     // layout: 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulate, A/B format fmt (1 = BF16 under
// kind::f16, 2 = TF32 under kind::tf32), both K-major, M = 128, N.
__host__ __device__ constexpr uint32_t idesc_of(int fmt, int N) {
    return (1u << 4) | (uint32_t(fmt) << 7) | (uint32_t(fmt) << 10) | (uint32_t(N >> 3) << 17) |
           (uint32_t(TILE_M >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    if constexpr (PREC == HRKAN_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

// Element type of the contraction.  An "element" is one basis position of
// the K layout; TERMS is the number of MMAs per slot and jet row (and of
// O-row weight tiles per W buffer).
template <int PREC>
struct Elem;
template <>
struct Elem<HRKAN_BF16> {
    static constexpr int PER_WORD = 2;   // elements per 32-bit word (TMEM column)
    static constexpr int SLOT = 16;      // K elements per MMA (one slot)
    static constexpr int BOX = 64;       // K elements per 128-byte W row tile
    static constexpr int FMT = 1;
    static constexpr int TERMS = 1;
};
template <>
struct Elem<HRKAN_TF32> {
    static constexpr int PER_WORD = 1, SLOT = 8, BOX = 32, FMT = 2, TERMS = 1;
};
// Three-term BF16 split in a pair layout: the 32-bit word of a basis holds
// (a_hi, a_lo) in its low and high halves, the two weight tiles hold
// (w_hi, w_hi) and (w_lo, 0) per basis, so the two BF16 MMAs of a slot add
// a_hi w_hi + a_lo w_hi and a_hi w_lo.  One basis per word, 8 per slot (the
// MMA's K of 16 BF16 elements), 32 per 128-byte W row.
template <>
struct Elem<TC_BF16X3> {
    static constexpr int PER_WORD = 1, SLOT = 8, BOX = 32, FMT = 1, TERMS = 2;
};

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

// Compile-time shape of the slot stream for units padded to NP elements.
template <int PREC, int NP>
struct Period {
    using E = Elem<PREC>;
    static constexpr int NW = NP / E::PER_WORD;                    // words per unit
    static constexpr int SW = E::SLOT / E::PER_WORD;               // words per slot (8)
    static constexpr int WORDS = NW / gcd_c(NW, SW) * SW;          // lcm(NW, SW)
    static constexpr int PS = WORDS / SW;                          // slots per period
    static constexpr int PU = WORDS / NW;                          // units per period
    static_assert(NP % E::PER_WORD == 0, "a unit starts on a word boundary");
    static_assert(SW == 8, "one slot is 8 TMEM columns");
};

// Within a unit's padded segment of NP elements the bases are stored by
// residue mod 4: basis i sits at element (i mod 4) * NP/4 + floor(i / 4).  The
// k+1 = 4 active bases c..c+3 have distinct residues, so each quarter of the
// segment holds exactly one of them and every 32-bit word of the segment at
// most one non-zero (BF16: in one half of the word).
template <int PREC, int NP>
struct Quarter {
    static constexpr int Q = NP / 4;                            // elements per quarter
    static constexpr int QW = Q / Elem<PREC>::PER_WORD;        // words per quarter
    static_assert(NP % 4 == 0 && Q % Elem<PREC>::PER_WORD == 0, "quarters start on word boundaries");
};

// The non-zero of each quarter of one unit: its word offset inside the quarter
// (out of range: none) and, per jet row, the word holding it.
template <int J>
struct UnitWin {
    int tw[4];
    uint32_t y[J][4];
};

// Active bases (Eq. 2) of the unit value z[0], evaluated directly in quarter
// order, the jet rows of the 4 non-zero columns, rounded to the MMA type.
// With c = 4a + s the cell and f the offset inside it, quarter k holds basis
// c + q_k, q_k = (k - s) mod 4, at element offset a + [k < s] of the quarter;
// its position inside the support is u = (f + 1 - q_k) / 2 (the u-form of Eq. 2
// for k+1 = 4 active bases: v = (1 - u^2)^4, v' = -8u(1 - u^2)^3 / a_s,
// v'' = (-8(1 - u^2)^3 + 48u^2(1 - u^2)^2) / a_s^2 with a_s the half-width).
template <unsigned MASK, int PREC>
__device__ __forceinline__ void unit_window(const float* z, const Grid& g, bool live, UnitWin<Jet<MASK>::J>& w) {
    using JT = Jet<MASK>;
    constexpr int J = JT::J;
    float t = (z[0] - g.lo) * g.inv_h;
    t = fminf(fmaxf(t, -1.0e9f), 1.0e9f);   // keep floorf's result in int range
    const float fc = floorf(t);
    const int c = int(fc);
    const float f = (z[0] - fmaf(fc, g.h, g.lo)) * g.inv_h;   // offset from the knot (see Active)
    const int base = c >> 2, s = c & 3;                        // arithmetic shift: floor also for c < 0
    float v[4], d1[4], d2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int q = (k - s) & 3;
        const float u = (f + float(1 - q)) * 0.5f;
        const float Q = fmaxf(1.0f - u * u, 0.0f);
        const float Q2 = Q * Q, Q3 = Q2 * Q;
        const bool ok = unsigned(c + q) < unsigned(g.n);
        v[k] = ok ? Q3 * Q : 0.0f;
        d1[k] = ok ? -8.0f * u * Q3 * g.inv_a : 0.0f;
        d2[k] = ok ? (-8.0f * Q3 + 48.0f * u * u * Q2) * (g.inv_a * g.inv_a) : 0.0f;
        const int tk = base + (k < s ? 1 : 0);
        if constexpr (Elem<PREC>::PER_WORD == 2) w.tw[k] = live ? (tk >> 1) : -(1 << 24);
        else w.tw[k] = live ? tk : -(1 << 24);
    }
    float a[J][4];
    JT::template rows<4>(z, v, d1, d2, a);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int tk = base + (k < s ? 1 : 0);
#pragma unroll
        for (int r = 0; r < J; ++r) {
            if constexpr (PREC == HRKAN_BF16) {
                w.y[r][k] = uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(a[r][k]))) << ((tk & 1) * 16);
            } else if constexpr (PREC == TC_BF16X3) {
                // hi = bf16(a); a - hi is exact in float32, lo = bf16(a - hi)
                const __nv_bfloat16 hi = __float2bfloat16_rn(a[r][k]);
                const __nv_bfloat16 lo = __float2bfloat16_rn(a[r][k] - __bfloat162float(hi));
                w.y[r][k] = uint32_t(__bfloat16_as_ushort(hi)) | (uint32_t(__bfloat16_as_ushort(lo)) << 16);
            } else {
                w.y[r][k] = tf32_bits(a[r][k]);
            }
        }
    }
    // bases outside [0, n) are zero already; a unit past the layer's inputs places nothing
}

// Work split between the PARTS producer warps of a TMEM lane quarter: warp
// part q takes the units u of a period with u % PARTS == q (the period is
// repeated until it holds a multiple of PARTS units), evaluates only those and
// stores only their words of each slot.
template <int PREC, int NP, int PARTS>
struct Split {
    using PD = Period<PREC, NP>;
    static constexpr int MUL = PARTS / gcd_c(PD::PU, PARTS);
    static constexpr int PU = PD::PU * MUL;
    static constexpr int PS = PD::PS * MUL;
    static constexpr int NW = PD::NW;
};

__device__ __forceinline__ void mbar_arrive_if(uint64_t* bar, bool pred) {
    asm volatile("{\n\t.reg .pred P;\n\tsetp.ne.b32 P, %1, 0;\n\t@P mbarrier.arrive.shared::cta.b64 _, [%0];\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(int(pred))
                 : "memory");
}
__device__ __forceinline__ void tmem_st2(uint32_t taddr, uint32_t a, uint32_t b) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

// Shared state of one CTA.
struct TcShared {
    uint64_t full[RS_MAX], empty[RS_MAX], wfull[NB], wempty[NB];
    uint64_t accfull, accempty, drain;
    uint32_t tmem_base;
    int abort;
};

// One producer warp (part PART of its lane quarter): A words of its units for
// every slot of every tile of this CTA, then its rows of each tile's epilogue.
template <unsigned MASK, int PREC, int NP, int PART>
__device__ __forceinline__ void produce(const TcLayer& p, TcShared& sh, uint32_t tbase, int quarter, int lane) {
    using JT = Jet<MASK>;
    using E = Elem<PREC>;
    using SP = Split<PREC, NP, PARTS>;
    constexpr int J = JT::J, PU = SP::PU, PS = SP::PS, NW = SP::NW, QW = Quarter<PREC, NP>::QW;
    constexpr int HU = PU / PARTS;   // units of this warp per period: u = PARTS * i + PART
    using Win = UnitWin<J>;
    volatile int* abort = &sh.abort;
    const long long wl = wait_limit(p.status);
    const int O = p.O, I = p.I, RS = p.ring, KS = p.ks;
    const int64_t N = p.N;
    const int ntiles = p.ntiles;
    const uint32_t A0 = uint32_t(J * O), RW = uint32_t(RS * 8);
    const uint32_t lane_base = uint32_t(quarter * 32) << 16;
    const int row = quarter * 32 + lane;
    int slot = 0;
    uint32_t ph = 0;        // parity of the current pass over the ring
    int pend_slot = -1;     // slot whose stores still have to be published
    const int nper = (KS + PS - 1) / PS;

    // z of this warp's units of the first period of the CTA's first tile; later
    // periods are loaded one period ahead
    float zn[HU][J];
    {
        const int64_t pt0 = int64_t(blockIdx.x) * TILE_M + row;
        const float* zp0 = p.z + (pt0 < N ? pt0 : N - 1);
#pragma unroll
        for (int i = 0; i < HU; ++i) {
            const int j = PARTS * i + PART;
#pragma unroll
            for (int r = 0; r < J; ++r) zn[i][r] = j < I ? zp0[(int64_t(r) * I + j) * N] : 0.0f;
        }
    }
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int64_t pt = int64_t(tile) * TILE_M + row;
        const bool valid = pt < N;
        const float* zp = p.z + (valid ? pt : N - 1);   // idle lanes compute on a real point, results dropped
        const int64_t ptn = pt + int64_t(gridDim.x) * TILE_M;   // same lane of the next tile
        const float* zpn = p.z + (ptn < N ? ptn : N - 1);
        for (int per = 0; per < nper; ++per) {
            float zc[HU][J];
#pragma unroll
            for (int i = 0; i < HU; ++i)
#pragma unroll
                for (int r = 0; r < J; ++r) zc[i][r] = zn[i][r];
            if (per + 1 < nper) {
#pragma unroll
                for (int i = 0; i < HU; ++i) {
                    const int j = (per + 1) * PU + PARTS * i + PART;
#pragma unroll
                    for (int r = 0; r < J; ++r) zn[i][r] = j < I ? zp[(int64_t(r) * I + j) * N] : 0.0f;
                }
            } else if (tile + int(gridDim.x) < ntiles) {
#pragma unroll
                for (int i = 0; i < HU; ++i) {
                    const int j = PARTS * i + PART;
#pragma unroll
                    for (int r = 0; r < J; ++r) zn[i][r] = j < I ? zpn[(int64_t(r) * I + j) * N] : 0.0f;
                }
            }
            Win uw[HU];
#pragma unroll
            for (int S = 0; S < PS; ++S) {
                // this warp's units whose first word falls in this slot are evaluated here
#pragma unroll
                for (int i = 0; i < HU; ++i)
                    if (((PARTS * i + PART) * NW) / 8 == S)
                        unit_window<MASK, PREC>(zc[i], p.g, per * PU + PARTS * i + PART < I, uw[i]);
                const int t = per * PS + S;
                if (t < KS) {
                    // own(w): word w of this slot belongs to a unit of this warp (a constant)
                    uint32_t v[J][8];
#pragma unroll
                    for (int w = 0; w < 8; ++w) {
                        const int gw = S * 8 + w, u = gw / NW, lw = gw % NW;
                        if (u % PARTS == PART) {
                            const int i = u / PARTS;
                            // word lw of the unit: quarter lw / QW, holding that quarter's
                            // non-zero when its offset is lw % QW
                            const int qr = lw / QW, qo = lw % QW;
                            const bool hit = uw[i].tw[qr] == qo;
#pragma unroll
                            for (int r = 0; r < J; ++r) v[r][w] = hit ? uw[i].y[r][qr] : 0u;
                        }
                    }
                    if (pend_slot >= 0) {   // publish the previous slot (its stores had time to land)
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        tc_fence_before();
                        __syncwarp();
                        mbar_arrive_if(&sh.full[pend_slot], lane == 0);
                    }
                    if (!__all_sync(0xffffffffu, mbar_wait(&sh.empty[slot], ph ^ 1u, abort, wl))) return;
                    tc_fence_after();
                    const uint32_t col = tbase + lane_base + A0 + uint32_t(slot * 8);
#define OWN(w) ((((S * 8 + (w)) / NW) % PARTS) == PART)
                    const bool all8 = OWN(0) && OWN(2) && OWN(4) && OWN(6);
#pragma unroll
                    for (int r = 0; r < J; ++r) {
                        const uint32_t c = col + uint32_t(r) * RW;
                        if (all8) {
                            tmem_st8(c, v[r]);
                        } else {
#pragma unroll
                            for (int q = 0; q < 8; q += 4) {
                                if (OWN(q) && OWN(q + 2)) {
                                    tmem_st4(c + q, v[r][q], v[r][q + 1], v[r][q + 2], v[r][q + 3]);
                                } else {
                                    if (OWN(q)) tmem_st2(c + q, v[r][q], v[r][q + 1]);
                                    if (OWN(q + 2)) tmem_st2(c + q + 2, v[r][q + 2], v[r][q + 3]);
                                }
                            }
                        }
                    }
#undef OWN
                    pend_slot = slot;
                    if (++slot == RS) { slot = 0; ph ^= 1u; }
                }
            }
        }
        if (pend_slot >= 0) {
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            mbar_arrive_if(&sh.full[pend_slot], lane == 0);
            pend_slot = -1;
        }
        // ---- epilogue: this warp's jet rows of the accumulators -> y [J][O][N]
        if (!__all_sync(0xffffffffu, mbar_wait(&sh.accfull, uint32_t(it & 1), abort, wl))) return;
        tc_fence_after();
#pragma unroll 1
        for (int r = PART; r < J; r += PARTS) {
#pragma unroll 1
            for (int c = 0; c < O; c += 16) {
                uint32_t v[16];
                tmem_ld16(tbase + lane_base + uint32_t(r * O + c), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (valid) {
                    float* yp = p.y + (int64_t(r) * O + c) * N + pt;
#pragma unroll
                    for (int e = 0; e < 16; ++e) yp[int64_t(e) * N] = __uint_as_float(v[e]);
                }
            }
        }
        tc_fence_before();
        __syncwarp();
        mbar_arrive_if(&sh.accempty, lane == 0);
    }
}

// Runs produce<..., part> for a warp-uniform runtime part.
template <unsigned MASK, int PREC, int NP, int Q>
__device__ __forceinline__ void produce_part(int part, const TcLayer& p, TcShared& sh, uint32_t tbase, int quarter,
                                             int lane) {
    if constexpr (Q < PARTS) {
        if (part == Q) produce<MASK, PREC, NP, Q>(p, sh, tbase, quarter, lane);
        else produce_part<MASK, PREC, NP, Q + 1>(part, p, sh, tbase, quarter, lane);
    }
}

template <unsigned MASK, int PREC, int NP>
__global__ void __launch_bounds__(THREADS, 1) tc_fwd_kernel(TcLayer p, const __grid_constant__ CUtensorMap tmap) {
    using JT = Jet<MASK>;
    using E = Elem<PREC>;
    constexpr int J = JT::J;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ TcShared sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int O = p.O, RS = p.ring, KS = p.ks;
    const uint32_t b_bytes = uint32_t(E::TERMS * O) * 128u;   // one W buffer: TERMS tiles of O rows
    const uint32_t A0 = uint32_t(J * O);            // first A column; accumulators at r * O
    const uint32_t RW = uint32_t(RS * 8);           // ring words per jet row
    volatile int* abort = &sh.abort;
    const long long wl = wait_limit(p.status);

    if (tid == 0) {
        for (int s = 0; s < RS_MAX; ++s) {
            mbar_init(&sh.full[s], PRODUCER_WARPS);   // one arrive per producer warp
            mbar_init(&sh.empty[s], 1);               // tcgen05.commit
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(&sh.wfull[b], 1);
            mbar_init(&sh.wempty[b], 1);
        }
        mbar_init(&sh.accfull, 1);
        mbar_init(&sh.accempty, PRODUCER_WARPS);
        mbar_init(&sh.drain, 1);
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sh.tmem_base;
    const int ntiles = p.ntiles;

    if (warp < PRODUCER_WARPS) {
        produce_part<MASK, PREC, NP, 0>(warp >> 2, p, sh, tbase, warp & 3, lane);
    } else if (warp == PRODUCER_WARPS) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = idesc_of(E::FMT, O);
            int slot = 0, wb = 0;
            uint32_t ph = 0, wph = 0;
            bool issued = false;
            int it = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                if (!mbar_wait(&sh.accempty, uint32_t(it & 1) ^ 1u, abort, wl)) break;
                tc_fence_after();
                uint64_t bd = 0, bd2 = 0;
                for (int t = 0; t < KS; ++t) {
                    if ((t & 3) == 0) {
                        if (!mbar_wait(&sh.wfull[wb], wph, abort, wl)) goto mma_out;
                        bd = sdesc_sw128(smem_u32(smem + size_t(wb) * b_bytes));
                        // second tile of the buffer (w_lo): O rows of 128 bytes further
                        bd2 = sdesc_sw128(smem_u32(smem + size_t(wb) * b_bytes + size_t(O) * 128));
                    }
                    if (!mbar_wait(&sh.full[slot], ph, abort, wl)) goto mma_out;
                    tc_fence_after();
#pragma unroll
                    for (int r = 0; r < J; ++r) {
                        const uint32_t d = tbase + uint32_t(r * O);
                        const uint32_t a = tbase + A0 + uint32_t(r) * RW + uint32_t(slot * 8);
                        mma_ts<PREC>(d, a, bd + uint64_t((t & 3) * 2),   // +32 bytes per slot (descriptor counts 16 B)
                                     idesc, t > 0 ? 1u : 0u);
                        if constexpr (E::TERMS == 2) mma_ts<PREC>(d, a, bd2 + uint64_t((t & 3) * 2), idesc, 1u);
                    }
                    issued = true;
                    mma_commit(&sh.empty[slot]);
                    if (++slot == RS) { slot = 0; ph ^= 1u; }
                    if ((t & 3) == 3 || t == KS - 1) {
                        mma_commit(&sh.wempty[wb]);
                        if (++wb == NB) { wb = 0; wph ^= 1u; }
                    }
                }
                mma_commit(&sh.accfull);
            }
        mma_out:
            if (*abort && issued) {   // wait (bounded) for this thread's MMAs before TMEM is freed
                mma_commit(&sh.drain);
                mbar_drain(&sh.drain, 0u);
            }
        }
    } else {
        // ------------------------------------------------------------ W tiles by TMA
        if (lane == 0) {
            const int nbox = p.nbox;
            int wb = 0;
            uint32_t wph = 0;
            uint32_t used = 0u, last_par = 0u;   // bit b: buffer b has had a load / parity of its last one
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                // rows of this tile's instance in the tensor map (batched path)
                const int y0 = p.blk_inst ? p.blk_inst[tile >> 1] * (E::TERMS * O) : 0;
                for (int bx = 0; bx < nbox; ++bx) {
                    if (!mbar_wait(&sh.wempty[wb], wph ^ 1u, abort, wl)) goto tma_out;
                    mbar_expect_tx(&sh.wfull[wb], b_bytes);
                    tma_load_2d(smem + size_t(wb) * b_bytes, &tmap, &sh.wfull[wb], bx * E::BOX, y0);
                    used |= 1u << wb;
                    last_par = (last_par & ~(1u << wb)) | (wph << wb);
                    if (++wb == NB) { wb = 0; wph ^= 1u; }
                }
            }
        tma_out:
            if (*abort)
                for (int b = 0; b < NB; ++b)
                    if ((used >> b) & 1u) mbar_drain(&sh.wfull[b], (last_par >> b) & 1u);
        }
    }
    __syncwarp();
    if (warp < PRODUCER_WARPS) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicExch(p.status, ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(p.tmem_cols) : "memory");
}

// Host side: launch one instantiation (tc_np*.cu).
template <unsigned MASK, int PREC, int NP>
cudaError_t launch_one(const TcLayer& p, const CUtensorMap& map, cudaStream_t s);

}  // namespace tck
}  // namespace hrkan
