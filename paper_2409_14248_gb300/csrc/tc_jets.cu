// Tensor-core (tcgen05 / TMEM / TMA) contraction of the stacked jet rows with
// the layer weights, for the hidden layers of wide networks (Sections 1-3:
// the KAN layer as a matrix operation; Eq. 2 bases).
//
//   Y_r[p, o] = sum_k A_r[p, k] W[o, k],  k = j*n + i,  r = 0..J-1 jet rows
//
// One CTA owns 128 points (the MMA's M) and all O outputs (N = O).  Per K
// step of 128 bytes of a row (64 BF16 or 32 TF32 elements):
//   * two threads per point (TMEM lane = point of the tile) evaluate the
//     active HR bases of the units the step covers, form the J jet rows (each
//     thread half of them), place their 4 non-zeros per unit into 32 registers
//     (the rest of the row is zero) and store them into the point's TMEM lane
//     with tcgen05.st (A operand in TMEM);
//   * one thread issues J x 4 tcgen05.mma (A from TMEM, B = W tile from
//     shared memory, FP32 accumulators in TMEM, one per jet row) and commits
//     them to an mbarrier;
//   * the W tile of the next step arrives by TMA (128-byte swizzle, K-major).
// Every mbarrier wait is bounded: on timeout the CTA records HRKAN_ETIMEOUT in
// a device status word, waits (bounded) for its own copies and MMAs, frees its
// TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <cuda_bf16.h>
#include <mutex>
#include <unordered_map>

#include "internal.h"
#include "tc.cuh"

namespace hrkan {
namespace {

constexpr int TC_M = 128;           // points per tile (the MMA M); the CTA has 2 threads per point
constexpr int TMEM_COLS = 512;
constexpr uint32_t A_COL0 = 320;    // A region after the accumulators (J * O <= 320 columns)
constexpr long long WAIT_CYCLES = 2000000000LL;   // ~1 s at 2 GHz
constexpr int ERR_TIMEOUT = -5;     // HRKAN_ETIMEOUT

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

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > WAIT_CYCLES) return false;
    return true;
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
           (uint32_t(TC_M >> 4) << 24);
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

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
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

// Elements of one value in a 32-bit TMEM column / A word.
template <int PREC>
struct Elem;
template <>
struct Elem<HRKAN_BF16> {
    static constexpr int PER_WORD = 2, PER_STEP = 64, MMA_K = 16, FMT = 1;
    __device__ static uint32_t bits(float x) {
        return uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x)));
    }
};
template <>
struct Elem<HRKAN_TF32> {
    static constexpr int PER_WORD = 1, PER_STEP = 32, MMA_K = 8, FMT = 2;
    __device__ static uint32_t bits(float x) {
        uint32_t r;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
        return r;
    }
};

// Stores the jet rows [R0, R1) of this thread's point for one K step into its
// TMEM lane.  The U units the step touches are the same for every point of
// the tile (they depend only on the step), so U is a compile-time constant of
// the call; only each unit's active window (cell) varies per point.
template <unsigned MASK, int PREC, int R0, int R1, int U>
__device__ __forceinline__ void build_rows(const TcLayer& p, int I, int n, int64_t N, int64_t ptc, int k0, int jf,
                                           uint32_t a_taddr) {
    using JT = Jet<MASK>;
    using E = Elem<PREC>;
    constexpr int J = JT::J;
    constexpr int NR = R1 - R0;
    constexpr int NS = E::PER_WORD == 2 ? 3 : 4;   // words the 4 values of a unit can span
    if constexpr (NR > 0) {
        int w0[U];
        uint32_t x[U][NR][NS];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = jf + u;
            float z[J];
#pragma unroll
            for (int r = 0; r < J; ++r) z[r] = p.z[(int64_t(r) * I + j) * N + ptc];
            Active<3, 4, 2> b;
            b.eval(z[0], p.g);
            float a[J][4];
            JT::template rows<4>(z, b.v, b.d1, b.d2, a);
            const int P = j * n + b.c - k0;   // element offset of the first active basis in this step
            if constexpr (E::PER_WORD == 2) {
                // 4 BF16 values at elements P..P+3 span words P>>1 .. (P+3)>>1
                const bool odd = (P & 1) != 0;
                w0[u] = (P - (odd ? 1 : 0)) / 2;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const uint32_t e0 = E::bits(a[R0 + r][0]), e1 = E::bits(a[R0 + r][1]);
                    const uint32_t e2 = E::bits(a[R0 + r][2]), e3 = E::bits(a[R0 + r][3]);
                    x[u][r][0] = odd ? (e0 << 16) : (e0 | (e1 << 16));
                    x[u][r][1] = odd ? (e1 | (e2 << 16)) : (e2 | (e3 << 16));
                    x[u][r][2] = odd ? e3 : 0u;
                }
            } else {
                w0[u] = P;
#pragma unroll
                for (int r = 0; r < NR; ++r)
#pragma unroll
                    for (int k = 0; k < NS; ++k) x[u][r][k] = E::bits(a[R0 + r][k]);
            }
            // a basis index outside [0, n) has value 0 already (Active masks it)
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            uint32_t v[32];
#pragma unroll
            for (int w = 0; w < 32; ++w) {
                uint32_t acc = 0u;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int d = w - w0[u];
#pragma unroll
                    for (int k = 0; k < NS; ++k) acc |= (d == k) ? x[u][r][k] : 0u;
                }
                v[w] = acc;
            }
            tmem_st32(a_taddr + uint32_t((R0 + r) * 32), v);
        }
    }
}

template <unsigned MASK, int PREC, int R0, int R1>
__device__ __forceinline__ void build_rows_u(int U, const TcLayer& p, int I, int n, int64_t N, int64_t ptc, int k0,
                                             int jf, uint32_t a_taddr) {
    switch (U) {
        case 1: build_rows<MASK, PREC, R0, R1, 1>(p, I, n, N, ptc, k0, jf, a_taddr); break;
        case 2: build_rows<MASK, PREC, R0, R1, 2>(p, I, n, N, ptc, k0, jf, a_taddr); break;
        case 3: build_rows<MASK, PREC, R0, R1, 3>(p, I, n, N, ptc, k0, jf, a_taddr); break;
        case 4: build_rows<MASK, PREC, R0, R1, 4>(p, I, n, N, ptc, k0, jf, a_taddr); break;
        case 5: build_rows<MASK, PREC, R0, R1, 5>(p, I, n, N, ptc, k0, jf, a_taddr); break;
        default: build_rows<MASK, PREC, R0, R1, 6>(p, I, n, N, ptc, k0, jf, a_taddr); break;
    }
}

template <unsigned MASK, int PREC>
__global__ void __launch_bounds__(2 * TC_M, 1) tc_fwd_kernel(TcLayer p, const __grid_constant__ CUtensorMap tmap) {
    using JT = Jet<MASK>;
    using E = Elem<PREC>;
    constexpr int J = JT::J;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bar_tma[2];
    __shared__ __align__(8) uint64_t bar_mma;
    __shared__ uint32_t tmem_base_sh;

    // 256 threads: thread t works on point (t mod 128) of the tile, i.e. TMEM lane
    // t mod 128; threads 0..127 build jet rows [0, JA), threads 128..255 rows [JA, J).
    constexpr int JA = (J + 1) / 2;
    const int tid = threadIdx.x, warp = tid >> 5, row = tid & (TC_M - 1), half = tid >> 7;
    const int O = p.O, I = p.I, n = p.g.n;
    const uint32_t b_bytes = uint32_t(O) * 128u;
    uint8_t* bbuf[2] = {smem, smem + b_bytes};

    if (tid == 0) {
        mbar_init(&bar_tma[0], 1);
        mbar_init(&bar_tma[1], 1);
        mbar_init(&bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base_sh;
    const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
    const uint32_t idesc = idesc_of(E::FMT, O);

    const int64_t N = p.N;
    const int64_t pt = int64_t(blockIdx.x) * TC_M + row;
    const bool valid = pt < N;
    const int64_t ptc = valid ? pt : N - 1;   // idle lanes compute on a real point, results dropped

    uint32_t tma_par[2] = {0u, 0u}, mma_par = 0u;
    bool tma_pending[2] = {false, false};
    bool mma_pending = false;
    int failed = 0;
    if (tid == 0) {
        mbar_expect_tx(&bar_tma[0], b_bytes);
        tma_load_2d(bbuf[0], &tmap, &bar_tma[0], 0, 0);
        tma_pending[0] = true;
    }
    for (int s = 0; s < p.ksteps; ++s) {
        const int buf = s & 1;
        if (tid == 0 && s + 1 < p.ksteps) {   // prefetch the next W tile (its buffer's last reader has finished)
            mbar_expect_tx(&bar_tma[buf ^ 1], b_bytes);
            tma_load_2d(bbuf[buf ^ 1], &tmap, &bar_tma[buf ^ 1], (s + 1) * E::PER_STEP, 0);
            tma_pending[buf ^ 1] = true;
        }
        // ---- A rows of this step into TMEM
        {
            const int k0 = s * E::PER_STEP;
            const int jf = k0 / n;
            const int jl = min(I - 1, (k0 + E::PER_STEP - 1) / n);
            const int U = jl - jf + 1;   // same for every point of the tile
            const uint32_t a_taddr = tbase + lane_base + A_COL0;
            if (half == 0) build_rows_u<MASK, PREC, 0, JA>(U, p, I, n, N, ptc, k0, jf, a_taddr);
            else build_rows_u<MASK, PREC, JA, J>(U, p, I, n, N, ptc, k0, jf, a_taddr);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        // ---- issue the MMAs
        if (tid == 0) {
            tc_fence_after();
            if (!mbar_wait(&bar_tma[buf], tma_par[buf])) {
                failed = 1;
            } else {
                tma_par[buf] ^= 1u;
                tma_pending[buf] = false;
                const uint64_t bd = sdesc_sw128(smem_u32(bbuf[buf]));
#pragma unroll
                for (int r = 0; r < J; ++r)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_ts<PREC>(tbase + uint32_t(r * O), tbase + A_COL0 + uint32_t(r * 32 + kk * 8),
                                     bd + uint64_t(kk * 2),   // +32 bytes per K slice (descriptor counts 16 B)
                                     idesc, (s > 0 || kk > 0) ? 1u : 0u);
                mma_commit(&bar_mma);
                mma_pending = true;
            }
        }
        if (__syncthreads_or(failed)) { failed = 1; break; }
        // ---- the step's MMAs must be done before A and the W buffer are reused
        bool ok = mbar_wait(&bar_mma, mma_par);
        mma_par ^= 1u;
        if (tid == 0 && ok) mma_pending = false;
        tc_fence_after();
        if (__syncthreads_or(!ok)) { failed = 1; break; }
    }
    if (!failed) {
        // ---- epilogue: accumulators -> output jets [J][O][N] (each half its own rows)
        const int r0 = half == 0 ? 0 : JA, r1 = half == 0 ? JA : J;
        for (int r = r0; r < r1; ++r) {
            for (int c = 0; c < O; c += 16) {
                uint32_t v[16];
                tmem_ld16(tbase + lane_base + uint32_t(r * O + c), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (valid)
#pragma unroll
                    for (int e = 0; e < 16; ++e) p.y[(int64_t(r) * O + c + e) * N + pt] = __uint_as_float(v[e]);
            }
        }
    } else if (tid == 0) {
        atomicExch(p.status, ERR_TIMEOUT);
        // wait (bounded) for this CTA's own copies and MMAs still in flight
        for (int b = 0; b < 2; ++b)
            if (tma_pending[b]) (void)mbar_wait(&bar_tma[b], tma_par[b]);
        if (mma_pending) (void)mbar_wait(&bar_mma, mma_par ^ 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------- weights
// W [O][I*n] float32 -> [O][Kpad] in the MMA's element type (BF16 bits, or
// TF32-rounded float32), zero beyond I*n.
template <int PREC>
__global__ void tc_prep_w_kernel(const float* __restrict__ W, void* out, int O, int K, int Kpad) {
    const int64_t total = int64_t(O) * Kpad;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int o = int(t / Kpad), k = int(t % Kpad);
        const float w = k < K ? W[int64_t(o) * K + k] : 0.0f;
        if constexpr (PREC == HRKAN_BF16)
            static_cast<uint16_t*>(out)[t] = uint16_t(Elem<HRKAN_BF16>::bits(w));
        else
            static_cast<uint32_t*>(out)[t] = Elem<HRKAN_TF32>::bits(w);
    }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        else
            cudaGetLastError();
    });
    return fn;
}

template <unsigned MASK, int PREC>
cudaError_t launch_mask(const TcLayer& p, const CUtensorMap& map, cudaStream_t s) {
    const size_t smem = 2 * size_t(p.O) * 128 + 1024;   // two W tiles + alignment slack
    auto kern = tc_fwd_kernel<MASK, PREC>;
    // at most one CTA per SM: each allocates all 512 TMEM columns
    const size_t want = std::max<size_t>(smem, 120 * 1024);
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> set;
    {
        std::lock_guard<std::mutex> lk(mu);
        size_t& cur = set[reinterpret_cast<const void*>(kern)];
        if (cur < want) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(want));
            if (e != cudaSuccess) { cudaGetLastError(); return e; }
            cur = want;
        }
    }
    const unsigned grid = unsigned((p.N + TC_M - 1) / TC_M);
    kern<<<grid, 2 * TC_M, want, s>>>(p, map);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_prec(const TcLayer& p, unsigned mask, const CUtensorMap& map, cudaStream_t s) {
    switch (mask) {
        case 0x01u: return launch_mask<0x01u, PREC>(p, map, s);
        case 0x0Fu: return launch_mask<0x0Fu, PREC>(p, map, s);
        case 0x1Fu: return launch_mask<0x1Fu, PREC>(p, map, s);
    }
    return cudaErrorNotSupported;
}

}  // namespace

bool tc_layer_supported(int prec, int I, int O, int n, unsigned mask) {
    const int J = __builtin_popcount(mask & 0x1Fu);
    if (prec != HRKAN_BF16 && prec != HRKAN_TF32) return false;
    if (O < 16 || O > 64 || O % 16 != 0 || J * O > int(A_COL0)) return false;
    const int per_step = prec == HRKAN_BF16 ? 64 : 32;
    // a K step of per_step elements touches at most ceil((per_step-1)/n) + 1 units; the kernel holds 6
    if ((per_step - 1 + n - 1) / n + 1 > 6) return false;
    return I >= 1 && (mask == 0x01u || mask == 0x0Fu || mask == 0x1Fu);
}

int64_t tc_w_elems(int O, int I, int n, int prec) {
    const int per_step = prec == HRKAN_BF16 ? 64 : 32;
    const int64_t K = int64_t(I) * n, Kpad = (K + per_step - 1) / per_step * per_step;
    return int64_t(O) * Kpad;
}

cudaError_t tc_forward_layer(const float* W, void* w_prep, const float* z, float* y, int I, int O, int64_t N,
                             const Grid& g, int prec, unsigned mask, int* status, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int n = g.n;
    const int per_step = prec == HRKAN_BF16 ? 64 : 32;
    const int K = I * n, Kpad = (K + per_step - 1) / per_step * per_step;
    const int64_t total = int64_t(O) * Kpad;
    const int pb = int(std::min<int64_t>((total + 255) / 256, 4096));
    if (prec == HRKAN_BF16)
        tc_prep_w_kernel<HRKAN_BF16><<<pb, 256, 0, s>>>(W, w_prep, O, K, Kpad);
    else
        tc_prep_w_kernel<HRKAN_TF32><<<pb, 256, 0, s>>>(W, w_prep, O, K, Kpad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[2] = {cuuint64_t(Kpad), cuuint64_t(O)};
    const cuuint64_t strides[1] = {cuuint64_t(Kpad) * (prec == HRKAN_BF16 ? 2 : 4)};
    const cuuint32_t box[2] = {cuuint32_t(per_step), cuuint32_t(O)};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, prec == HRKAN_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                     w_prep, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    TcLayer p{};
    p.z = z;
    p.y = y;
    p.I = I;
    p.O = O;
    p.N = N;
    p.ksteps = Kpad / per_step;
    p.g = g;
    p.status = status;
    return prec == HRKAN_BF16 ? launch_prec<HRKAN_BF16>(p, mask, map, s) : launch_prec<HRKAN_TF32>(p, mask, map, s);
}

}  // namespace hrkan
