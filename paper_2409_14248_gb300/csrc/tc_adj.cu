// Tensor-core (tcgen05) input adjoint of one hidden layer in BF16 with FP32
// accumulation (reverse mode of the layer contraction w.r.t. its input jets,
// Sections 2-3, through v''' of Eq. 2):
//
//   G_r[p, k] = sum_o gy_r[p, o] W[o, k]                    (dense, tensor cores)
//   dA_r[p, j, q] = G_r[p, k(j, c_pj + q)],  q = 0..3          (the active bases;
//                   k(j, i) = j*NP + (i mod 4)*NP/4 + i/4, the forward's layout)
//   gz[p, j] = rows_adjoint(z[p, j], v', v'', v''', dA[p, j]) (FP32, per unit)
//
// A CTA owns UK consecutive units (a K-range of N = UK*NP columns, NP the
// forward's unit padding) and a chunk of 128-point tiles.  Its W tile
// [N x O] stays in shared memory; gy_r tiles [128 points x O] stream in by TMA.
// Both operands are MN-major in the 128-byte swizzle (points / k contiguous,
// o the MMA's K); D_r = 128 x N accumulates in one of two TMEM buffers so the
// MMAs of jet row r+1 overlap the epilogue of row r.  The epilogue warps
// (thread = point = TMEM lane; two warps per lane quarter, each half of the
// CTA's units) copy their lane's row of D to shared memory and read back the
// four entries of each unit at its cell.  For NP = 16 (two units per CTA)
// each row's share of the adjoint is added at once (the map is linear in dA,
// so no row is kept) and the next tile's jets arrive by cp.async meanwhile:
// 96 registers, two CTAs per SM (one CTA of four units per SM, at 168
// registers with spills, took 8% longer; two units at one CTA per SM 50%
// longer).  Wider units keep the J rows and apply the adjoint after the last.
// Every wait is bounded as in the forward kernel.
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "internal.h"
#include "tc.cuh"
#include "tc_kernel.cuh"

namespace hrkan {
namespace tcadj {

using tck::mbar_arrive_if;
using tck::mbar_drain;
using tck::mbar_expect_tx;
using tck::mbar_init;
using tck::mbar_wait;
using tck::mma_commit;
using tck::smem_u32;
using tck::tc_fence_after;
using tck::tc_fence_before;

constexpr int TILE = 128;   // points per tile (the MMA's M)
constexpr int NSB = 6;      // gy tile ring
constexpr int EPI_WARPS = 8;   // two per TMEM lane quarter, each half of the CTA's units
constexpr int THREADS = 32 * EPI_WARPS + 64;

struct AdjParams {
    const float* z;          // layer input jets [J][I][N]
    float* gz;               // dL/d(input jets) [J][I][N] (written)
    int I, O, n;
    int64_t N;
    int ntiles, nkr, nchunk;
    uint32_t tmem_cols;
    Grid g;
    int* status;
    // many instances (batched path): chunk c covers points [chunks[c].x,
    // chunks[c].y) (multiples of 256) of instance chunks[c].w, whose W rows
    // start at chunks[c].w * O of the W tensor map; nullptr: tiles split evenly
    const int4* chunks = nullptr;
    // non-null: gz goes out as BF16 [J * I][npad] (zero past N), the operand
    // layout of the layer below's tensor-core kernels, instead of FP32 into gz
    uint16_t* gz_bf = nullptr;
    int64_t npad = 0;
};

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
}

template <int NP>
struct Shape {
    // NP = 16: two units per CTA and the row-wise epilogue (96 registers, two CTAs per
    // SM); wider units: four units per CTA (two for NP >= 48) with the rows kept, one
    // CTA per SM (two units at two CTAs per SM spill there, and twice the K-ranges read
    // every gy tile: 2.90 against 1.91 ms per step of [2,64,64,64,1] G=32)
    static constexpr bool ROWWISE = NP == 16;
    static constexpr int UK = ROWWISE ? 2 : ((NP * 4 <= 160) ? 4 : 2);   // units per CTA (two epilogue halves)
    static constexpr int MINB = ROWWISE ? 2 : 1;         // resident CTAs per SM the registers allow
    static constexpr int UH = UK / 2;                    // units per epilogue warp
    static constexpr int NC = UK * NP;                   // D columns
    static constexpr int NBW = (NC + 63) / 64;           // W boxes of 64 k
    static constexpr int PS = UH * NP + 4;               // pick-row stride (floats) of one half
    static_assert(NC % 16 == 0 && NC <= 256 && 2 * NC <= 512, "MMA N, two D buffers in TMEM");
};

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFF) >> 4);
    d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(2) << 61;   // 128-byte swizzle
    return d;
}

template <unsigned MASK, int NP>
__global__ void __launch_bounds__(THREADS, Shape<NP>::MINB)
    tc_adj_kernel(AdjParams p, const __grid_constant__ CUtensorMap gmap, const __grid_constant__ CUtensorMap wmap) {
    using JT = Jet<MASK>;
    using SH = Shape<NP>;
    constexpr int J = JT::J, UK = SH::UK, NC = SH::NC, NBW = SH::NBW, PS = SH::PS;
    static_assert(UK % 2 == 0, "two epilogue halves");

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bar_gfull[NSB], bar_gempty[NSB], bar_dfull[2], bar_dempty[2];
    __shared__ __align__(8) uint64_t bar_wfull, bar_drain;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    volatile int* abort = &abort_sh;
    const long long wl = tck::wait_limit(p.status);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int O = p.O, I = p.I;
    const uint32_t box_bytes = uint32_t(O) * 128u;        // one 64-wide box of O rows
    const uint32_t g_bytes = 2u * box_bytes;              // gy tile: 128 points
    uint8_t* wtile = smem;                                // NBW boxes
    uint8_t* gring = smem + size_t(NBW) * box_bytes;      // NSB tiles
    float* pick = reinterpret_cast<float*>(gring + size_t(NSB) * g_bytes);   // [128][PS]
    const int kr = blockIdx.x % p.nkr, chunk = blockIdx.x / p.nkr;
    const int j0 = kr * UK;
    const int t0 = p.chunks ? p.chunks[chunk].x / TILE : int(int64_t(chunk) * p.ntiles / p.nchunk);
    const int t1 = p.chunks ? p.chunks[chunk].y / TILE : int(int64_t(chunk + 1) * p.ntiles / p.nchunk);
    const int w_row0 = p.chunks ? p.chunks[chunk].w * O : 0;
    const int nt = t1 - t0;

    if (tid == 0) {
        for (int b = 0; b < NSB; ++b) {
            mbar_init(&bar_gfull[b], 1);
            mbar_init(&bar_gempty[b], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar_dfull[b], 1);
            mbar_init(&bar_dempty[b], EPI_WARPS);
        }
        mbar_init(&bar_wfull, 1);
        mbar_init(&bar_drain, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base_sh;

    if (warp < EPI_WARPS) {
        // ------------------------------------------------------------ epilogue (thread = point)
        constexpr int UH = SH::UH;
        const int quarter = warp & 3, half = warp >> 2;
        const int row = quarter * 32 + lane;
        const uint32_t lane_base = uint32_t(quarter * 32) << 16;
        float* prow = pick + (half * TILE + row) * PS;
        const int ju = j0 + half * UH;                 // this warp's first unit
        const int64_t N = p.N;
        if constexpr (SH::ROWWISE) {
            // the next tile's jets go to shared memory by cp.async while this tile is
            // processed (two buffers [2][UH * J][256 threads]; each thread reads back only
            // its own entries, so its own wait_group orders them)
            float* zbuf = pick + size_t(2 * TILE) * PS;
            auto prefetch_z = [&](int ti) {
                const int64_t pt = int64_t(t0 + ti) * TILE + row;
                const float* zp = p.z + (pt < N ? pt : N - 1);
                float* dst = zbuf + size_t(ti & 1) * (UH * J * 32 * EPI_WARPS) + tid;
#pragma unroll
                for (int u = 0; u < UH; ++u) {
                    const int j = min(ju + u, I - 1);
#pragma unroll
                    for (int r = 0; r < J; ++r)
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                                         smem_u32(dst + (u * J + r) * (32 * EPI_WARPS))),
                                     "l"(zp + (int64_t(r) * I + j) * N)
                                     : "memory");
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
            if (nt > 0) prefetch_z(0);
            int q = 0;
            for (int ti = 0; ti < nt; ++ti) {
                const int64_t pt = int64_t(t0 + ti) * TILE + row;
                const bool valid = pt < N;
                float z[UH][J];
                asm volatile("cp.async.wait_group 0;" ::: "memory");
                {
                    const float* src = zbuf + size_t(ti & 1) * (UH * J * 32 * EPI_WARPS) + tid;
#pragma unroll
                    for (int u = 0; u < UH; ++u)
#pragma unroll
                        for (int r = 0; r < J; ++r) z[u][r] = src[(u * J + r) * (32 * EPI_WARPS)];
                }
                if (ti + 1 < nt) prefetch_z(ti + 1);   // next tile's jets, one tile ahead
                // basis derivatives of each unit at its value (v', v'', v'''), and where its
                // four active bases sit in a D row: basis i at element (i mod 4) * NP/4 + i/4
                // of the unit; bases outside [0, n) read a clamped entry (their derivatives are 0)
                float d1[UH][4], d2[UH][4], d3[UH][4], g[UH][J];
                int pos[UH][4];
#pragma unroll
                for (int u = 0; u < UH; ++u) {
                    Active<3, 4, 3> b;
                    b.eval(z[u][0], p.g);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        d1[u][k] = b.d1[k];
                        d2[u][k] = b.d2[k];
                        d3[u][k] = b.d3[k];
                        const int i = b.c + k;
                        const int ps = (i & 3) * (NP / 4) + (i >> 2);
                        pos[u][k] = u * NP + (ps < 0 ? 0 : (ps > NP - 1 ? NP - 1 : ps));
                    }
#pragma unroll
                    for (int r = 0; r < J; ++r) g[u][r] = 0.0f;
                }
#pragma unroll
                for (int r = 0; r < J; ++r, ++q) {
                    const int b = q & 1;
                    if (!__all_sync(0xffffffffu, mbar_wait(&bar_dfull[b], uint32_t(q >> 1) & 1u, abort, wl))) goto done;
                    tc_fence_after();
                    const uint32_t col0 = uint32_t(b * NC + half * UH * NP);
#pragma unroll
                    for (int c = 0; c < UH * NP; c += 8) {
                        uint32_t v[8];
                        tmem_ld8(tbase + lane_base + col0 + uint32_t(c), v);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        *reinterpret_cast<uint4*>(prow + c) = make_uint4(v[0], v[1], v[2], v[3]);
                        *reinterpret_cast<uint4*>(prow + c + 4) = make_uint4(v[4], v[5], v[6], v[7]);
                    }
                    tc_fence_before();
                    __syncwarp();
                    mbar_arrive_if(&bar_dempty[b], lane == 0);
#pragma unroll
                    for (int u = 0; u < UH; ++u) {
                        float a[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) a[k] = prow[pos[u][k]];
                        JT::template row_adjoint<4>(r, z[u], d1[u], d2[u], d3[u], a, g[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < UH; ++u) {
                    if (ju + u >= I) break;
                    if (p.gz_bf) {
                        if (pt < p.npad)
#pragma unroll
                            for (int r = 0; r < J; ++r)
                                p.gz_bf[(int64_t(r) * I + ju + u) * p.npad + pt] =
                                    __bfloat16_as_ushort(__float2bfloat16_rn(valid ? g[u][r] : 0.0f));
                    } else if (valid) {
#pragma unroll
                        for (int r = 0; r < J; ++r) p.gz[(int64_t(r) * I + ju + u) * N + pt] = g[u][r];
                    }
                }
            }
        } else {
            // the J rows of dA kept per unit, the reverse of the jet rows after the last
            // one; the next tile's jets in registers
            auto load_z = [&](int ti, float (&zz)[UH][J]) {
                const int64_t pt = int64_t(t0 + ti) * TILE + row;
                const float* zp = p.z + (pt < N ? pt : N - 1);
#pragma unroll
                for (int u = 0; u < UH; ++u) {
                    const int j = min(ju + u, I - 1);
#pragma unroll
                    for (int r = 0; r < J; ++r) zz[u][r] = zp[(int64_t(r) * I + j) * N];
                }
            };
            float zn[UH][J];
            if (nt > 0) load_z(0, zn);
            int q = 0;
            for (int ti = 0; ti < nt; ++ti) {
                const int64_t pt = int64_t(t0 + ti) * TILE + row;
                const bool valid = pt < N;
                float z[UH][J];
#pragma unroll
                for (int u = 0; u < UH; ++u)
#pragma unroll
                    for (int r = 0; r < J; ++r) z[u][r] = zn[u][r];
                if (ti + 1 < nt) load_z(ti + 1, zn);   // next tile's jets, one tile ahead
                int cell[UH];
#pragma unroll
                for (int u = 0; u < UH; ++u) {
                    Active<3, 4, 2> b;
                    b.eval(z[u][0], p.g);
                    cell[u] = b.c;
                }
                float dA[UH][J][4];
#pragma unroll
                for (int r = 0; r < J; ++r, ++q) {
                    const int b = q & 1;
                    if (!__all_sync(0xffffffffu, mbar_wait(&bar_dfull[b], uint32_t(q >> 1) & 1u, abort, wl))) goto done;
                    tc_fence_after();
                    const uint32_t col0 = uint32_t(b * NC + half * UH * NP);
#pragma unroll
                    for (int c = 0; c < UH * NP; c += 8) {
                        uint32_t v[8];
                        tmem_ld8(tbase + lane_base + col0 + uint32_t(c), v);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        *reinterpret_cast<uint4*>(prow + c) = make_uint4(v[0], v[1], v[2], v[3]);
                        *reinterpret_cast<uint4*>(prow + c + 4) = make_uint4(v[4], v[5], v[6], v[7]);
                    }
                    tc_fence_before();
                    __syncwarp();
                    mbar_arrive_if(&bar_dempty[b], lane == 0);
#pragma unroll
                    for (int u = 0; u < UH; ++u)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            // basis i at element (i mod 4) * NP/4 + i/4 of the unit; bases outside
                            // [0, n) read a clamped entry (their derivatives are 0)
                            const int i = cell[u] + k;
                            int pos = (i & 3) * (NP / 4) + (i >> 2);
                            pos = pos < 0 ? 0 : (pos > NP - 1 ? NP - 1 : pos);
                            dA[u][r][k] = prow[u * NP + pos];
                        }
                }
#pragma unroll
                for (int u = 0; u < UH; ++u) {
                    if (ju + u >= I) break;
                    Active<3, 4, 3> b;
                    b.eval(z[u][0], p.g);
                    float g[J];
                    JT::template rows_adjoint<4>(z[u], b.d1, b.d2, b.d3, dA[u], g);
                    if (p.gz_bf) {
                        if (pt < p.npad)
#pragma unroll
                            for (int r = 0; r < J; ++r)
                                p.gz_bf[(int64_t(r) * I + ju + u) * p.npad + pt] =
                                    __bfloat16_as_ushort(__float2bfloat16_rn(valid ? g[r] : 0.0f));
                    } else if (valid) {
#pragma unroll
                        for (int r = 0; r < J; ++r) p.gz[(int64_t(r) * I + ju + u) * N + pt] = g[r];
                    }
                }
            }
        }
    } else if (warp == EPI_WARPS) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0 && nt > 0) {
            // kind::f16, BF16, A (gy, points contiguous) and B (W, k contiguous) MN-major, FP32 D, M = 128, N = NC
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                   (uint32_t(NC >> 3) << 17) | (uint32_t(TILE >> 4) << 24);
            bool issued = false;
            if (mbar_wait(&bar_wfull, 0u, abort, wl)) {
                tc_fence_after();
                const uint32_t wbase = smem_u32(wtile);
                const int total = nt * J;
                for (int q = 0; q < total; ++q) {
                    const int gb = q % NSB, db = q & 1;
                    if (!mbar_wait(&bar_gfull[gb], uint32_t(q / NSB) & 1u, abort, wl)) break;
                    if (!mbar_wait(&bar_dempty[db], (uint32_t(q >> 1) & 1u) ^ 1u, abort, wl)) break;
                    tc_fence_after();
                    const uint32_t gbase = smem_u32(gring + size_t(gb) * g_bytes);
                    for (int s = 0; s < O / 16; ++s) {
                        // 16 o per step = two 8-row K groups (1 KB apart) of both operands
                        const uint64_t ad = sdesc(gbase + uint32_t(s) * 2048u, box_bytes, 1024);
                        const uint64_t bd = sdesc(wbase + uint32_t(s) * 2048u, box_bytes, 1024);
                        asm volatile(
                            "{\n\t.reg .pred pa;\n\tsetp.ne.b32 pa, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n\t}" ::"r"(
                                tbase + uint32_t(db * NC)),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(s > 0 ? 1u : 0u)
                            : "memory");
                    }
                    issued = true;
                    mma_commit(&bar_gempty[gb]);
                    mma_commit(&bar_dfull[db]);
                }
            }
            if (*abort && issued) {
                mma_commit(&bar_drain);
                mbar_drain(&bar_drain, 0u);
            }
        }
    } else {
        // ------------------------------------------------------------ W tile once, gy tiles by TMA
        if (lane == 0 && nt > 0) {
            mbar_expect_tx(&bar_wfull, uint32_t(NBW) * box_bytes);
            for (int bx = 0; bx < NBW; ++bx)
                tck::tma_load_2d(wtile + size_t(bx) * box_bytes, &wmap, &bar_wfull, j0 * NP + 64 * bx, w_row0);
            const int total = nt * J;
            uint32_t used = 0u, last_par = 0u;
            for (int q = 0; q < total; ++q) {
                const int b = q % NSB, ti = q / J, r = q % J;
                const uint32_t ph = uint32_t(q / NSB) & 1u;
                if (!mbar_wait(&bar_gempty[b], ph ^ 1u, abort, wl)) break;
                mbar_expect_tx(&bar_gfull[b], g_bytes);
                uint8_t* dst = gring + size_t(b) * g_bytes;
                const int x = (t0 + ti) * TILE;
                tck::tma_load_2d(dst, &gmap, &bar_gfull[b], x, r * O);
                tck::tma_load_2d(dst + box_bytes, &gmap, &bar_gfull[b], x + 64, r * O);
                used |= 1u << b;
                last_par = (last_par & ~(1u << b)) | (ph << b);
            }
            if (*abort) {
                (void)mbar_wait(&bar_wfull, 0u, abort);
                mbar_drain(&bar_wfull, 0u);
                for (int b = 0; b < NSB; ++b)
                    if ((used >> b) & 1u) mbar_drain(&bar_gfull[b], (last_par >> b) & 1u);
            }
        }
    }
done:
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicExch(p.status, tck::ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(p.tmem_cols)
                     : "memory");
}

// W [O][I][n] float32 -> [O][Kt] BF16, element k = j * NP + pos holding basis
// i = 4 * (pos mod NP/4) + pos / (NP/4) (zero for i >= n or j >= I).
// Many instances: instance c's layer at W + c * w_stride goes to out + c * O * Kt.
__global__ void w_bf16_kernel(const float* __restrict__ W, uint16_t* __restrict__ out, int O, int I, int n, int NP,
                              int Kt, int n_inst, int64_t w_stride) {
    const int64_t total = int64_t(O) * Kt;
    for (int64_t u = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < total * n_inst;
         u += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = u / total, t = u % total;
        const int o = int(t / Kt), k = int(t % Kt);
        const int j = k / NP, pos = k % NP, q = NP / 4, i = 4 * (pos % q) + pos / q;
        const float w = (j < I && i < n) ? W[c * w_stride + (int64_t(o) * I + j) * n + i] : 0.0f;
        out[u] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
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

int np_of(int n) {
    for (int np : {16, 24, 32, 40, 48, 64})
        if (n <= np) return np;
    return 0;
}

template <unsigned MASK, int NP>
cudaError_t launch(const AdjParams& p, const CUtensorMap& gm, const CUtensorMap& wm, unsigned grid, cudaStream_t s) {
    using SH = Shape<NP>;
    const size_t box = size_t(p.O) * 128;
    const size_t smem = size_t(SH::NBW) * box + size_t(NSB) * 2 * box + size_t(2 * TILE) * SH::PS * 4 +
                        (SH::ROWWISE ? size_t(2 * SH::UH * Jet<MASK>::J * 32 * EPI_WARPS) * 4 : 0) + 1024;
    auto kern = tc_adj_kernel<MASK, NP>;
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> set;
    {
        std::lock_guard<std::mutex> lk(mu);
        size_t& cur = set[reinterpret_cast<const void*>(kern)];
        if (cur < smem) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (e != cudaSuccess) { cudaGetLastError(); return e; }
            cur = smem;
        }
    }
    kern<<<grid, THREADS, smem, s>>>(p, gm, wm);
    return cudaGetLastError();
}

template <unsigned MASK>
cudaError_t launch_np(int np, const AdjParams& p, const CUtensorMap& gm, const CUtensorMap& wm, unsigned grid,
                      cudaStream_t s) {
    switch (np) {
        case 16: return launch<MASK, 16>(p, gm, wm, grid, s);
        case 24: return launch<MASK, 24>(p, gm, wm, grid, s);
        case 32: return launch<MASK, 32>(p, gm, wm, grid, s);
        case 40: return launch<MASK, 40>(p, gm, wm, grid, s);
        case 48: return launch<MASK, 48>(p, gm, wm, grid, s);
        case 64: return launch<MASK, 64>(p, gm, wm, grid, s);
    }
    return cudaErrorNotSupported;
}

int units_per_cta(int np) {
    switch (np) {
        case 16: return Shape<16>::UK;
        case 24: return Shape<24>::UK;
        case 32: return Shape<32>::UK;
        case 40: return Shape<40>::UK;
        case 48: return Shape<48>::UK;
        case 64: return Shape<64>::UK;
    }
    return 0;
}

}  // namespace tcadj

bool tc_adj_supported(int prec, int I, int O, int n, unsigned mask) {
    return tc_dw_supported(prec, I, O, n, mask) && tcadj::np_of(n) != 0 && mask != 0x01u;
}

int64_t tc_adj_w_elems(int O, int I, int n) {
    const int np = tcadj::np_of(n);
    return int64_t(O) * ((int64_t(I) * np + 63) / 64 * 64);
}

cudaError_t tc_adj_layer(const float* W, void* w_bf, const void* gy_bf, const float* z, float* gz, int I, int O,
                         int64_t N, const Grid& g, unsigned mask, int* status, cudaStream_t s, int n_inst,
                         int64_t w_stride, const int4* chunks, int nchunk, void* gz_bf) {
    using namespace tcadj;
    if (N == 0) return cudaSuccess;
    if (n_inst < 1 || (chunks && nchunk < 1) || (n_inst > 1 && !chunks)) return cudaErrorInvalidValue;
    const int n = g.n, np = np_of(n);
    const int J = __builtin_popcount(mask & 0x1Fu);
    const int Kt = int((int64_t(I) * np + 63) / 64 * 64);
    {
        const int64_t total = int64_t(O) * Kt * n_inst;
        const int pb = int(std::min<int64_t>((total + 255) / 256, 4096));
        w_bf16_kernel<<<pb, 256, 0, s>>>(W, static_cast<uint16_t*>(w_bf), O, I, n, np, Kt, n_inst, w_stride);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int64_t Npad = (N + 63) / 64 * 64;
    CUtensorMap gm, wm;
    {
        const cuuint64_t dims[2] = {cuuint64_t(Npad), cuuint64_t(int64_t(J) * O)};
        const cuuint64_t strides[1] = {cuuint64_t(Npad) * 2};
        const cuuint32_t box[2] = {64, cuuint32_t(O)};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&gm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(gy_bf), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[2] = {cuuint64_t(Kt), cuuint64_t(O) * cuuint64_t(n_inst)};
        const cuuint64_t strides[1] = {cuuint64_t(Kt) * 2};
        const cuuint32_t box[2] = {64, cuuint32_t(O)};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&wm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, w_bf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    AdjParams p{};
    p.z = z;
    p.gz = gz;
    p.I = I;
    p.O = O;
    p.n = n;
    p.N = N;
    p.ntiles = int((N + TILE - 1) / TILE);
    const int uk = units_per_cta(np);
    p.nkr = (I + uk - 1) / uk;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // at most one CTA per SM over the K-ranges (a single wave), at least one tile each;
    // the batched path takes its instances' chunks
    p.nchunk = chunks ? nchunk : std::max(1, std::min(p.ntiles, nsm / p.nkr));
    p.chunks = chunks;
    p.gz_bf = static_cast<uint16_t*>(gz_bf);
    p.npad = Npad;
    const int cols = 2 * uk * np;
    p.tmem_cols = cols <= 32 ? 32u : cols <= 64 ? 64u : cols <= 128 ? 128u : cols <= 256 ? 256u : 512u;
    p.g = g;
    p.status = status;
    const unsigned grid = unsigned(p.nkr) * unsigned(p.nchunk);
    switch (mask) {
        case 0x0Fu: return launch_np<0x0Fu>(np, p, gm, wm, grid, s);
        case 0x1Fu: return launch_np<0x1Fu>(np, p, gm, wm, grid, s);
    }
    return cudaErrorNotSupported;
}

}  // namespace hrkan
