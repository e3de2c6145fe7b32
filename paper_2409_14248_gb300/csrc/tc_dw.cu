// Tensor-core (tcgen05) weight gradient of one hidden layer in BF16 with FP32
// accumulation (reverse mode of the layer contraction, Sections 2-3), hidden
// layers and (FIRST) the first layer, whose inputs are the coordinates:
//
//   dW[o, k] = sum_p sum_r gy_r[p, o] * A_r[p, k]
//
// with k running over the units padded to NP8 elements, bases stored by residue
// mod 4 inside a unit (basis i at j*NP8 + (i mod 4)*NP8/4 + i/4, as the forward).
//
// i.e. D = A_r^T gy_r summed over jet rows r and points p.  The MMA's M runs
// over 128 consecutive k (one "K-range" per CTA), N over the O outputs and its
// K over points.  A_r^T is the A operand in shared memory in the MN-major
// 128-byte-swizzle layout (k contiguous per point), which the producers build
// point by point exactly like the forward does (active bases, jet rows, BF16
// windows, selects) but store with st.shared; gy_r is the B operand (K-major:
// points contiguous), streamed from a BF16 copy by TMA.  Each CTA owns one
// K-range and one chunk of points and writes its slice of one partial row;
// the rows are summed in a fixed order afterwards (deterministic).
//
// Warp roles (320 threads): warps 0-7 produce (thread = point of a 64-point
// group x one of four unit classes), warp 8 issues the MMAs, warp 9 loads gy
// tiles.  A ring of group slots, each holding one group's J A tiles (128 k x
// 64 points, 16 KB each) and its J gy tiles (O x 64 points): one wait, one
// proxy fence and one arrive per producer warp and group, one tcgen05.commit
// per group.  Where only one slot fits (J = 5, O >= 48: EARLY) the producers
// evaluate a group's unit windows before they wait for its slot, so that they
// still overlap the MMAs; with two or more slots they evaluate and store unit
// by unit (fewer live registers).  Measured on the weight gradients of the
// batching workload ([2,16,16,1], four launches per step): 2.3 ms per step
// against 3.8 with a slot per (group, jet row) and four producer warps; on
// [2,64,64,64,1] (six launches, EARLY): 2.4 ms against 3.0.  Every wait is
// bounded as in the forward kernel.
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "internal.h"
#include "tc.cuh"
#include "tc_kernel.cuh"

namespace hrkan {
namespace tcdw {

using tck::mbar_arrive_if;
using tck::mbar_drain;
using tck::mbar_expect_tx;
using tck::mbar_init;
using tck::mbar_wait;
using tck::mma_commit;
using tck::smem_u32;
using tck::tc_fence_after;
using tck::tc_fence_before;
using tck::tmem_ld16;

constexpr int GROUP = 64;        // points per group (the gy tile's 128 bytes)
constexpr int NPROD = 8;         // producer warps
constexpr int NPAR = NPROD / 2;  // unit classes: two warps cover a group's points, a class takes every NPAR-th unit
constexpr int NSB = 8;           // most group slots; p.nsb of them are used
constexpr int A_BYTES = 128 * GROUP * 2;   // 128 k x 64 points BF16
constexpr int SLOT_BUDGET = 200 * 1024;    // shared memory for the group slots
constexpr int THREADS = 32 * (NPROD + 2);

struct DwParams {
    const float* z;        // layer input jets [J][I][N]
    float* partial;        // [rows][P]
    int64_t P, col0;
    int row0, nchunk;      // this call writes rows [row0, row0 + nchunk)
    int I, O, n, np8;
    int64_t N;
    int ngroups;           // groups of 64 points over the padded point range
    int nkr;               // K-ranges of 128 k
    uint32_t tmem_cols;
    Grid g;
    int* status;
    // many instances (batched path): chunk c covers points [chunks[c].x,
    // chunks[c].y) (multiples of 256) and writes partial row chunks[c].z;
    // nullptr: the groups split evenly, chunk c into row row0 + c
    const int4* chunks = nullptr;
    int nsb = NSB;         // group slots in use
};

// Byte offset of element (m = k within the K-range, p = point within the group)
// in an A tile: MN-major, 128-byte swizzle; 8-point groups 2048 B apart, the two
// 64-k halves 1024 B apart (descriptor LBO = 1024, SBO = 2048).
__device__ __forceinline__ uint32_t a_off(int m, int p) {
    return uint32_t((p >> 3) * 2048 + (m >> 6) * 1024 + (p & 7) * 128 + ((((m & 63) >> 3) ^ (p & 7)) << 4));
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFF) >> 4);
    d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(2) << 61;   // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

template <unsigned MASK, int NC, bool FIRST, bool EARLY>
__global__ void __launch_bounds__(THREADS, 1) tc_dw_kernel(DwParams p, const __grid_constant__ CUtensorMap gmap) {
    using JT = Jet<MASK>;
    constexpr int J = JT::J;
    constexpr int NP8 = 8 * NC;                                  // elements per padded unit
    constexpr int MAXU = ((127 / NP8) + 2 + NPAR - 1) / NPAR;    // units of one class overlapping 128 k
    using Win = tck::UnitWin<J>;
    constexpr int QW = NP8 / 8;                                  // words per residue quarter of a unit

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bar_full[NSB], bar_empty[NSB];
    __shared__ __align__(8) uint64_t bar_accfull, bar_drain;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    volatile int* abort = &abort_sh;
    const long long wl = tck::wait_limit(p.status);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int O = p.O, I = p.I;
    const uint32_t b_bytes = uint32_t(O) * 128u;
    // one ring slot per group: J A tiles, then J gy tiles
    const uint32_t slot_bytes = uint32_t(J) * (uint32_t(A_BYTES) + b_bytes);
    const int kr = blockIdx.x % p.nkr, chunk = blockIdx.x / p.nkr;
    const int k0 = kr * 128;
    const int nsg = p.nsb;
    const int g0 = p.chunks ? p.chunks[chunk].x / GROUP : int(int64_t(chunk) * p.ngroups / p.nchunk);
    const int g1 = p.chunks ? p.chunks[chunk].y / GROUP : int(int64_t(chunk + 1) * p.ngroups / p.nchunk);
    const int out_row = p.chunks ? p.chunks[chunk].z : p.row0 + chunk;
    const int ng = g1 - g0;

    if (tid == 0) {
        for (int b = 0; b < NSB; ++b) {
            mbar_init(&bar_full[b], NPROD + 1);   // the producer warps + the TMA's expect_tx
            mbar_init(&bar_empty[b], 1);
        }
        mbar_init(&bar_accfull, 1);
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

    if (warp < NPROD) {
        // ------------------------------------------------------------ producers
        // thread = point pp of the group x unit class par: units jlo + par + NPAR * u
        const int pp = tid & (GROUP - 1), par = tid >> 6;
        const int jlo = k0 / NP8;
        const int jhi = min(I - 1, (k0 + 127) / NP8);
        int jn[MAXU];
        int nu = 0;
#pragma unroll
        for (int u = 0; u < MAXU; ++u) {
            jn[u] = jlo + par + NPAR * u;
            if (jn[u] <= jhi) nu = u + 1;
        }
        const int64_t N = p.N;
        auto load_z = [&](int g, float (&zz)[MAXU][J]) {
            const int64_t pt = int64_t(g) * GROUP + pp;
            const float* zp = p.z + (pt < N ? pt : N - 1);
#pragma unroll
            for (int u = 0; u < MAXU; ++u)
#pragma unroll
                for (int r = 0; r < J; ++r) {
                    if constexpr (FIRST) {
                        // first layer: the coordinate x_j, dx_j/dx_d = [j == d], no second derivative
                        const int j = u < nu ? jn[u] : 0;
                        if (r == 0) zz[u][r] = zp[int64_t(j) * N];
                        else if (r == JT::RF0 && JT::F0) zz[u][r] = j == 0 ? 1.0f : 0.0f;
                        else if (r == JT::RF1 && JT::F1) zz[u][r] = j == 1 ? 1.0f : 0.0f;
                        else zz[u][r] = 0.0f;
                    } else {
                        zz[u][r] = u < nu ? zp[(int64_t(r) * I + jn[u]) * N] : 0.0f;
                    }
                }
        };
        // K-range entries of no unit (past the last one) must be zero: no unit
        // ever writes them, so they are cleared once in every A tile of every
        // slot (the first publication of each slot makes them visible to the MMAs)
        if (par == 0) {
            for (int m = (jhi + 1) * NP8 - k0; m < 128; m += 8) {
                if (m < 0) continue;
                for (int b = 0; b < nsg; ++b)
                    for (int r = 0; r < J; ++r)
                        st_shared_v4(smem_u32(smem + size_t(b) * slot_bytes + size_t(r) * A_BYTES) + a_off(m, pp),
                                     0u, 0u, 0u, 0u);
            }
        }
        float zn[MAXU][J];
        if (ng > 0) load_z(g0, zn);
        for (int gi = 0; gi < ng; ++gi) {
            float zc[MAXU][J];
#pragma unroll
            for (int u = 0; u < MAXU; ++u)
#pragma unroll
                for (int r = 0; r < J; ++r) zc[u][r] = zn[u][r];
            if (gi + 1 < ng) load_z(g0 + gi + 1, zn);
            // store unit u's J rows (its NC chunks of 8 elements that fall in the range) into the slot
            auto store_unit = [&](int u, const Win& w, uint32_t sbase) {
                const int kb = jn[u] * NP8 - k0;   // k of the unit's first element, relative to the range
#pragma unroll
                for (int ci = 0; ci < NC; ++ci) {
                    const int m = kb + 8 * ci;
                    if (m >= 0 && m < 128) {
                        const uint32_t off = a_off(m, pp);
#pragma unroll
                        for (int r = 0; r < J; ++r) {
                            uint32_t v[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int lw = 4 * ci + e, qr = lw / QW, qo = lw % QW;
                                v[e] = w.tw[qr] == qo ? w.y[r][qr] : 0u;
                            }
                            st_shared_v4(sbase + uint32_t(r) * A_BYTES + off, v[0], v[1], v[2], v[3]);
                        }
                    }
                }
            };
            const int b = gi % nsg;
            const uint32_t ph = uint32_t(gi / nsg) & 1u;
            const uint32_t sbase = smem_u32(smem + size_t(b) * slot_bytes);
            if constexpr (EARLY) {
                Win w[MAXU];
#pragma unroll
                for (int u = 0; u < MAXU; ++u)
                    if (u < nu) tck::unit_window<MASK, HRKAN_BF16>(zc[u], p.g, true, w[u]);
                if (!__all_sync(0xffffffffu, mbar_wait(&bar_empty[b], ph ^ 1u, abort, wl))) goto done;
#pragma unroll
                for (int u = 0; u < MAXU; ++u)
                    if (u < nu) store_unit(u, w[u], sbase);
            } else {
                if (!__all_sync(0xffffffffu, mbar_wait(&bar_empty[b], ph ^ 1u, abort, wl))) goto done;
#pragma unroll
                for (int u = 0; u < MAXU; ++u) {
                    if (u < nu) {
                        Win w;
                        tck::unit_window<MASK, HRKAN_BF16>(zc[u], p.g, true, w);
                        store_unit(u, w, sbase);
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            mbar_arrive_if(&bar_full[b], lane == 0);
        }
        // ---- epilogue (warps 0-3, one TMEM lane quarter each): D (lanes = k of the range) -> partial row
        if (warp < 4) {
            if (ng > 0) {
                if (!__all_sync(0xffffffffu, mbar_wait(&bar_accfull, 0u, abort, wl))) goto done;
            }
            tc_fence_after();
            const int k = k0 + warp * 32 + lane;
            // element pos of the unit holds basis 4 * (pos mod NP8/4) + pos / (NP8/4)
            const int j = k / NP8, pos = k % NP8, i = 4 * (pos % (NP8 / 4)) + pos / (NP8 / 4);
            const bool live = j < I && i < p.n;
            float* out = p.partial + int64_t(out_row) * p.P + p.col0 + int64_t(j) * p.n + i;
            const uint32_t lane_base = uint32_t(warp * 32) << 16;
#pragma unroll 1
            for (int c = 0; c < O; c += 16) {
                uint32_t v[16];
                if (ng > 0) {
                    tmem_ld16(tbase + lane_base + uint32_t(c), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] = 0u;
                }
                if (live)
#pragma unroll
                    for (int e = 0; e < 16; ++e) out[int64_t(c + e) * I * p.n] = __uint_as_float(v[e]);
            }
        }
    } else if (warp == NPROD) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0 && ng > 0) {
            // kind::f16, BF16 A (MN-major) and B (K-major), FP32 D, M = 128, N = O
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (uint32_t(O >> 3) << 17) |
                                   (uint32_t(128 >> 4) << 24);
            bool issued = false;
            for (int gi = 0; gi < ng; ++gi) {
                const int b = gi % nsg;
                if (!mbar_wait(&bar_full[b], uint32_t(gi / nsg) & 1u, abort, wl)) break;
                tc_fence_after();
                const uint32_t sbase = smem_u32(smem + size_t(b) * slot_bytes);
#pragma unroll
                for (int r = 0; r < J; ++r) {
                    const uint32_t abase = sbase + uint32_t(r) * A_BYTES;
                    const uint64_t bd = sdesc(sbase + uint32_t(J) * A_BYTES + uint32_t(r) * b_bytes, 16, 1024);
#pragma unroll
                    for (int ks = 0; ks < GROUP / 16; ++ks) {
                        const uint64_t ad = sdesc(abase + uint32_t(ks) * 4096u, 1024, 2048);
                        const uint32_t acc = (gi > 0 || r > 0 || ks > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred pa;\n\tsetp.ne.b32 pa, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n\t}" ::"r"(tbase),
                            "l"(ad), "l"(bd + uint64_t(2 * ks)), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                }
                issued = true;
                mma_commit(&bar_empty[b]);
            }
            if (!*abort) mma_commit(&bar_accfull);
            else if (issued) {
                mma_commit(&bar_drain);
                mbar_drain(&bar_drain, 0u);
            }
        }
    } else {
        // ------------------------------------------------------------ a group's J gy tiles by TMA
        if (lane == 0 && ng > 0) {
            uint32_t used = 0u, last_par = 0u;
            for (int gi = 0; gi < ng; ++gi) {
                const int b = gi % nsg;
                const uint32_t ph = uint32_t(gi / nsg) & 1u;
                if (!mbar_wait(&bar_empty[b], ph ^ 1u, abort, wl)) break;
                mbar_expect_tx(&bar_full[b], uint32_t(J) * b_bytes);
                uint8_t* gdst = smem + size_t(b) * slot_bytes + size_t(J) * A_BYTES;
                for (int r = 0; r < J; ++r)
                    tck::tma_load_2d(gdst + size_t(r) * b_bytes, &gmap, &bar_full[b], (g0 + gi) * GROUP, r * O);
                used |= 1u << b;
                last_par = (last_par & ~(1u << b)) | (ph << b);
            }
            if (*abort)
                for (int b = 0; b < nsg; ++b)
                    if ((used >> b) & 1u) mbar_drain(&bar_full[b], (last_par >> b) & 1u);
        }
    }
done:
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicExch(p.status, tck::ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(p.tmem_cols)
                     : "memory");
}

// gy [J][O][N] float32 -> [J*O][Npad] BF16, zero for points >= N; one thread
// converts 8 consecutive points of a row and stores them as one 16-byte word.
__global__ void gy_bf16_kernel(const float* __restrict__ gy, uint16_t* __restrict__ out, int64_t rows, int64_t N,
                               int64_t Npad) {
    const int64_t per_row = Npad / 8, total = rows * per_row;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t row = t / per_row, c0 = (t % per_row) * 8;
        const float* src = gy + row * N + c0;
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float a = c0 + 2 * e < N ? src[2 * e] : 0.0f;
            const float b = c0 + 2 * e + 1 < N ? src[2 * e + 1] : 0.0f;
            w[e] = uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(a))) |
                   (uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(b))) << 16);
        }
        *reinterpret_cast<uint4*>(out + row * Npad + c0) = make_uint4(w[0], w[1], w[2], w[3]);
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

int np8_of(int n) { return std::max(16, (n + 7) / 8 * 8); }

template <unsigned MASK, int NC, bool FIRST, bool EARLY>
cudaError_t launch(const DwParams& p, const CUtensorMap& map, unsigned grid, cudaStream_t s) {
    const int J = __builtin_popcount(MASK & 0x1Fu);
    const size_t smem = size_t(p.nsb) * J * (A_BYTES + size_t(p.O) * 128) + 1024;
    auto kern = tc_dw_kernel<MASK, NC, FIRST, EARLY>;
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
    kern<<<grid, THREADS, smem, s>>>(p, map);
    return cudaGetLastError();
}

template <unsigned MASK, int NC, bool FIRST>
cudaError_t launch_e(bool early, const DwParams& p, const CUtensorMap& map, unsigned grid, cudaStream_t s) {
    // a single slot only fits for J = 5 (mask 0x1F) and O >= 48
    if constexpr (MASK == 0x1Fu)
        if (early) return launch<MASK, NC, FIRST, true>(p, map, grid, s);
    return launch<MASK, NC, FIRST, false>(p, map, grid, s);
}

template <unsigned MASK, bool FIRST>
cudaError_t launch_nc(int nc, const DwParams& p, const CUtensorMap& map, unsigned grid, cudaStream_t s) {
    const bool early = p.nsb == 1;
    switch (nc) {
        case 2: return launch_e<MASK, 2, FIRST>(early, p, map, grid, s);
        case 3: return launch_e<MASK, 3, FIRST>(early, p, map, grid, s);
        case 4: return launch_e<MASK, 4, FIRST>(early, p, map, grid, s);
        case 5: return launch_e<MASK, 5, FIRST>(early, p, map, grid, s);
        case 6: return launch_e<MASK, 6, FIRST>(early, p, map, grid, s);
        case 7: return launch_e<MASK, 7, FIRST>(early, p, map, grid, s);
        case 8: return launch_e<MASK, 8, FIRST>(early, p, map, grid, s);
    }
    return cudaErrorNotSupported;
}

}  // namespace tcdw

cudaError_t tc_gy_to_bf16(const float* gy, void* gy_bf, int J, int O, int64_t N, cudaStream_t s) {
    const int64_t Npad = (std::max<int64_t>(N, 1) + 63) / 64 * 64;
    const int64_t rows = int64_t(J) * O, total = rows * (Npad / 8);
    const int pb = int(std::min<int64_t>((total + 255) / 256, 8192));
    tcdw::gy_bf16_kernel<<<pb, 256, 0, s>>>(gy, static_cast<uint16_t*>(gy_bf), rows, N, Npad);
    return cudaGetLastError();
}

bool tc_dw_supported(int prec, int I, int O, int n, unsigned mask) {
    if (prec != HRKAN_BF16) return false;
    if (O < 16 || O > 64 || O % 16 != 0 || n > 64 || n < 1 || I < 1) return false;
    return mask == 0x01u || mask == 0x0Fu || mask == 0x1Fu;
}

int64_t tc_dw_gy_elems(int J, int O, int64_t N) { return int64_t(J) * O * ((N + 63) / 64 * 64); }

cudaError_t tc_dw_layer(const float* z, const float* gy, void* gy_bf, int I, int O, int64_t N, const Grid& g,
                        unsigned mask, bool first, float* partial, int64_t P, int64_t col0, int row0, int nchunk,
                        int* status, cudaStream_t s, const int4* chunks, bool gy_ready) {
    using namespace tcdw;
    const int J = __builtin_popcount(mask & 0x1Fu);
    const int n = g.n, np8 = np8_of(n);
    const int64_t Npad = (std::max<int64_t>(N, 1) + 63) / 64 * 64;
    const int64_t rows = int64_t(J) * O;
    if (!gy_ready)
        if (cudaError_t e = tc_gy_to_bf16(gy, gy_bf, J, O, N, s)) return e;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[2] = {cuuint64_t(Npad), cuuint64_t(rows)};
    const cuuint64_t strides[1] = {cuuint64_t(Npad) * 2};
    const cuuint32_t box[2] = {cuuint32_t(GROUP), cuuint32_t(O)};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, gy_bf, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    DwParams p{};
    p.z = z;
    p.partial = partial;
    p.P = P;
    p.col0 = col0;
    p.row0 = row0;
    p.nchunk = nchunk;
    p.I = I;
    p.O = O;
    p.n = n;
    p.np8 = np8;
    p.N = N;
    p.ngroups = int(Npad / GROUP);
    p.nkr = (I * np8 + 127) / 128;
    p.tmem_cols = O <= 32 ? 32u : 64u;
    p.g = g;
    p.status = status;
    p.chunks = chunks;
    // ring: all NSB buffers (measured on the 16-wide hidden layer: a ring of
    // J = 5 buffers with two CTAs per SM took 5.1 ms per step against 4.05 ms
    // with 8 buffers and one CTA, since a group waits for all J of them)
    // one CTA per SM: as many group slots as SLOT_BUDGET holds (J = 5, O = 16: two)
    p.nsb = std::max(1, std::min(NSB, int(SLOT_BUDGET / (size_t(J) * (A_BYTES + size_t(O) * 128)))));
    const unsigned grid = unsigned(p.nkr) * unsigned(nchunk);
    const int nc = np8 / 8;
    if (first) {
        switch (mask) {
            case 0x01u: return launch_nc<0x01u, true>(nc, p, map, grid, s);
            case 0x0Fu: return launch_nc<0x0Fu, true>(nc, p, map, grid, s);
            case 0x1Fu: return launch_nc<0x1Fu, true>(nc, p, map, grid, s);
        }
    } else {
        switch (mask) {
            case 0x01u: return launch_nc<0x01u, false>(nc, p, map, grid, s);
            case 0x0Fu: return launch_nc<0x0Fu, false>(nc, p, map, grid, s);
            case 0x1Fu: return launch_nc<0x1Fu, false>(nc, p, map, grid, s);
        }
    }
    return cudaErrorNotSupported;
}

}  // namespace hrkan
