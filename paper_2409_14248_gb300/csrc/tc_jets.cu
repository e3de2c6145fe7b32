// Host side of the tensor-core layer (kernel: tc_kernel.cuh): weight
// conversion into the padded K layout, the TMA descriptor, the choice of the
// unit padding NP and of the A ring, and the launch.
#include <cuda.h>

#include <algorithm>
#include <cuda_bf16.h>
#include <mutex>

#include "internal.h"
#include "tc.cuh"

namespace hrkan {

cudaError_t tc_launch_np16(const TcLayer&, const CUtensorMap&, int, unsigned, cudaStream_t);
cudaError_t tc_launch_np24(const TcLayer&, const CUtensorMap&, int, unsigned, cudaStream_t);
cudaError_t tc_launch_np32(const TcLayer&, const CUtensorMap&, int, unsigned, cudaStream_t);
cudaError_t tc_launch_np40(const TcLayer&, const CUtensorMap&, int, unsigned, cudaStream_t);
cudaError_t tc_launch_np48(const TcLayer&, const CUtensorMap&, int, unsigned, cudaStream_t);
cudaError_t tc_launch_np64(const TcLayer&, const CUtensorMap&, int, unsigned, cudaStream_t);

namespace {

constexpr int TMEM_COLS = 512;
constexpr int RING_MAX = 8;

// Smallest supported padding of a unit's n bases (0 = none).
int np_of(int n) {
    for (int np : {16, 24, 32, 40, 48, 64})
        if (n <= np) return np;
    return 0;
}
// Basis positions per slot (one MMA) and per 128-byte W row: 8 and 32 for
// TF32 and for the BF16 pair layout (one 32-bit word per basis).
int slot_elems(int) { return 8; }
int box_elems(int) { return 32; }
// Weight tiles of O rows per W buffer: (w_hi, w_hi) and (w_lo, 0) for BF16.
int w_terms(int prec) { return prec == HRKAN_BF16 ? 2 : 1; }
// A ring slots left in `cols` TMEM columns after the J * O accumulator columns
// (8 columns per slot and jet row).
int ring_slots(int J, int O, int cols = TMEM_COLS) { return std::min(RING_MAX, (cols - J * O) / (8 * J)); }
// Small layers (J * O + 4 ring slots within 256 columns) allocate half of TMEM
// so that two CTAs share an SM: twice the producer warps per SM to hide the
// latency of the per-slot hand-offs, and one CTA's tile boundary (the drain of
// the MMA pipe before its epilogue) overlaps the other's work.
int tmem_cols_for(int J, int O, int prec) {
    const size_t wbytes = size_t(TC_W_BUFFERS) * w_terms(prec) * O * 128 + 1024;   // shared memory of one CTA
    return ring_slots(J, O, 256) >= 4 && 2 * wbytes <= 200 * 1024 ? 256 : TMEM_COLS;
}

// W [O][I][n] float32 -> 32-bit words [TERMS][O][Kt]: word k = j * NP + pos
// holds W[o][j][i], i = 4 * (pos mod NP/4) + pos / (NP/4) (the bases of a unit
// stored by residue mod 4), for i < n and j < I, zero elsewhere.  TF32: the
// TF32-rounded float32.  BF16 (three-term split): tile 0 holds (w_hi, w_hi) in
// the word's low and high halves, tile 1 (w_lo, 0), w_hi = bf16(w),
// w_lo = bf16(w - w_hi).
// Many instances: instance c's layer at W + c * w_stride goes to
// out + c * TERMS * O * Kt.
template <int PREC>
__global__ void tc_prep_w_kernel(const float* __restrict__ W, uint32_t* out, int O, int I, int n, int NP, int Kt,
                                 int n_inst, int64_t w_stride) {
    const int64_t total = int64_t(O) * Kt;
    constexpr int TERMS = PREC == HRKAN_BF16 ? 2 : 1;
    for (int64_t u = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < total * n_inst;
         u += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = u / total, t = u % total;
        const int o = int(t / Kt), k = int(t % Kt);
        const int j = k / NP, pos = k % NP, q = NP / 4, i = 4 * (pos % q) + pos / q;
        const float w = (j < I && i < n) ? W[c * w_stride + (int64_t(o) * I + j) * n + i] : 0.0f;
        uint32_t* oc = out + c * TERMS * total;
        if constexpr (PREC == HRKAN_BF16) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(w);
            const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(w - __bfloat162float(hi)));
            const uint32_t hb = __bfloat16_as_ushort(hi);
            oc[t] = hb | (hb << 16);
            oc[total + t] = lo;
        } else {
            uint32_t r;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(w));
            oc[t] = r;
        }
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

// K layout of one layer: slots (one MMA each) over I units of NP elements, and
// the W tiles of 128 bytes per row that cover them.
struct KLayout {
    int np, ks, nbox, kt;
};
KLayout k_layout(int I, int n, int prec) {
    KLayout L{};
    L.np = np_of(n);
    const int se = slot_elems(prec), be = box_elems(prec);
    L.ks = (I * L.np + se - 1) / se;
    L.nbox = (L.ks * se + be - 1) / be;
    L.kt = L.nbox * be;
    return L;
}

}  // namespace

bool tc_layer_supported(int prec, int I, int O, int n, unsigned mask) {
    const int J = __builtin_popcount(mask & 0x1Fu);
    if (prec != HRKAN_BF16 && prec != HRKAN_TF32) return false;
    if (O < 16 || O > 64 || O % 16 != 0 || J * O > 320) return false;
    if (np_of(n) == 0 || ring_slots(J, O) < 2) return false;
    return I >= 1 && (mask == 0x01u || mask == 0x0Fu || mask == 0x1Fu);
}

int64_t tc_w_elems(int O, int I, int n, int prec) { return int64_t(w_terms(prec)) * O * k_layout(I, n, prec).kt; }

cudaError_t tc_forward_layer(const float* W, void* w_prep, const float* z, float* y, int I, int O, int64_t N,
                             const Grid& g, int prec, unsigned mask, int* status, cudaStream_t s, int n_inst,
                             int64_t w_stride, const int* blk_inst) {
    if (N == 0) return cudaSuccess;
    if (n_inst < 1 || (n_inst > 1 && !blk_inst)) return cudaErrorInvalidValue;
    const int n = g.n;
    const KLayout L = k_layout(I, n, prec);
    const int64_t total = int64_t(O) * L.kt * n_inst;
    const int pb = int(std::min<int64_t>((total + 255) / 256, 4096));
    uint32_t* wp = static_cast<uint32_t*>(w_prep);
    if (prec == HRKAN_BF16)
        tc_prep_w_kernel<HRKAN_BF16><<<pb, 256, 0, s>>>(W, wp, O, I, n, L.np, L.kt, n_inst, w_stride);
    else
        tc_prep_w_kernel<HRKAN_TF32><<<pb, 256, 0, s>>>(W, wp, O, I, n, L.np, L.kt, n_inst, w_stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // rows of 32-bit words: per instance the TERMS tiles of O rows each
    // stacked, one box (32 words x TERMS*O rows) per W buffer of the kernel
    const int rows = w_terms(prec) * O;
    CUtensorMap map;
    const cuuint64_t dims[2] = {cuuint64_t(L.kt), cuuint64_t(rows) * cuuint64_t(n_inst)};
    const cuuint64_t strides[1] = {cuuint64_t(L.kt) * 4};
    const cuuint32_t box[2] = {cuuint32_t(box_elems(prec)), cuuint32_t(rows)};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, w_prep, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int J = __builtin_popcount(mask & 0x1Fu);
    TcLayer p{};
    p.z = z;
    p.y = y;
    p.I = I;
    p.O = O;
    p.N = N;
    p.ks = L.ks;
    p.nbox = L.nbox;
    p.tmem_cols = uint32_t(tmem_cols_for(J, O, prec));
    p.ring = ring_slots(J, O, int(p.tmem_cols));
    p.ntiles = int((N + 127) / 128);
    p.g = g;
    p.status = status;
    p.blk_inst = n_inst > 1 ? blk_inst : nullptr;
    switch (L.np) {
        case 16: return tc_launch_np16(p, map, prec, mask, s);
        case 24: return tc_launch_np24(p, map, prec, mask, s);
        case 32: return tc_launch_np32(p, map, prec, mask, s);
        case 40: return tc_launch_np40(p, map, prec, mask, s);
        case 48: return tc_launch_np48(p, map, prec, mask, s);
        case 64: return tc_launch_np64(p, map, prec, mask, s);
    }
    return cudaErrorNotSupported;
}

}  // namespace hrkan
