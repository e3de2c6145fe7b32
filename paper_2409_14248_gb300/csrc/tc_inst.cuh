// Instantiates the tensor-core kernels for one unit padding HRKAN_TC_NP and
// defines its launcher (included by tc_np*.cu, one translation unit each so
// that they compile in parallel).
#pragma once

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "tc_kernel.cuh"

namespace hrkan {
namespace tck {

template <unsigned MASK, int PREC, int NP>
cudaError_t launch_one(const TcLayer& p, const CUtensorMap& map, cudaStream_t s) {
    // NB W buffers (TERMS tiles of O rows each) + alignment slack.  A CTA that
    // allocates all 512 TMEM columns asks for at least 120 KB so that it holds
    // an SM alone; with 256 columns two CTAs share an SM
    const size_t wbytes = size_t(NB) * Elem<PREC>::TERMS * p.O * 128 + 1024;
    const size_t want = p.tmem_cols >= 512 ? std::max<size_t>(wbytes, 120 * 1024) : wbytes;
    const int per_sm = p.tmem_cols >= 512 ? 1 : 2;   // the host picks 256 columns only when two fit
    auto kern = tc_fwd_kernel<MASK, PREC, NP>;
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
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = unsigned(std::max(1, std::min(p.ntiles, per_sm * nsm)));
    kern<<<grid, THREADS, want, s>>>(p, map);
    return cudaGetLastError();
}

}  // namespace tck

#define HRKAN_TC_CAT2(a, b) a##b
#define HRKAN_TC_CAT(a, b) HRKAN_TC_CAT2(a, b)
cudaError_t HRKAN_TC_CAT(tc_launch_np, HRKAN_TC_NP)(const TcLayer& p, const CUtensorMap& map, int prec,
                                                     unsigned mask, cudaStream_t s) {
    constexpr int NP = HRKAN_TC_NP;
    if (prec == HRKAN_BF16) {   // the three-term split (TC_BF16X3)
        switch (mask) {
            case 0x01u: return tck::launch_one<0x01u, TC_BF16X3, NP>(p, map, s);
            case 0x0Fu: return tck::launch_one<0x0Fu, TC_BF16X3, NP>(p, map, s);
            case 0x1Fu: return tck::launch_one<0x1Fu, TC_BF16X3, NP>(p, map, s);
        }
    } else if (prec == HRKAN_TF32) {
        switch (mask) {
            case 0x01u: return tck::launch_one<0x01u, HRKAN_TF32, NP>(p, map, s);
            case 0x0Fu: return tck::launch_one<0x0Fu, HRKAN_TF32, NP>(p, map, s);
            case 0x1Fu: return tck::launch_one<0x1Fu, HRKAN_TF32, NP>(p, map, s);
        }
    }
    return cudaErrorNotSupported;
}

}  // namespace hrkan
