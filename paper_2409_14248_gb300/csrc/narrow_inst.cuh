// Instantiates the fused narrow-network kernels of one shape and a launcher.
#pragma once

#include <mutex>
#include <unordered_map>

#include "internal.h"
#include "narrow.cuh"

namespace hrkan {

// Raise a kernel's dynamic shared-memory limit to what a launch needs; the
// limit only grows, so repeated launches (including ones under stream
// capture) make no attribute calls.
template <class KernelT>
static cudaError_t allow_big_smem(KernelT kern, size_t bytes) {
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> set_to;
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = set_to[reinterpret_cast<const void*>(kern)];
    if (bytes <= cur) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) cur = bytes;
    else cudaGetLastError();
    return e;
}

template <class Net, class KernelT>
static cudaError_t narrow_go(KernelT kern, size_t smem, int64_t tiles, const NarrowParams& p, int* grid,
                             int max_grid, bool launch, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024 && (e = allow_big_smem(kern, smem)) != cudaSuccess) return e;
    if (*grid <= 0) {
        int dev = 0, nsm = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NARROW_BLOCK, smem)) != cudaSuccess)
            return e;
        int64_t g = int64_t(nsm) * (occ > 0 ? occ : 1);
        if (g > max_grid) g = max_grid;
        if (g > tiles) g = tiles;
        *grid = (int)(g > 0 ? g : 1);
    }
    if (!launch) return cudaSuccess;
    kern<<<*grid, NARROW_BLOCK, smem, s>>>(p);
    return cudaGetLastError();
}

template <class Net>
static cudaError_t narrow_launch_net(int mode, unsigned mask, const NarrowParams& p, int* grid, int max_grid,
                                     bool launch, cudaStream_t s) {
    const int n = p.grid.n;
    const size_t sf = size_t(Net::smem_floats(n)) * sizeof(float);
    const int64_t t0 = (p.n0 + NARROW_BLOCK - 1) / NARROW_BLOCK;
    const int64_t t1 = (p.n1 + NARROW_BLOCK - 1) / NARROW_BLOCK;
    if (mode == MODE_FWD) {
        switch (mask) {
            case 0x01u: return narrow_go<Net>(narrow_fwd_kernel<Net, 0x01u>, sf, t0, p, grid, max_grid, launch, s);
            case 0x0Fu: return narrow_go<Net>(narrow_fwd_kernel<Net, 0x0Fu>, sf, t0, p, grid, max_grid, launch, s);
            case 0x1Fu: return narrow_go<Net>(narrow_fwd_kernel<Net, 0x1Fu>, sf, t0, p, grid, max_grid, launch, s);
        }
    } else if (mode == MODE_BWD) {
        switch (mask) {
            case 0x01u: return narrow_go<Net>(narrow_grad_kernel<Net, 0x01u, MODE_BWD>, (1 + Net::COPIES) * sf, t0, p, grid, max_grid, launch, s);
            case 0x0Fu: return narrow_go<Net>(narrow_grad_kernel<Net, 0x0Fu, MODE_BWD>, (1 + Net::COPIES) * sf, t0, p, grid, max_grid, launch, s);
            case 0x1Fu: return narrow_go<Net>(narrow_grad_kernel<Net, 0x1Fu, MODE_BWD>, (1 + Net::COPIES) * sf, t0, p, grid, max_grid, launch, s);
        }
    } else if (mode == MODE_TRAIN) {
        switch (mask) {
            case 0x0Fu: return narrow_go<Net>(narrow_grad_kernel<Net, 0x0Fu, MODE_TRAIN>, (1 + Net::COPIES) * sf, t0 + t1, p, grid, max_grid, launch, s);
            case 0x1Fu: return narrow_go<Net>(narrow_grad_kernel<Net, 0x1Fu, MODE_TRAIN>, (1 + Net::COPIES) * sf, t0 + t1, p, grid, max_grid, launch, s);
        }
    }
    return cudaErrorNotSupported;
}

template <class Net>
static cudaError_t narrow_batch_launch_net(int mode, unsigned mask, const BatchParams& p, int* grid, int max_grid,
                                           bool launch, cudaStream_t s) {
    const size_t sf = size_t(Net::smem_floats(p.grid.n)) * sizeof(float);
    const int64_t items = p.n_items;
    auto go = [&](auto kern, size_t smem) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (smem > 48 * 1024 && (e = allow_big_smem(kern, smem)) != cudaSuccess) return e;
        if (*grid <= 0) {
            int dev = 0, nsm = 0, occ = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NARROW_BLOCK, smem)) != cudaSuccess)
                return e;
            int64_t g = int64_t(nsm) * (occ > 0 ? occ : 1);
            if (g > max_grid) g = max_grid;
            if (g > items) g = items;
            *grid = (int)(g > 0 ? g : 1);
        }
        if (!launch) return cudaSuccess;
        kern<<<*grid, NARROW_BLOCK, smem, s>>>(p);
        return cudaGetLastError();
    };
    if (mode == MODE_FWD) {
        switch (mask) {
            case 0x01u: return go(narrow_batch_fwd_kernel<Net, 0x01u>, sf);
            case 0x0Fu: return go(narrow_batch_fwd_kernel<Net, 0x0Fu>, sf);
            case 0x1Fu: return go(narrow_batch_fwd_kernel<Net, 0x1Fu>, sf);
        }
    } else if (mode == MODE_TRAIN) {
        switch (mask) {
            case 0x0Fu: return go(narrow_batch_kernel<Net, 0x0Fu>, (1 + Net::COPIES) * sf);
            case 0x1Fu: return go(narrow_batch_kernel<Net, 0x1Fu>, (1 + Net::COPIES) * sf);
        }
    }
    return cudaErrorNotSupported;
}

}  // namespace hrkan

#define HRKAN_NARROW_INSTANCE(FN, NL, WH)                                                               \
    namespace hrkan {                                                                                   \
    cudaError_t FN(int mode, unsigned mask, const NarrowParams& p, int* grid, int max_grid, bool launch, \
                   cudaStream_t s) {                                                                    \
        return narrow_launch_net<NarrowNet<NL, WH, 3, 4>>(mode, mask, p, grid, max_grid, launch, s);   \
    }                                                                                                   \
    cudaError_t FN##_batch(int mode, unsigned mask, const BatchParams& p, int* grid, int max_grid,       \
                           bool launch, cudaStream_t s) {                                               \
        return narrow_batch_launch_net<NarrowNet<NL, WH, 3, 4>>(mode, mask, p, grid, max_grid, launch, s); \
    }                                                                                                   \
    }
