// hrkan_backward_noalloc: the weight-gradient backward of the fused narrow
// networks for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another framework's
// memory pool or allocator hooks, inside a region where allocation would break
// a stream-ordered or capture-time contract, or embedded hosts whose device
// memory is fully reserved up front.  Such a caller cannot create a handle
// (hrkan_init allocates its workspace), so this entry point takes the network
// shape directly and keeps its per-block gradient partials in a file-scope
// static device array instead of a handle's workspace.  It allocates nothing:
// no cudaMalloc, no cudaFree, no allocating library routine.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "../../include/hrkan.h"
#include "internal.h"
#include "narrow.cuh"

namespace {

using namespace hrkan;

// 1 Mi floats (4 MiB) of per-block partial rows, held by every device that
// loads the library until the process exits.
constexpr int64_t kScratchFloats = int64_t(1) << 20;
static __device__ __align__(256) float g_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the scratch address and the id of the context it was looked up
// in.  A module-scope __device__ array lives in the context's copy of the
// module: after cudaDeviceReset, or when the primary context is released and
// created again, the module is loaded anew and the array may sit elsewhere,
// so the address is looked up again whenever the current context's id differs.
struct ScratchAddr {
    float* ptr;
    unsigned long long ctx_id;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the current driver context (0: none, or the driver lacks cuCtxGetId).
unsigned long long current_ctx_id() {
    static std::once_flag once;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        else
            cudaGetLastError();
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        else
            cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_scratch on the current device.  The name g_scratch in
// host code is only a host-side stand-in, so the address is looked up (with
// that device current) on the first call in each context and cached with the
// context's id.
int scratch_on_current_device(float** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_last_error(HRKAN_ECUDA, "hrkan_backward_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return set_last_error(HRKAN_EUNSUPPORTED, "hrkan_backward_noalloc: device ordinal >= 64");
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchAddr& a = g_scratch_addr[dev];
    const unsigned long long id = current_ctx_id();
    if (!a.ptr || id == 0 || id != a.ctx_id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);   // makes the device's primary context current if needed
        if (e != cudaSuccess || !p) {
            char buf[256];
            snprintf(buf, sizeof buf, "hrkan_backward_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return set_last_error(HRKAN_ECUDA, buf);
        }
        a.ptr = static_cast<float*>(p);
        a.ctx_id = current_ctx_id();
    }
    *out = a.ptr;
    return HRKAN_OK;
}

}  // namespace

extern "C" int hrkan_backward_noalloc(const hrkan_cfg* cfg, const float* W, const float* x, int64_t N,
                                      unsigned jet_mask, const float* dL_djets, float* dW, int accumulate,
                                      hrkan_stream_t stream) {
    char buf[256];
    if (!cfg) return set_last_error(HRKAN_EINVAL, "hrkan_backward_noalloc: cfg is NULL");
    const int64_t P = hrkan_param_count(cfg);
    if (P <= 0) return set_last_error(HRKAN_EINVAL, "hrkan_backward_noalloc: invalid network configuration");
    if (cfg->k != 3 || cfg->m != 4 || cfg->prec != HRKAN_FP32 || cfg->n_instances != 1 || cfg->widths[0] != 2)
        return set_last_error(HRKAN_EUNSUPPORTED, "hrkan_backward_noalloc: needs k=3, m=4, FP32, one instance, D=2");
    const int L = cfg->n_widths - 1;
    bool uniform = true;
    for (int l = 1; l < L; ++l) uniform &= (cfg->widths[l] == cfg->widths[1]);
    const int net_id = uniform ? narrow_net_id(L, cfg->widths[1]) : -1;
    if (net_id < 0) return set_last_error(HRKAN_EUNSUPPORTED, "hrkan_backward_noalloc: no fused kernel for this shape");
    if (P > kScratchFloats) {
        snprintf(buf, sizeof buf, "hrkan_backward_noalloc: %lld weights exceed the static scratch of %lld floats",
                 (long long)P, (long long)kScratchFloats);
        return set_last_error(HRKAN_EINVAL, buf);
    }
    if (N < 0) return set_last_error(HRKAN_EINVAL, "hrkan_backward_noalloc: N < 0");
    if (!(jet_mask & 1u) || (jet_mask & ~0x1Fu) || ((jet_mask & 0x08u) && !(jet_mask & 0x02u)) ||
        ((jet_mask & 0x10u) && !(jet_mask & 0x04u)))
        return set_last_error(HRKAN_EINVAL, "hrkan_backward_noalloc: invalid jet mask");
    if (!W || !dW || (N > 0 && (!x || !dL_djets)))
        return set_last_error(HRKAN_EINVAL, "hrkan_backward_noalloc: NULL device pointer");
    cudaStream_t s = (cudaStream_t)stream;
    if (N == 0) {
        if (!accumulate && cudaMemsetAsync(dW, 0, size_t(P) * sizeof(float), s) != cudaSuccess)
            return set_last_error(HRKAN_ECUDA, "hrkan_backward_noalloc: cudaMemsetAsync failed");
        return HRKAN_OK;
    }
    float* scratch = nullptr;
    if (int rc = scratch_on_current_device(&scratch)) return rc;

    const double hh = (cfg->grid_hi - cfg->grid_lo) / cfg->G;
    NarrowParams p{};
    p.W = W;
    p.grid.lo = float(cfg->grid_lo);
    p.grid.h = float(hh);
    p.grid.inv_h = float(1.0 / hh);
    p.grid.inv_a = float(2.0 / ((cfg->k + 1) * hh));
    p.grid.m = cfg->m;
    p.grid.n = cfg->G + cfg->k;
    p.P = P;
    p.x0 = x;
    p.n0 = N;
    p.dL = dL_djets;
    p.partial = scratch;   // every block overwrites its whole row: nothing to clear
    // one partial row per block: the grid is capped by the rows that fit
    const int max_rows = int(kScratchFloats / P);
    int grid = 0;
    cudaError_t e = narrow_launch(net_id, MODE_BWD, jet_mask, p, &grid, max_rows, true, s);
    if (e == cudaErrorNotSupported)
        return set_last_error(HRKAN_EUNSUPPORTED, "hrkan_backward_noalloc: jet mask has no backward kernel");
    if (e != cudaSuccess) {
        snprintf(buf, sizeof buf, "hrkan_backward_noalloc: launch failed: %s", cudaGetErrorString(e));
        return set_last_error(HRKAN_ECUDA, buf);
    }
    ReduceParams q{};
    q.partial = scratch;
    q.G = grid;
    q.P = P;
    q.dW = dW;
    q.accumulate = accumulate ? 1 : 0;
    e = launch_reduce(q, s);
    if (e != cudaSuccess) {
        snprintf(buf, sizeof buf, "hrkan_backward_noalloc: reduce launch failed: %s", cudaGetErrorString(e));
        return set_last_error(HRKAN_ECUDA, buf);
    }
    return HRKAN_OK;
}
