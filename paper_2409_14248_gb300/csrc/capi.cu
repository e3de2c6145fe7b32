// C ABI of the HRKAN library (declared in include/hrkan.h): argument
// validation, the handle (workspace and Adam moments), and dispatch to the
// kernels.  Nothing here computes on the host beyond launch geometry.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

#include "../../include/hrkan.h"
#include "internal.h"
#include "narrow.cuh"
#include "wide.cuh"
#include "tc.cuh"

using namespace hrkan;

struct hrkan_ctx {
    hrkan_cfg cfg;
    int L = 0;            // layers
    int n = 0;            // bases per unit
    int64_t P = 0;        // weights per network
    int net_id = -1;      // fused narrow shape id
    Grid grid{};
    int device = 0;
    int nsm = 0;
    int max_grid = 0;     // rows of partial
    float* partial = nullptr;        // [max_grid][P]
    int max_grid_l = 0;   // rows of loss_partial
    double* loss_partial = nullptr;  // [max_grid_l][2]
    double* m1 = nullptr;
    double* m2 = nullptr;
    int* t_counter = nullptr;        // [2] device Adam step counter (t = 0 mode)
    int* status = nullptr;           // device error word written by bounded waits
    // first layer: coordinates that jet directions 0 and 1 differentiate along
    // (a three-input network runs its jets as two passes: x and y, then z)
    int seed0 = 0, seed1 = 1;
    // multi-instance work lists (rebuilt only when the offsets or problems change)
    struct Batch {
        std::vector<int64_t> off0, off1;
        std::vector<double> ab;
        int items_points = 0;
        int n_items = 0, cap_items = 0, n_inst = 0, cap_inst = 0;
        BatchItem* items = nullptr;
        BatchInst* inst = nullptr;
        int* item_off = nullptr;
        float* counts = nullptr;
        float* partial = nullptr;
        size_t partial_cap = 0;     // floats
        double* loss_partial = nullptr;
    } train_batch, fwd_batch;
    int batch_items_points = 1024;  // points per work item (layer-wise path: per weight-gradient chunk)
    bool batch_layerwise = false;   // fused shapes: run the multi-instance step on the layer-wise kernels
    // multi-instance path 2: every layer's forward on the FP32 SIMT kernels (the
    // tensor cores for the weight gradient and the input adjoint only)
    bool batch_fwd_simt = false;
    // the layer-wise multi-instance step runs the boundary set's kernels on
    // this stream, forked from and joined back into the caller's stream
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // layer-wise multi-instance layout: every instance's points in whole blocks
    // of LB_BLOCK (rebuilt only when the offsets, problems or chunk size change)
    struct LBatch {
        std::vector<int64_t> off0, off1;
        std::vector<double> ab;
        int n_inst = 0, chunk_blocks = 0;
        bool built = false;
        int64_t NPi = 0, NPb = 0;        // padded point counts of the interior / boundary sets
        int nbi = 0, nbb = 0;            // their point blocks
        int nci = 0, ncb = 0;            // their weight-gradient chunks
        int rows = 0, lrows = 0;         // gradient-partial rows (chunks) and loss-partial rows (blocks)
        void* mem = nullptr;             // every device table below, in one allocation
        size_t mem_bytes = 0;
        int *blk_inst_i = nullptr, *blk_valid_i = nullptr, *pt_src_i = nullptr, *lrow_i = nullptr;
        int *blk_inst_b = nullptr, *blk_valid_b = nullptr, *pt_src_b = nullptr, *lrow_b = nullptr;
        int4 *chunks_i = nullptr, *chunks_b = nullptr;
        int *row_off = nullptr, *loss_off = nullptr;
        BatchInst* inst = nullptr;
        float* counts = nullptr;
        float* partial = nullptr;        // [rows][P]
        size_t partial_cap = 0;
        double* loss_partial = nullptr;  // [lrows][2]
        size_t lp_cap = 0;
    } lb_train, lb_fwd;
    // layer-wise path (shapes without a fused kernel)
    std::vector<int64_t> layer_off;  // first weight of each layer
    int wide_gp = 0;                 // point groups of the weight-gradient kernels
    std::vector<std::pair<float*, size_t>> ws;   // growing scratch slots (floats)
    // kernel timing
    bool prof = false;
    struct Ev { cudaEvent_t a, b; int cls; };
    std::vector<Ev> pending;
    std::vector<Ev> pool;
    double prof_ms[HRKAN_KERNEL_CLASSES] = {};
    int64_t prof_n[HRKAN_KERNEL_CLASSES] = {};
};

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(HRKAN_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define HR_CUDA(call, what)                          \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

int64_t count_params(const hrkan_cfg* c) {
    int64_t P = 0, n = int64_t(c->G) + c->k;
    for (int l = 0; l + 1 < c->n_widths; ++l) P += int64_t(c->widths[l]) * c->widths[l + 1] * n;
    return P;
}

int check_cfg(const hrkan_cfg* c) {
    if (!c) return fail(HRKAN_EINVAL, "cfg is NULL");
    if (c->n_widths < 2 || c->n_widths > HRKAN_MAX_WIDTHS)
        return fail(HRKAN_EINVAL, "n_widths=%d outside [2, %d]", c->n_widths, HRKAN_MAX_WIDTHS);
    for (int l = 0; l < c->n_widths; ++l)
        if (c->widths[l] < 1 || c->widths[l] > 64)
            return fail(HRKAN_EINVAL, "widths[%d]=%d outside [1, 64]", l, c->widths[l]);
    if (c->widths[0] != 2 && c->widths[0] != 3)
        return fail(HRKAN_EUNSUPPORTED, "widths[0]=%d: D = 2 or 3 inputs", c->widths[0]);
    if (c->widths[c->n_widths - 1] != 1)
        return fail(HRKAN_EINVAL, "last width %d: the network has one output", c->widths[c->n_widths - 1]);
    if (c->G < 1 || c->G > 4096) return fail(HRKAN_EINVAL, "G=%d outside [1, 4096]", c->G);
    if (c->k < 0 || c->m < 1) return fail(HRKAN_EINVAL, "k=%d, m=%d", c->k, c->m);
    if (c->k != 3 || c->m < 2 || c->m > 6)
        return fail(HRKAN_EUNSUPPORTED, "k=%d, m=%d: this library has k=3 and m in [2, 6]", c->k, c->m);
    if (!(c->grid_lo < c->grid_hi) || !std::isfinite(c->grid_lo) || !std::isfinite(c->grid_hi))
        return fail(HRKAN_EINVAL, "grid [%g, %g]", c->grid_lo, c->grid_hi);
    if (c->n_instances < 1) return fail(HRKAN_EINVAL, "n_instances=%d", c->n_instances);
    if (c->prec < HRKAN_FP32 || c->prec > HRKAN_TF32) return fail(HRKAN_EINVAL, "prec=%d", c->prec);
    return HRKAN_OK;
}

bool valid_mask(unsigned m) {
    if (!(m & 1u) || (m & ~0xFFFu)) return false;
    if ((m & 0x08u) && !(m & 0x02u)) return false;
    if ((m & 0x10u) && !(m & 0x04u)) return false;
    if ((m & 0x20u) && !(m & 0x08u)) return false;
    if ((m & 0x40u) && !(m & 0x10u)) return false;
    if ((m & 0x80u) && (m & 0x06u) != 0x06u) return false;
    if ((m & 0x100u) && !(m & 0x20u)) return false;    // fourth derivative along x_0 needs the third
    if ((m & 0x200u) && !(m & 0x40u)) return false;
    if ((m & 0x400u) && !(m & 0x100u)) return false;   // fifth needs the fourth
    if ((m & 0x800u) && !(m & 0x200u)) return false;
    return true;
}


int use_device(hrkan_t h) {
    int cur = -1;
    HR_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
    if (cur != h->device) HR_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    return HRKAN_OK;
}

PdeParams make_pde(const pinn_problem* p) {
    PdeParams q{};
    q.kind = p->kind;
    q.a = float(p->a);
    q.b = float(p->b);
    // Poisson source factor (a^2 + b^2) pi^2; in three coordinates (kind 3) c = lam joins it
    const double c2 = p->kind == HRKAN_POISSON3 ? p->lam * p->lam : 0.0;
    q.src = float((p->a * p->a + p->b * p->b + c2) * M_PI * M_PI);
    q.lam = float(p->lam);
    q.nu = float(p->nu);
    q.alpha = float(p->alpha);
    return q;
}

int check_problem(const pinn_problem* p) {
    if (!p) return fail(HRKAN_EINVAL, "problem is NULL");
    if (p->kind != HRKAN_POISSON && p->kind != HRKAN_BURGERS && p->kind != HRKAN_KDV && p->kind != HRKAN_POISSON3)
        return fail(HRKAN_EINVAL, "problem kind %d", p->kind);
    if (!std::isfinite(p->a) || !std::isfinite(p->b) || !std::isfinite(p->lam) || !std::isfinite(p->nu) ||
        !std::isfinite(p->alpha))
        return fail(HRKAN_EINVAL, "non-finite problem coefficient");
    return HRKAN_OK;
}

// The Poisson kind in three coordinates needs a three-input network, every other kind a
// two-input one.
int check_kind_inputs(const pinn_problem* p, int inputs) {
    if ((p->kind == HRKAN_POISSON3) != (inputs == 3))
        return fail(HRKAN_EUNSUPPORTED, "problem kind %d on a network of %d inputs (kind %d takes three inputs, the "
                    "others two)", p->kind, inputs, HRKAN_POISSON3);
    return HRKAN_OK;
}

// Bracket one launch with CUDA events when profiling is on.
struct ProfScope {
    hrkan_t h;
    cudaStream_t s;
    int slot = -1;
    ProfScope(hrkan_t h_, int cls, cudaStream_t s_) : h(h_), s(s_) {
        if (!h->prof) return;
        hrkan_ctx::Ev ev{};
        if (!h->pool.empty()) {
            ev = h->pool.back();
            h->pool.pop_back();
        } else if (cudaEventCreate(&ev.a) != cudaSuccess) {
            return;
        } else if (cudaEventCreate(&ev.b) != cudaSuccess) {
            cudaEventDestroy(ev.a);
            return;
        }
        ev.cls = cls;
        if (cudaEventRecord(ev.a, s) != cudaSuccess) { h->pool.push_back(ev); return; }
        h->pending.push_back(ev);
        slot = int(h->pending.size()) - 1;
    }
    ~ProfScope() {
        if (slot >= 0) cudaEventRecord(h->pending[slot].b, s);
    }
};

NarrowParams base_params(hrkan_t h, const float* W) {
    NarrowParams p{};
    p.W = W;
    p.grid = h->grid;
    p.P = h->P;
    return p;
}

}  // namespace

namespace {

// Validates the offsets and (re)builds the work list of a multi-instance call.
// Host-to-device copies happen only when the offsets, problems or item size
// changed since the previous call, so a repeated call enqueues kernels only.
int build_batch(hrkan_t h, hrkan_ctx::Batch& b, int n_inst, const pinn_problem* probs, const int64_t* off0,
                const int64_t* off1, bool train, cudaStream_t stream) {
    const int ip = h->batch_items_points;
    for (int i = 0; i < n_inst; ++i) {
        if (off0[i + 1] < off0[i]) return fail(HRKAN_EINVAL, "interior offsets decrease at instance %d", i);
        if (train && off1[i + 1] < off1[i]) return fail(HRKAN_EINVAL, "boundary offsets decrease at instance %d", i);
    }
    if (off0[0] != 0 || (train && off1[0] != 0)) return fail(HRKAN_EINVAL, "offsets must start at 0");
    std::vector<double> ab;
    if (probs)
        for (int i = 0; i < n_inst; ++i) {
            ab.push_back(probs[i].a);
            ab.push_back(probs[i].b);
            ab.push_back(probs[i].alpha);
        }
    std::vector<int64_t> o0(off0, off0 + n_inst + 1), o1;
    if (train) o1.assign(off1, off1 + n_inst + 1);
    if (b.n_inst == n_inst && b.items_points == ip && b.off0 == o0 && b.off1 == o1 && b.ab == ab) return HRKAN_OK;

    // earlier launches on this stream may still read the old list
    if (b.n_items > 0) {
        cudaError_t se = cudaStreamSynchronize(stream);
        if (se != cudaSuccess) return cuda_fail(se, "cudaStreamSynchronize before rebuilding the work list");
    }
    // forget the cached key first: if the rebuild fails part-way, no later call may reuse the old list
    b.off0.clear();
    b.off1.clear();
    b.ab.clear();
    b.items_points = 0;
    b.n_items = 0;
    b.n_inst = 0;
    std::vector<BatchItem> items;
    std::vector<BatchInst> inst(n_inst);
    std::vector<int> item_off(n_inst + 1, 0);
    std::vector<float> counts(2 * n_inst, 0.0f);
    for (int i = 0; i < n_inst; ++i) {
        item_off[i] = int(items.size());
        for (int64_t a = off0[i]; a < off0[i + 1]; a += ip) items.push_back({i, 0, a, std::min<int64_t>(a + ip, off0[i + 1])});
        if (train)
            for (int64_t a = off1[i]; a < off1[i + 1]; a += ip)
                items.push_back({i, 1, a, std::min<int64_t>(a + ip, off1[i + 1])});
        const double ni = double(off0[i + 1] - off0[i]), nb = train ? double(off1[i + 1] - off1[i]) : 0.0;
        counts[2 * i] = float(ni);
        counts[2 * i + 1] = float(nb);
        if (probs) {
            const double a = probs[i].a, bb = probs[i].b;
            inst[i] = {float(a), float(bb), float((a * a + bb * bb) * M_PI * M_PI),
                       ni > 0 ? float(2.0 * probs[i].alpha / ni) : 0.0f, nb > 0 ? float(2.0 / nb) : 0.0f};
        }
    }
    item_off[n_inst] = int(items.size());
    const int n_items = int(items.size());
    cudaError_t e;
    if (n_items > b.cap_items || n_inst > b.cap_inst || !b.inst) {
        cudaFree(b.items); cudaFree(b.loss_partial); cudaFree(b.inst); cudaFree(b.item_off); cudaFree(b.counts);
        b.items = nullptr; b.loss_partial = nullptr; b.inst = nullptr; b.item_off = nullptr; b.counts = nullptr;
        const int cap = std::max(n_items, 1);
        if ((e = cudaMalloc(&b.items, sizeof(BatchItem) * cap)) != cudaSuccess ||
            (e = cudaMalloc(&b.loss_partial, sizeof(double) * 2 * cap)) != cudaSuccess ||
            (e = cudaMalloc(&b.inst, sizeof(BatchInst) * std::max(n_inst, 1))) != cudaSuccess ||
            (e = cudaMalloc(&b.item_off, sizeof(int) * (n_inst + 1))) != cudaSuccess ||
            (e = cudaMalloc(&b.counts, sizeof(float) * 2 * std::max(n_inst, 1))) != cudaSuccess) {
            b.cap_items = 0;
            b.cap_inst = 0;
            return fail(HRKAN_ENOMEM, "cudaMalloc of the work list: %s", cudaGetErrorString(e));
        }
        b.cap_items = cap;
        b.cap_inst = std::max(n_inst, 1);
    }
    if (train && size_t(n_items) * size_t(h->P) > b.partial_cap) {
        cudaFree(b.partial);
        b.partial = nullptr;
        b.partial_cap = 0;
        if ((e = cudaMalloc(&b.partial, sizeof(float) * size_t(n_items) * size_t(h->P))) != cudaSuccess)
            return fail(HRKAN_ENOMEM, "cudaMalloc of the gradient partials: %s", cudaGetErrorString(e));
        b.partial_cap = size_t(n_items) * size_t(h->P);
    }
    if (n_items && (e = cudaMemcpy(b.items, items.data(), sizeof(BatchItem) * n_items, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "work list upload");
    if ((e = cudaMemcpy(b.inst, inst.data(), sizeof(BatchInst) * n_inst, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b.item_off, item_off.data(), sizeof(int) * (n_inst + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b.counts, counts.data(), sizeof(float) * 2 * n_inst, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "work list upload");
    b.n_items = n_items;
    b.n_inst = n_inst;
    b.items_points = ip;
    b.off0 = std::move(o0);
    b.off1 = std::move(o1);
    b.ab = std::move(ab);
    return HRKAN_OK;
}

}  // namespace

namespace {

// Scratch slot `slot` with at least `floats` floats (grows; never shrinks).
float* ws_get(hrkan_t h, int slot, size_t floats, int* rc) {
    if (int(h->ws.size()) <= slot) h->ws.resize(slot + 1, {nullptr, 0});
    auto& w = h->ws[slot];
    if (w.second < floats) {
        cudaFree(w.first);
        w.first = nullptr;
        w.second = 0;
        cudaError_t e = cudaMalloc(&w.first, std::max<size_t>(floats, 1) * sizeof(float));
        if (e != cudaSuccess) {
            *rc = fail(HRKAN_ENOMEM, "cudaMalloc of %zu floats of scratch: %s", floats, cudaGetErrorString(e));
            return nullptr;
        }
        w.second = floats;
    }
    return w.first;
}

int jets_of(unsigned mask) { return __builtin_popcount(mask & 0xFFFu); }

// Offset (floats) of layer l's input jets (l >= 1) inside a tape for N points.
int64_t tape_offset(hrkan_t h, int l, int64_t N, int J) {
    int64_t off = 0;
    for (int t = 1; t < l; ++t) off += int64_t(J) * h->cfg.widths[t] * N;
    return off;
}

int64_t tape_total(hrkan_t h, int64_t N, int J) { return tape_offset(h, h->L, N, J); }

WideLayer wide_layer(hrkan_t h, const float* W, int l, int64_t N) {
    WideLayer p{};
    p.W = W + h->layer_off[l];
    p.I = h->cfg.widths[l];
    p.O = h->cfg.widths[l + 1];
    p.N = N;
    p.g = h->grid;
    p.seed0 = h->seed0;
    p.seed1 = h->seed1;
    return p;
}

// One layer's forward: the tensor-core kernel for hidden layers when the
// handle's precision is BF16/TF32 and the shape fits it, else FP32 SIMT.
int forward_layer(hrkan_t h, const float* W, int l, const float* in, float* out, int64_t N, unsigned mask,
                  cudaStream_t s) {
    WideLayer p = wide_layer(h, W, l, N);
    p.z = in;
    p.y = out;
    if (N == 0) return HRKAN_OK;
    if (l > 0 && tc_layer_supported(h->cfg.prec, p.I, p.O, h->n, mask)) {
        int rc = HRKAN_OK;
        const int64_t welems = tc_w_elems(p.O, p.I, h->n, h->cfg.prec);
        float* wp = ws_get(h, 10, size_t(welems), &rc);   // 4-byte slots cover both element sizes
        if (!wp) return rc;
        cudaError_t e;
        {
            ProfScope ps(h, HRKAN_KERNEL_TENSOR, s);
            ProfScope pk(h, HRKAN_KERNEL_TC_FWD, s);
            e = tc_forward_layer(p.W, wp, in, out, p.I, p.O, N, h->grid, h->cfg.prec, mask, h->status, s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core layer launch");
        return HRKAN_OK;
    }
    cudaError_t e;
    {
        ProfScope pk(h, HRKAN_KERNEL_LAYER_FWD, s);
        e = wide_forward_layer(p, mask, l == 0, s);
    }
    if (e == cudaErrorNotSupported) return fail(HRKAN_EUNSUPPORTED, "jet mask 0x%x has no layer kernel", mask);
    if (e != cudaSuccess) return cuda_fail(e, "layer forward launch");
    return HRKAN_OK;
}

// Forward of one point set through every layer.  Layer inputs go to `tape`
// when given (layer l at tape_offset(l)), else to two ping-pong scratch slots
// (zslot, zslot + 1).  The output jets go to `out` [J][N].
int wide_forward_set(hrkan_t h, const float* W, const float* x, int64_t N, unsigned mask, float* out, float* tape,
                     int zslot, cudaStream_t s) {
    if (N == 0) return HRKAN_OK;
    const int J = jets_of(mask), L = h->L;
    int rc = HRKAN_OK;
    const float* in = x;
    for (int l = 0; l < L; ++l) {
        const int O = h->cfg.widths[l + 1];
        float* y;
        if (l == L - 1) y = out;
        else if (tape) y = tape + tape_offset(h, l + 1, N, J);
        else if (!(y = ws_get(h, zslot + (l % 2), size_t(J) * O * N, &rc))) return rc;
        if ((rc = forward_layer(h, W, l, in, y, N, mask, s))) return rc;
        in = y;
    }
    return HRKAN_OK;
}

// Weight gradient of layer l into partial rows [d.row0, d.row0 + d.GP): the
// tensor-core kernel for the BF16 layers it supports (hidden layers and the
// first layer), else FP32 SIMT.
int layer_dw(hrkan_t h, const WideDw& d, int l, unsigned mask, cudaStream_t s) {
    cudaError_t e;
    if (tc_dw_supported(h->cfg.prec, d.I, d.O, h->n, mask)) {
        int rc = HRKAN_OK;
        const int64_t el = tc_dw_gy_elems(jets_of(mask), d.O, d.N);
        float* gbf = ws_get(h, 11, size_t((el + 1) / 2), &rc);   // 2-byte elements in 4-byte slots
        if (!gbf) return rc;
        ProfScope ps(h, HRKAN_KERNEL_TENSOR, s);
        ProfScope pk(h, HRKAN_KERNEL_TC_DW, s);
        e = tc_dw_layer(d.z, d.gy, gbf, d.I, d.O, d.N, d.g, mask, l == 0, d.partial, d.P, d.col0, d.row0, d.GP,
                        h->status, s);
    } else {
        ProfScope ps(h, HRKAN_KERNEL_FUSED, s);
        ProfScope pk(h, HRKAN_KERNEL_LAYER_DW, s);
        e = wide_dw_layer(d, mask, l == 0, s);
    }
    if (e == cudaErrorNotSupported) return fail(HRKAN_EUNSUPPORTED, "jet mask 0x%x has no layer kernel", mask);
    if (e != cudaSuccess) return cuda_fail(e, "weight-gradient launch");
    return HRKAN_OK;
}

// Backward of one point set: weight-gradient partial rows [row0, row0 + GP)
// of h->partial and, for every layer but the first, the input adjoint.  Layer
// inputs come from `tape`, or are recomputed from x when tape is null.
int wide_backward_set(hrkan_t h, const float* W, const float* x, int64_t N, unsigned mask, const float* tape,
                      const float* gy_out, int row0, cudaStream_t s) {
    const int J = jets_of(mask), L = h->L;
    int rc = HRKAN_OK;
    const float* gy = gy_out;
    for (int l = L - 1; l >= 0; --l) {
        const float* zl = x;
        if (l > 0) {
            if (tape) {
                zl = tape + tape_offset(h, l, N, J);
            } else {
                // recompute layer l's input jets from the coordinates
                const float* in = x;
                for (int t = 0; t < l; ++t) {
                    float* y = ws_get(h, 0 + (t % 2), size_t(J) * h->cfg.widths[t + 1] * N, &rc);
                    if (!y) return rc;
                    if ((rc = forward_layer(h, W, t, in, y, N, mask, s))) return rc;
                    in = y;
                }
                zl = in;
            }
        }
        WideDw d{};
        d.z = zl;
        d.gy = gy;
        d.I = h->cfg.widths[l];
        d.O = h->cfg.widths[l + 1];
        d.N = N;
        d.partial = h->partial;
        d.P = h->P;
        d.col0 = h->layer_off[l];
        d.row0 = row0;
        d.GP = h->wide_gp;
        d.g = h->grid;
        d.seed0 = h->seed0;
        d.seed1 = h->seed1;
        if ((rc = layer_dw(h, d, l, mask, s))) return rc;
        cudaError_t e;
        if (l > 0) {
            WideLayer a = wide_layer(h, W, l, N);
            a.z = zl;
            a.gy = gy;
            float* gz = ws_get(h, 2 + (l % 2), size_t(J) * a.I * N, &rc);
            if (!gz) return rc;
            a.gz = gz;
            if (tc_adj_supported(h->cfg.prec, a.I, a.O, h->n, mask) &&
                tc_dw_supported(h->cfg.prec, a.I, a.O, h->n, mask)) {
                // the weight-gradient call above left the BF16 gy copy in slot 11
                float* gbf = ws_get(h, 11, size_t((tc_dw_gy_elems(J, a.O, N) + 1) / 2), &rc);
                float* wbf = gbf ? ws_get(h, 12, size_t((tc_adj_w_elems(a.O, a.I, h->n) + 1) / 2), &rc) : nullptr;
                if (!wbf) return rc;
                ProfScope ps(h, HRKAN_KERNEL_TENSOR, s);
                ProfScope pk(h, HRKAN_KERNEL_TC_ADJ, s);
                e = tc_adj_layer(a.W, wbf, gbf, zl, gz, a.I, a.O, N, h->grid, mask, h->status, s);
            } else {
                ProfScope pk(h, HRKAN_KERNEL_LAYER_ADJ, s);
                e = wide_adjoint_layer(a, mask, s);
            }
            if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
            gy = gz;
        }
    }
    return HRKAN_OK;
}

// Training step of the layer-wise path: forward (interior and boundary),
// residual, backward of both sets into disjoint partial rows, then the same
// fixed-order reduction + Adam as the fused path.
// Ni_tot / Nb_tot: the point counts the loss means divide by (this call's own
// counts, or a data-parallel step's totals over every shard); adam = false
// leaves W and the moments alone (the shard's loss contributions and gradient only).
int wide_train_step(hrkan_t h, const pinn_problem* prob, float* W, const float* x_int, int64_t N_int,
                    const float* x_bnd, const float* g_bnd, int64_t N_bnd, double lr, double b1, double b2,
                    double eps, int t, double* loss, float* dW, cudaStream_t s, int64_t Ni_tot, int64_t Nb_tot,
                    bool adam) {
    const unsigned mask = pde_mask(prob->kind);
    const int J = jets_of(mask);
    int rc = HRKAN_OK;
    float* jets = ws_get(h, 4, size_t(J) * std::max<int64_t>(N_int, 1), &rc);
    float* dli = jets ? ws_get(h, 5, size_t(J) * std::max<int64_t>(N_int, 1), &rc) : nullptr;
    float* ub = dli ? ws_get(h, 6, size_t(std::max<int64_t>(N_bnd, 1)), &rc) : nullptr;
    float* dlb = ub ? ws_get(h, 7, size_t(std::max<int64_t>(N_bnd, 1)), &rc) : nullptr;
    if (!dlb) return rc;
    // keep the interior tape while it fits the budget, else recompute in the backward
    const int64_t tape_i = tape_total(h, N_int, J), tape_b = tape_total(h, N_bnd, 1);
    const size_t budget = h->cfg.hbm_budget_bytes;
    const bool store = budget == 0 || size_t(tape_i + tape_b) * sizeof(float) <= budget;
    float* ti = nullptr;
    float* tb = nullptr;
    if (store) {
        if (tape_i > 0 && !(ti = ws_get(h, 8, size_t(tape_i), &rc))) return rc;
        if (tape_b > 0 && !(tb = ws_get(h, 9, size_t(tape_b), &rc))) return rc;
    }
    {
        ProfScope ps(h, HRKAN_KERNEL_FORWARD, s);
        if ((rc = wide_forward_set(h, W, x_int, N_int, mask, jets, ti, 0, s))) return rc;
        if ((rc = wide_forward_set(h, W, x_bnd, N_bnd, 0x1u, ub, tb, 0, s))) return rc;
    }
    ResidualParams r{};
    r.pde = make_pde(prob);
    r.mask = mask;
    r.x = x_int;
    r.jets = jets;
    r.N = N_int;
    r.dL = dli;
    r.u_bnd = ub;
    r.g_bnd = g_bnd;
    r.Nb = N_bnd;
    r.dLb = dlb;
    r.scale0 = Ni_tot > 0 ? float(2.0 * prob->alpha / double(Ni_tot)) : 0.0f;
    r.scale1 = Nb_tot > 0 ? float(2.0 / double(Nb_tot)) : 0.0f;
    r.loss_partial = h->loss_partial;
    r.t_counter = adam && t == 0 ? h->t_counter : nullptr;
    int64_t rg = (std::max(N_int, N_bnd) + 255) / 256;
    rg = std::min<int64_t>(std::max<int64_t>(rg, 1), h->max_grid_l);
    {
        ProfScope ps(h, HRKAN_KERNEL_RESIDUAL, s);
        HR_CUDA(launch_residual(r, int(rg), s), "residual launch");
    }
    if ((rc = wide_backward_set(h, W, x_int, N_int, mask, ti, dli, 0, s))) return rc;
    if ((rc = wide_backward_set(h, W, x_bnd, N_bnd, 0x1u, tb, dlb, h->wide_gp, s))) return rc;
    ReduceParams q{};
    q.partial = h->partial;
    q.G = 2 * h->wide_gp;
    q.P = h->P;
    q.dW = dW;
    q.do_adam = adam ? 1 : 0;
    q.W = W;
    q.m1 = h->m1;
    q.m2 = h->m2;
    q.lr = lr; q.b1 = b1; q.b2 = b2; q.eps = eps;
    q.c1 = 1.0 - std::pow(b1, t > 0 ? t : 1);
    q.c2 = 1.0 - std::pow(b2, t > 0 ? t : 1);
    q.t_counter = adam && t == 0 ? h->t_counter : nullptr;
    q.loss_partial = h->loss_partial;
    q.Gl = int(rg);
    q.loss = loss;
    q.status = h->status;
    q.alpha = prob->alpha;
    q.n0 = Ni_tot;
    q.n1 = Nb_tot;
    {
        ProfScope ps(h, HRKAN_KERNEL_REDUCE, s);
        HR_CUDA(launch_reduce(q, s), "reduce/Adam launch");
    }
    return HRKAN_OK;
}


// ------------------------------------------------ layer-wise, many instances

// Builds (or reuses) the block-padded layout of a multi-instance call on the
// layer-wise path.  Instance i's interior points [off0[i], off0[i+1]) take
// ceil(n/LB_BLOCK) whole blocks (the last one filled with copies of the
// instance's last point), likewise its boundary points when off1 is given.
// Weight-gradient chunks (at most chunk_blocks blocks of one instance and set)
// and loss rows (one per block) are numbered instance by instance, so that
// instance i's gradient partials are rows [row_off[i], row_off[i+1]) and its
// loss partials rows [loss_off[i], loss_off[i+1]).
int build_lbatch(hrkan_t h, hrkan_ctx::LBatch& b, int n_inst, const pinn_problem* probs, const int64_t* off0,
                 const int64_t* off1, cudaStream_t stream) {
    const bool train = off1 != nullptr;
    for (int i = 0; i < n_inst; ++i) {
        if (off0[i + 1] < off0[i]) return fail(HRKAN_EINVAL, "interior offsets decrease at instance %d", i);
        if (train && off1[i + 1] < off1[i]) return fail(HRKAN_EINVAL, "boundary offsets decrease at instance %d", i);
    }
    if (off0[0] != 0 || (train && off1[0] != 0)) return fail(HRKAN_EINVAL, "offsets must start at 0");
    const int64_t tot0 = off0[n_inst], tot1 = train ? off1[n_inst] : 0;
    const int64_t cb = std::max<int64_t>(1, (int64_t(h->batch_items_points) + LB_BLOCK - 1) / LB_BLOCK);
    // block counts, padded sizes and chunk rows must stay in int range
    if ((tot0 + int64_t(LB_BLOCK) * n_inst) / LB_BLOCK > (int64_t(1) << 30) / LB_BLOCK ||
        (tot1 + int64_t(LB_BLOCK) * n_inst) / LB_BLOCK > (int64_t(1) << 30) / LB_BLOCK)
        return fail(HRKAN_EINVAL, "more than 2^30 padded points in one set");
    std::vector<double> ab;
    if (probs)
        for (int i = 0; i < n_inst; ++i) {
            ab.push_back(probs[i].a);
            ab.push_back(probs[i].b);
            ab.push_back(probs[i].alpha);
        }
    std::vector<int64_t> o0(off0, off0 + n_inst + 1), o1;
    if (train) o1.assign(off1, off1 + n_inst + 1);
    if (b.built && b.n_inst == n_inst && b.chunk_blocks == int(cb) && b.off0 == o0 && b.off1 == o1 && b.ab == ab)
        return HRKAN_OK;
    if (b.built) {   // earlier launches on this stream may still read the old tables
        cudaError_t se = cudaStreamSynchronize(stream);
        if (se != cudaSuccess) return cuda_fail(se, "cudaStreamSynchronize before rebuilding the batch layout");
    }
    b.built = false;

    struct Set {
        std::vector<int> blk_inst, blk_valid, pt_src, lrow;
        std::vector<int4> chunks;
    } set[2];
    std::vector<int> row_off(n_inst + 1, 0), loss_off(n_inst + 1, 0);
    std::vector<BatchInst> inst(n_inst);
    std::vector<float> counts(2 * n_inst, 0.0f);
    int row = 0, lrow = 0;
    for (int i = 0; i < n_inst; ++i) {
        row_off[i] = row;
        loss_off[i] = lrow;
        for (int sidx = 0; sidx < (train ? 2 : 1); ++sidx) {
            const int64_t* off = sidx == 0 ? off0 : off1;
            Set& S = set[sidx];
            const int64_t n = off[i + 1] - off[i];
            const int nb = int((n + LB_BLOCK - 1) / LB_BLOCK);
            const int b0 = int(S.blk_inst.size());
            for (int k = 0; k < nb; ++k) {
                S.blk_inst.push_back(i);
                S.blk_valid.push_back(int(std::min<int64_t>(LB_BLOCK, n - int64_t(k) * LB_BLOCK)));
                S.lrow.push_back(lrow++);
                for (int t = 0; t < LB_BLOCK; ++t)
                    S.pt_src.push_back(int(off[i] + std::min<int64_t>(int64_t(k) * LB_BLOCK + t, n - 1)));
            }
            for (int k = 0; k < nb; k += int(cb)) {
                const int e = std::min(nb, k + int(cb));
                S.chunks.push_back(make_int4((b0 + k) * LB_BLOCK, (b0 + e) * LB_BLOCK, row++, i));
            }
        }
        const double ni = double(off0[i + 1] - off0[i]), nb = train ? double(off1[i + 1] - off1[i]) : 0.0;
        counts[2 * i] = float(ni);
        counts[2 * i + 1] = float(nb);
        if (probs) {
            const double a = probs[i].a, bb = probs[i].b;
            inst[i] = {float(a), float(bb), float((a * a + bb * bb) * M_PI * M_PI),
                       ni > 0 ? float(2.0 * probs[i].alpha / ni) : 0.0f, nb > 0 ? float(2.0 / nb) : 0.0f};
        }
    }
    row_off[n_inst] = row;
    loss_off[n_inst] = lrow;
    // one device allocation holding every table
    std::vector<char> host;
    auto put = [&](const void* src, size_t bytes) {
        const size_t at = (host.size() + 255) & ~size_t(255);
        host.resize(at + std::max<size_t>(bytes, 16));
        if (bytes) std::memcpy(host.data() + at, src, bytes);
        return at;
    };
    const size_t a_bi = put(set[0].blk_inst.data(), set[0].blk_inst.size() * sizeof(int));
    const size_t a_bv = put(set[0].blk_valid.data(), set[0].blk_valid.size() * sizeof(int));
    const size_t a_ps = put(set[0].pt_src.data(), set[0].pt_src.size() * sizeof(int));
    const size_t a_lr = put(set[0].lrow.data(), set[0].lrow.size() * sizeof(int));
    const size_t a_ch = put(set[0].chunks.data(), set[0].chunks.size() * sizeof(int4));
    const size_t b_bi = put(set[1].blk_inst.data(), set[1].blk_inst.size() * sizeof(int));
    const size_t b_bv = put(set[1].blk_valid.data(), set[1].blk_valid.size() * sizeof(int));
    const size_t b_ps = put(set[1].pt_src.data(), set[1].pt_src.size() * sizeof(int));
    const size_t b_lr = put(set[1].lrow.data(), set[1].lrow.size() * sizeof(int));
    const size_t b_ch = put(set[1].chunks.data(), set[1].chunks.size() * sizeof(int4));
    const size_t a_ro = put(row_off.data(), row_off.size() * sizeof(int));
    const size_t a_lo = put(loss_off.data(), loss_off.size() * sizeof(int));
    const size_t a_in = put(inst.data(), inst.size() * sizeof(BatchInst));
    const size_t a_co = put(counts.data(), counts.size() * sizeof(float));
    cudaError_t e;
    if (host.size() > b.mem_bytes) {
        cudaFree(b.mem);
        b.mem = nullptr;
        b.mem_bytes = 0;
        if ((e = cudaMalloc(&b.mem, host.size())) != cudaSuccess)
            return fail(HRKAN_ENOMEM, "cudaMalloc of the batch layout: %s", cudaGetErrorString(e));
        b.mem_bytes = host.size();
    }
    if ((e = cudaMemcpy(b.mem, host.data(), host.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "batch layout upload");
    char* m = static_cast<char*>(b.mem);
    b.blk_inst_i = reinterpret_cast<int*>(m + a_bi);
    b.blk_valid_i = reinterpret_cast<int*>(m + a_bv);
    b.pt_src_i = reinterpret_cast<int*>(m + a_ps);
    b.lrow_i = reinterpret_cast<int*>(m + a_lr);
    b.chunks_i = reinterpret_cast<int4*>(m + a_ch);
    b.blk_inst_b = reinterpret_cast<int*>(m + b_bi);
    b.blk_valid_b = reinterpret_cast<int*>(m + b_bv);
    b.pt_src_b = reinterpret_cast<int*>(m + b_ps);
    b.lrow_b = reinterpret_cast<int*>(m + b_lr);
    b.chunks_b = reinterpret_cast<int4*>(m + b_ch);
    b.row_off = reinterpret_cast<int*>(m + a_ro);
    b.loss_off = reinterpret_cast<int*>(m + a_lo);
    b.inst = reinterpret_cast<BatchInst*>(m + a_in);
    b.counts = reinterpret_cast<float*>(m + a_co);
    b.nbi = int(set[0].blk_inst.size());
    b.nbb = int(set[1].blk_inst.size());
    b.NPi = int64_t(b.nbi) * LB_BLOCK;
    b.NPb = int64_t(b.nbb) * LB_BLOCK;
    b.nci = int(set[0].chunks.size());
    b.ncb = int(set[1].chunks.size());
    b.rows = row;
    b.lrows = lrow;
    if (train) {
        const size_t pf = size_t(std::max(row, 1)) * size_t(h->P);
        if (pf > b.partial_cap) {
            cudaFree(b.partial);
            b.partial = nullptr;
            b.partial_cap = 0;
            if ((e = cudaMalloc(&b.partial, pf * sizeof(float))) != cudaSuccess)
                return fail(HRKAN_ENOMEM, "cudaMalloc of the gradient partials: %s", cudaGetErrorString(e));
            b.partial_cap = pf;
        }
        const size_t lf = size_t(std::max(lrow, 1)) * 2;
        if (lf > b.lp_cap) {
            cudaFree(b.loss_partial);
            b.loss_partial = nullptr;
            b.lp_cap = 0;
            if ((e = cudaMalloc(&b.loss_partial, lf * sizeof(double))) != cudaSuccess)
                return fail(HRKAN_ENOMEM, "cudaMalloc of the loss partials: %s", cudaGetErrorString(e));
            b.lp_cap = lf;
        }
    }
    b.n_inst = n_inst;
    b.chunk_blocks = int(cb);
    b.off0 = std::move(o0);
    b.off1 = std::move(o1);
    b.ab = std::move(ab);
    b.built = true;
    return HRKAN_OK;
}

// One layer's forward over a block-padded multi-instance point set.
int lb_forward_layer(hrkan_t h, const float* W, int l, const float* in, float* out, int64_t N, unsigned mask,
                     const int* blk_inst, cudaStream_t s, int wslot = 20) {
    if (N == 0) return HRKAN_OK;
    WideLayer p = wide_layer(h, W, l, N);
    p.z = in;
    p.y = out;
    p.blk_inst = blk_inst;
    p.w_stride = h->P;
    const int n_inst = h->cfg.n_instances;
    if (l > 0 && !h->batch_fwd_simt && tc_layer_supported(h->cfg.prec, p.I, p.O, h->n, mask)) {
        int rc = HRKAN_OK;
        const int64_t welems = tc_w_elems(p.O, p.I, h->n, h->cfg.prec) * n_inst;
        float* wp = ws_get(h, wslot, size_t(welems), &rc);
        if (!wp) return rc;
        cudaError_t e;
        {
            ProfScope ps(h, HRKAN_KERNEL_TENSOR, s);
            ProfScope pk(h, HRKAN_KERNEL_TC_FWD, s);
            e = tc_forward_layer(p.W, wp, in, out, p.I, p.O, N, h->grid, h->cfg.prec, mask, h->status, s, n_inst,
                                 h->P, blk_inst);
        }
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core layer launch (batched)");
        return HRKAN_OK;
    }
    cudaError_t e;
    {
        ProfScope ps(h, HRKAN_KERNEL_FORWARD, s);
        ProfScope pk(h, HRKAN_KERNEL_LAYER_FWD, s);
        e = wide_forward_layer(p, mask, l == 0, s);
    }
    if (e == cudaErrorNotSupported) return fail(HRKAN_EUNSUPPORTED, "jet mask 0x%x has no layer kernel", mask);
    if (e != cudaSuccess) return cuda_fail(e, "layer forward launch (batched)");
    return HRKAN_OK;
}

// Forward of one padded set through every layer: layer inputs into `tape`
// (layer l at tape_offset(l)) or, without a tape, ping-pong slots zslot and
// zslot + 1; output jets into out [J][N].
// nlayers < L stops before layer nlayers (its input jets are then the last
// ones the tape receives).
int lb_forward_set(hrkan_t h, const float* W, const float* x, int64_t N, unsigned mask, float* out, float* tape,
                   const int* blk_inst, int zslot, cudaStream_t s, int nlayers = -1, int wslot = 20) {
    if (N == 0) return HRKAN_OK;
    const int J = jets_of(mask), L = h->L;
    int rc = HRKAN_OK;
    const float* in = x;
    const int stop = nlayers < 0 ? L : nlayers;
    for (int l = 0; l < stop; ++l) {
        const int O = h->cfg.widths[l + 1];
        float* y;
        if (l == L - 1) y = out;
        else if (tape) y = tape + tape_offset(h, l + 1, N, J);
        else if (!(y = ws_get(h, zslot + (l % 2), size_t(J) * O * N, &rc))) return rc;
        if ((rc = lb_forward_layer(h, W, l, in, y, N, mask, blk_inst, s, wslot))) return rc;
        in = y;
    }
    return HRKAN_OK;
}

// Backward of one padded set (its tape kept by the forward): every layer's
// weight-gradient chunks into their partial rows and, past the first layer,
// the input adjoint.
// l_top: the layer whose output gradient gy_out is (the last one by default;
// L - 2 when the output layer's reverse ran in the fused output-layer kernel).
// gy_bf_in (optional): that gradient already in BF16 ([J * O][N], the
// tensor-core operand layout) instead of gy_out.
// A layer whose weight gradient and input adjoint both run on the tensor
// cores reads its output gradient only in BF16; the layer above then writes
// it so (lb_layer_takes_bf16).
bool lb_layer_takes_bf16(hrkan_t h, int l, unsigned mask) {
    const int I = h->cfg.widths[l], O = h->cfg.widths[l + 1];
    if (!tc_dw_supported(h->cfg.prec, I, O, h->n, mask)) return false;
    return l == 0 || tc_adj_supported(h->cfg.prec, I, O, h->n, mask);
}

int lb_backward_set(hrkan_t h, const float* W, const float* x, int64_t N, unsigned mask, const float* tape,
                    const float* gy_out, const int* blk_inst, const int4* chunks, int nchunk, float* partial,
                    cudaStream_t s, int l_top = -1, void* gy_bf_in = nullptr, int gy_bf_slot = 38, int shift = 0) {
    if (N == 0) return HRKAN_OK;
    const int J = jets_of(mask), L = h->L, n_inst = h->cfg.n_instances;
    int rc = HRKAN_OK;
    const float* gy = gy_out;
    void* gybf = gy_bf_in;          // non-null: this layer's output gradient is ready in BF16
    // BF16 gradients alternate between slots 38 and 39; the first one written
    // must not be the slot gy_bf_in lives in (the adjoint reads it meanwhile)
    int bf_slot = gy_bf_in && gy_bf_slot == 38 ? 39 : 38;
    for (int l = l_top < 0 ? L - 1 : l_top; l >= 0; --l) {
        const float* zl = l > 0 ? tape + tape_offset(h, l, N, J) : x;
        WideDw d{};
        d.z = zl;
        d.gy = gy;
        d.I = h->cfg.widths[l];
        d.O = h->cfg.widths[l + 1];
        d.N = N;
        d.partial = partial;
        d.P = h->P;
        d.col0 = h->layer_off[l];
        d.row0 = 0;
        d.GP = nchunk;
        d.g = h->grid;
        d.chunks = chunks;
        cudaError_t e;
        const bool tc_dw = tc_dw_supported(h->cfg.prec, d.I, d.O, h->n, mask);
        if (!tc_dw && !gy) return fail(HRKAN_EUNSUPPORTED, "layer %d: FP32 weight gradient without an FP32 gradient", l);
        void* gbf = gybf;
        if (tc_dw) {
            if (!gbf) {   // convert the FP32 gradient into slot 21 (+ shift)
                const int64_t el = tc_dw_gy_elems(J, d.O, N);
                if (!(gbf = ws_get(h, 21 + shift, size_t((el + 1) / 2), &rc))) return rc;
            }
            ProfScope ps(h, HRKAN_KERNEL_TENSOR, s);
            ProfScope pk(h, HRKAN_KERNEL_TC_DW, s);
            e = tc_dw_layer(d.z, d.gy, gbf, d.I, d.O, N, d.g, mask, l == 0, partial, h->P, d.col0, 0, nchunk,
                            h->status, s, chunks, gybf != nullptr);
        } else {
            ProfScope ps(h, HRKAN_KERNEL_FUSED, s);
            ProfScope pk(h, HRKAN_KERNEL_LAYER_DW, s);
            e = wide_dw_layer(d, mask, l == 0, s);
        }
        if (e == cudaErrorNotSupported) return fail(HRKAN_EUNSUPPORTED, "jet mask 0x%x has no layer kernel", mask);
        if (e != cudaSuccess) return cuda_fail(e, "weight-gradient launch (batched)");
        if (l > 0) {
            WideLayer a = wide_layer(h, W, l, N);
            a.z = zl;
            a.gy = gy;
            a.blk_inst = blk_inst;
            a.w_stride = h->P;
            const bool tc_adj = tc_dw && tc_adj_supported(h->cfg.prec, a.I, a.O, h->n, mask);
            if (!tc_adj && !gy) return fail(HRKAN_EUNSUPPORTED, "layer %d: FP32 adjoint without an FP32 gradient", l);
            // the layer below takes its gradient in BF16 only: write it so (tensor-core adjoint)
            const bool out_bf = tc_adj && lb_layer_takes_bf16(h, l - 1, mask);
            float* gz = nullptr;
            void* gz_bf = nullptr;
            if (out_bf) {
                const int64_t el = tc_dw_gy_elems(J, a.I, N);
                if (!(gz_bf = ws_get(h, bf_slot, size_t((el + 1) / 2), &rc))) return rc;
                bf_slot = bf_slot == 38 ? 39 : 38;
            } else if (!(gz = ws_get(h, 23 + shift + (l % 2), size_t(J) * a.I * N, &rc))) {
                return rc;
            }
            a.gz = gz;
            if (tc_adj) {
                float* wbf = ws_get(h, 22, size_t((tc_adj_w_elems(a.O, a.I, h->n) * n_inst + 1) / 2), &rc);
                if (!wbf) return rc;
                ProfScope ps(h, HRKAN_KERNEL_TENSOR, s);
                ProfScope pk(h, HRKAN_KERNEL_TC_ADJ, s);
                e = tc_adj_layer(a.W, wbf, gbf, zl, gz, a.I, a.O, N, h->grid, mask, h->status, s, n_inst, h->P, chunks,
                                 nchunk, gz_bf);
            } else {
                ProfScope ps(h, HRKAN_KERNEL_FUSED, s);
                ProfScope pk(h, HRKAN_KERNEL_LAYER_ADJ, s);
                e = wide_adjoint_layer(a, mask, s);
            }
            if (e != cudaSuccess) return cuda_fail(e, "adjoint launch (batched)");
            gy = gz;
            gybf = gz_bf;
        }
    }
    return HRKAN_OK;
}

// The same step for networks of a single layer (no layer below the output
// layer): the output layer's forward, the residual and its reverse as separate
// launches.
int lb_train_step_unfused(hrkan_t h, const pinn_problem* probs, float* W, const float* x_int, const int64_t* off_int,
                  const float* x_bnd, const float* g_bnd, const int64_t* off_bnd, double lr, double b1, double b2,
                  double eps, int t, double* loss, float* dW, cudaStream_t s) {
    const int n_inst = h->cfg.n_instances;
    auto& b = h->lb_train;
    if (int rc = build_lbatch(h, b, n_inst, probs, off_int, off_bnd, s)) return rc;
    const unsigned mask = pde_mask(probs[0].kind);
    if (!residual_mask_supported(mask)) return fail(HRKAN_EUNSUPPORTED, "no residual kernel for mask 0x%x", mask);
    const int J = jets_of(mask);
    const int64_t Ni = b.NPi, Nb = b.NPb;
    int rc = HRKAN_OK;
    float* xi = ws_get(h, 25, size_t(2 * std::max<int64_t>(Ni, 1)), &rc);
    float* xb = xi ? ws_get(h, 26, size_t(2 * std::max<int64_t>(Nb, 1)), &rc) : nullptr;
    float* gb = xb ? ws_get(h, 27, size_t(std::max<int64_t>(Nb, 1)), &rc) : nullptr;
    float* ti = gb ? ws_get(h, 28, size_t(std::max<int64_t>(tape_total(h, Ni, J), 1)), &rc) : nullptr;
    float* tb = ti ? ws_get(h, 29, size_t(std::max<int64_t>(tape_total(h, Nb, 1), 1)), &rc) : nullptr;
    float* jets = tb ? ws_get(h, 30, size_t(J) * std::max<int64_t>(Ni, 1), &rc) : nullptr;
    float* dli = jets ? ws_get(h, 31, size_t(J) * std::max<int64_t>(Ni, 1), &rc) : nullptr;
    float* ub = dli ? ws_get(h, 32, size_t(std::max<int64_t>(Nb, 1)), &rc) : nullptr;
    float* dlb = ub ? ws_get(h, 33, size_t(std::max<int64_t>(Nb, 1)), &rc) : nullptr;
    if (!dlb) return rc;
    const int64_t n0 = off_int[n_inst], n1 = off_bnd[n_inst];
    HR_CUDA(lb_gather(x_int, n0, b.pt_src_i, xi, Ni, 2, s), "point gather");
    HR_CUDA(lb_gather(x_bnd, n1, b.pt_src_b, xb, Nb, 2, s), "point gather");
    HR_CUDA(lb_gather(g_bnd, n1, b.pt_src_b, gb, Nb, 1, s), "point gather");
    if ((rc = lb_forward_set(h, W, xi, Ni, mask, jets, ti, b.blk_inst_i, 0, s))) return rc;
    if ((rc = lb_forward_set(h, W, xb, Nb, 0x1u, ub, tb, b.blk_inst_b, 0, s))) return rc;
    LbResidualParams r{};
    r.pde = make_pde(&probs[0]);
    r.mask = mask;
    r.inst = b.inst;
    r.x = xi;
    r.jets = jets;
    r.Ni = Ni;
    r.dL = dli;
    r.u_bnd = ub;
    r.g_bnd = gb;
    r.Nb = Nb;
    r.dLb = dlb;
    r.nbi = b.nbi;
    r.nbb = b.nbb;
    r.blk_inst_int = b.blk_inst_i;
    r.blk_valid_int = b.blk_valid_i;
    r.blk_inst_bnd = b.blk_inst_b;
    r.blk_valid_bnd = b.blk_valid_b;
    r.lrow_int = b.lrow_i;
    r.lrow_bnd = b.lrow_b;
    r.loss_partial = b.loss_partial;
    r.t_counter = t == 0 ? h->t_counter : nullptr;
    {
        ProfScope ps(h, HRKAN_KERNEL_RESIDUAL, s);
        HR_CUDA(lb_residual(r, s), "residual launch (batched)");
    }
    if ((rc = lb_backward_set(h, W, xi, Ni, mask, ti, dli, b.blk_inst_i, b.chunks_i, b.nci, b.partial, s))) return rc;
    if ((rc = lb_backward_set(h, W, xb, Nb, 0x1u, tb, dlb, b.blk_inst_b, b.chunks_b, b.ncb, b.partial, s))) return rc;
    BatchReduceParams q{};
    q.partial = b.partial;
    q.item_off = b.row_off;
    q.loss_off = b.loss_off;
    q.n_inst = n_inst;
    q.P = h->P;
    q.W = W;
    q.m1 = h->m1;
    q.m2 = h->m2;
    q.lr = lr; q.b1 = b1; q.b2 = b2; q.eps = eps;
    q.c1 = 1.0 - std::pow(b1, t > 0 ? t : 1);
    q.c2 = 1.0 - std::pow(b2, t > 0 ? t : 1);
    q.t_counter = t == 0 ? h->t_counter : nullptr;
    q.loss_partial = b.loss_partial;
    q.counts = b.counts;
    q.loss = loss;
    q.status = h->status;
    q.dW = dW;
    q.alpha = probs[0].alpha;
    {
        ProfScope ps(h, HRKAN_KERNEL_REDUCE, s);
        HR_CUDA(launch_batch_reduce(q, s), "multi-instance reduce launch (batched)");
    }
    return HRKAN_OK;
}

// Multi-instance training step on the layer-wise path: gather both point sets
// into the block-padded layout, forward of the layers below the output layer
// with the tape kept, the output layer with the residual/loss per instance and
// its reverse in one launch per set, backward of the layers below into
// per-chunk partial rows, then the per-instance fixed-order reduction and Adam.
// The boundary set's chain of kernels runs on the handle's side stream,
// forked from the caller's stream at the start of the step and joined back
// before the per-instance reduction, so that its small launches overlap the
// interior set's; the two chains share no buffer they write (own tape, gradient and
// scratch slots, distinct partial and loss rows).  The join also runs on an
// early error return, keeping the caller's stream ordered after the side
// stream's work (and a stream capture closed).  With kernel timing on
// (hrkan_profile_enable) both sets run in order on the caller's stream, so
// that each launch's events time that launch alone.
struct SideJoin {
    hrkan_t h;
    cudaStream_t s;
    bool active = false;
    void join() {
        if (!active) return;
        active = false;
        cudaEventRecord(h->join_ev, h->side);
        cudaStreamWaitEvent(s, h->join_ev, 0);
    }
    ~SideJoin() { join(); }
};

int side_stream(hrkan_t h) {
    if (h->side) return HRKAN_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "side stream");
    return HRKAN_OK;
}

int lb_train_step(hrkan_t h, const pinn_problem* probs, float* W, const float* x_int, const int64_t* off_int,
                  const float* x_bnd, const float* g_bnd, const int64_t* off_bnd, double lr, double b1, double b2,
                  double eps, int t, double* loss, float* dW, cudaStream_t s) {
    const int n_inst = h->cfg.n_instances;
    auto& b = h->lb_train;
    if (int rc = build_lbatch(h, b, n_inst, probs, off_int, off_bnd, s)) return rc;
    const unsigned mask = pde_mask(probs[0].kind);
    if (!residual_mask_supported(mask)) return fail(HRKAN_EUNSUPPORTED, "no residual kernel for mask 0x%x", mask);
    const int J = jets_of(mask);
    const int64_t Ni = b.NPi, Nb = b.NPb;
    const int L = h->L;
    if (L < 2) return lb_train_step_unfused(h, probs, W, x_int, off_int, x_bnd, g_bnd, off_bnd, lr, b1, b2, eps, t,
                                            loss, dW, s);
    int rc = HRKAN_OK;
    float* xi = ws_get(h, 25, size_t(2 * std::max<int64_t>(Ni, 1)), &rc);
    float* xb = xi ? ws_get(h, 26, size_t(2 * std::max<int64_t>(Nb, 1)), &rc) : nullptr;
    float* gb = xb ? ws_get(h, 27, size_t(std::max<int64_t>(Nb, 1)), &rc) : nullptr;
    float* ti = gb ? ws_get(h, 28, size_t(std::max<int64_t>(tape_total(h, Ni, J), 1)), &rc) : nullptr;
    float* tb = ti ? ws_get(h, 29, size_t(std::max<int64_t>(tape_total(h, Nb, 1), 1)), &rc) : nullptr;
    if (!tb) return rc;
    const int I_out = h->cfg.widths[L - 1];
    // the output layer's input adjoint (the gradient the layers below start
    // from): BF16 for the interior set when the layer below reads it only so
    const bool gzi_bf = lb_layer_takes_bf16(h, L - 2, mask);
    float* gzi = nullptr;
    void* gzi_b = nullptr;
    if (gzi_bf) {
        gzi_b = ws_get(h, 38, size_t((tc_dw_gy_elems(J, I_out, std::max<int64_t>(Ni, 1)) + 1) / 2), &rc);
        if (!gzi_b) return rc;
    } else if (!(gzi = ws_get(h, 23 + ((L - 1) % 2), size_t(J) * I_out * std::max<int64_t>(Ni, 1), &rc))) {
        return rc;
    }
    float* gzb = ws_get(h, 30, size_t(I_out) * std::max<int64_t>(Nb, 1), &rc);
    if (!gzb) return rc;
    const int64_t n0 = off_int[n_inst], n1 = off_bnd[n_inst];
    // the boundary set on the side stream when both sets have points
    cudaStream_t sb = s;
    SideJoin sj{h, s};
    if (Ni > 0 && Nb > 0 && !h->prof) {
        if ((rc = side_stream(h))) return rc;
        HR_CUDA(cudaEventRecord(h->fork_ev, s), "fork event");
        HR_CUDA(cudaStreamWaitEvent(h->side, h->fork_ev, 0), "fork wait");
        sb = h->side;
        sj.active = true;
    }
    HR_CUDA(lb_gather(x_int, n0, b.pt_src_i, xi, Ni, 2, s), "point gather");
    HR_CUDA(lb_gather(x_bnd, n1, b.pt_src_b, xb, Nb, 2, sb), "point gather");
    HR_CUDA(lb_gather(g_bnd, n1, b.pt_src_b, gb, Nb, 1, sb), "point gather");
    // layers below the output layer; their outputs (the output layer's inputs) go to the tape
    if ((rc = lb_forward_set(h, W, xi, Ni, mask, nullptr, ti, b.blk_inst_i, 0, s, L - 1))) return rc;
    if ((rc = lb_forward_set(h, W, xb, Nb, 0x1u, nullptr, tb, b.blk_inst_b, 0, sb, L - 1, 40))) return rc;
    // the output layer, residual / boundary misfit, its reverse: one launch per set
    LbTailParams tp{};
    tp.W = W + h->layer_off[L - 1];
    tp.w_stride = h->P;
    tp.I = I_out;
    tp.g = h->grid;
    tp.pde = make_pde(&probs[0]);
    tp.inst = b.inst;
    tp.partial = b.partial;
    tp.P = h->P;
    tp.col0 = h->layer_off[L - 1];
    tp.loss_partial = b.loss_partial;
    {
        LbTailParams ti_p = tp;
        ti_p.z = ti + tape_offset(h, L - 1, Ni, J);
        ti_p.gz = gzi;
        ti_p.gz_bf = static_cast<uint16_t*>(gzi_b);
        ti_p.N = Ni;
        ti_p.x = xi;
        ti_p.blk_valid = b.blk_valid_i;
        ti_p.lrow = b.lrow_i;
        ti_p.chunks = b.chunks_i;
        ti_p.t_counter = t == 0 && b.nci > 0 ? h->t_counter : nullptr;
        {
            ProfScope ps(h, HRKAN_KERNEL_RESIDUAL, s);
            HR_CUDA(lb_tail(ti_p, mask, false, b.nci, s), "output-layer launch (batched)");
        }
        LbTailParams tb_p = tp;
        tb_p.z = tb + tape_offset(h, L - 1, Nb, 1);
        tb_p.gz = gzb;
        tb_p.N = Nb;
        tb_p.g_bnd = gb;
        tb_p.blk_valid = b.blk_valid_b;
        tb_p.lrow = b.lrow_b;
        tb_p.chunks = b.chunks_b;
        tb_p.t_counter = t == 0 && b.nci == 0 ? h->t_counter : nullptr;
        {
            ProfScope ps(h, HRKAN_KERNEL_RESIDUAL, sb);
            HR_CUDA(lb_tail(tb_p, mask, true, b.ncb, sb), "output-layer launch (batched)");
        }
    }
    if (L >= 2) {
        if ((rc = lb_backward_set(h, W, xi, Ni, mask, ti, gzi, b.blk_inst_i, b.chunks_i, b.nci, b.partial, s, L - 2,
                                  gzi_b, 38)))
            return rc;
        if ((rc = lb_backward_set(h, W, xb, Nb, 0x1u, tb, gzb, b.blk_inst_b, b.chunks_b, b.ncb, b.partial, sb, L - 2,
                                  nullptr, 38, 20)))
            return rc;
    }
    sj.join();
    BatchReduceParams q{};
    q.partial = b.partial;
    q.item_off = b.row_off;
    q.loss_off = b.loss_off;
    q.n_inst = n_inst;
    q.P = h->P;
    q.W = W;
    q.m1 = h->m1;
    q.m2 = h->m2;
    q.lr = lr; q.b1 = b1; q.b2 = b2; q.eps = eps;
    q.c1 = 1.0 - std::pow(b1, t > 0 ? t : 1);
    q.c2 = 1.0 - std::pow(b2, t > 0 ? t : 1);
    q.t_counter = t == 0 ? h->t_counter : nullptr;
    q.loss_partial = b.loss_partial;
    q.counts = b.counts;
    q.loss = loss;
    q.status = h->status;
    q.dW = dW;
    q.alpha = probs[0].alpha;
    {
        ProfScope ps(h, HRKAN_KERNEL_REDUCE, s);
        HR_CUDA(launch_batch_reduce(q, s), "multi-instance reduce launch (batched)");
    }
    return HRKAN_OK;
}

// Output jets of every instance on the layer-wise path: gather, forward, scatter.
int lb_forward_batched(hrkan_t h, const float* W, const float* x, const int64_t* offsets, unsigned mask, float* jets,
                       cudaStream_t s) {
    const int n_inst = h->cfg.n_instances;
    auto& b = h->lb_fwd;
    if (int rc = build_lbatch(h, b, n_inst, nullptr, offsets, nullptr, s)) return rc;
    const int J = jets_of(mask);
    const int64_t Np = b.NPi, N = offsets[n_inst];
    if (N == 0) return HRKAN_OK;
    int rc = HRKAN_OK;
    float* xp = ws_get(h, 34, size_t(2 * Np), &rc);
    float* out = xp ? ws_get(h, 35, size_t(J) * Np, &rc) : nullptr;
    if (!out) return rc;
    HR_CUDA(lb_gather(x, N, b.pt_src_i, xp, Np, 2, s), "point gather");
    if ((rc = lb_forward_set(h, W, xp, Np, mask, out, nullptr, b.blk_inst_i, 36, s))) return rc;
    HR_CUDA(lb_scatter(out, Np, b.pt_src_i, b.blk_valid_i, jets, N, J, s), "jet scatter");
    return HRKAN_OK;
}

}  // namespace

namespace hrkan {
// Records the message hrkan_last_error() returns (for entry points in other files).
int set_last_error(int code, const char* msg) {
    g_err = msg;
    return code;
}
}  // namespace hrkan

// Three-input networks (D = 3).  The jet mask has bit 0 = u, bit 1+d =
// du/dx_d, bit 4+d = d2u/dx_d^2 (d = 0, 1, 2).  A jet row along direction d
// depends only on derivatives along d, so the network runs as two passes of
// the two-direction kernels: directions (x, y) with the first layer's seeds
// (0, 1), then direction z with seeds (2, none); the rows are then gathered in
// the mask's bit order.
bool valid_mask3(unsigned m) {
    if (!(m & 1u) || (m & ~0x7Fu)) return false;
    return !((m & 0x10u) && !(m & 0x02u)) && !((m & 0x20u) && !(m & 0x04u)) && !((m & 0x40u) && !(m & 0x08u));
}

// The layer kernels' two-direction mask that covers m2 (0x01, 0x0F or 0x1F;
// a pass computes its extra rows and leaves them unused).
unsigned covering_mask(unsigned m2) { return m2 == 1u ? 1u : (m2 & ~0x0Fu) ? 0x1Fu : 0x0Fu; }

// Pass masks (two-direction encoding) of a three-input mask; mb = 0: no z pass.
void split3(unsigned m, unsigned* ma, unsigned* mb) {
    *ma = covering_mask(1u | (m & 0x02u) | (m & 0x04u) | ((m & 0x10u) ? 0x08u : 0u) | ((m & 0x20u) ? 0x10u : 0u));
    *mb = (m & 0x48u) ? covering_mask(1u | ((m & 0x08u) ? 0x02u : 0u) | ((m & 0x40u) ? 0x08u : 0u)) : 0u;
}

// For bit b of a three-input mask: which pass holds it (0 = xy, 1 = z) and its bit there.
void bit3_source(int b, int* pass, int* bit2) {
    static const int P[7] = {0, 0, 0, 1, 0, 0, 1}, B[7] = {0, 1, 2, 1, 3, 4, 3};
    *pass = P[b];
    *bit2 = B[b];
}

int row_of_bit(unsigned mask, int bit) { return __builtin_popcount(mask & ((1u << bit) - 1u)); }

int forward3(hrkan_t h, const float* W, const float* x, int64_t N, unsigned m, float* jets, cudaStream_t s) {
    unsigned ma, mb;
    split3(m, &ma, &mb);
    int rc = HRKAN_OK;
    float* y[2] = {ws_get(h, 16, size_t(jets_of(ma)) * N, &rc), nullptr};
    if (!y[0]) return rc;
    if (mb && !(y[1] = ws_get(h, 17, size_t(jets_of(mb)) * N, &rc))) return rc;
    h->seed0 = 0;
    h->seed1 = 1;
    rc = wide_forward_set(h, W, x, N, ma, y[0], nullptr, 0, s);
    if (!rc && mb) {
        h->seed0 = 2;
        h->seed1 = -1;
        rc = wide_forward_set(h, W, x, N, mb, y[1], nullptr, 0, s);
    }
    h->seed0 = 0;
    h->seed1 = 1;
    if (rc) return rc;
    int r = 0;
    for (int b = 0; b < 7; ++b) {
        if (!(m & (1u << b))) continue;
        int pass, b2;
        bit3_source(b, &pass, &b2);
        const float* src = y[pass] + size_t(row_of_bit(pass ? mb : ma, b2)) * N;
        HR_CUDA(cudaMemcpyAsync(jets + size_t(r) * N, src, size_t(N) * sizeof(float), cudaMemcpyDeviceToDevice, s),
                "cudaMemcpyAsync");
        ++r;
    }
    return HRKAN_OK;
}

// Weight-gradient partial rows of both passes: [row0, row0 + GP) and, with a z pass,
// [row0 + GP, row0 + 2 GP).
int backward3(hrkan_t h, const float* W, const float* x, int64_t N, unsigned m, const float* dL, int* rows,
              cudaStream_t s, int row0 = 0) {
    unsigned ma, mb;
    split3(m, &ma, &mb);
    int rc = HRKAN_OK;
    float* g[2] = {ws_get(h, 18, size_t(jets_of(ma)) * N, &rc), nullptr};
    if (!g[0]) return rc;
    if (mb && !(g[1] = ws_get(h, 19, size_t(jets_of(mb)) * N, &rc))) return rc;
    int r = 0;
    // rows the mask does not request (and the z pass's u row) get zero gradient
    HR_CUDA(cudaMemsetAsync(g[0], 0, size_t(jets_of(ma)) * N * sizeof(float), s), "cudaMemsetAsync");
    if (mb) HR_CUDA(cudaMemsetAsync(g[1], 0, size_t(jets_of(mb)) * N * sizeof(float), s), "cudaMemsetAsync");
    for (int b = 0; b < 7; ++b) {
        if (!(m & (1u << b))) continue;
        int pass, b2;
        bit3_source(b, &pass, &b2);
        float* dst = g[pass] + size_t(row_of_bit(pass ? mb : ma, b2)) * N;
        HR_CUDA(cudaMemcpyAsync(dst, dL + size_t(r) * N, size_t(N) * sizeof(float), cudaMemcpyDeviceToDevice, s),
                "cudaMemcpyAsync");
        ++r;
    }
    h->seed0 = 0;
    h->seed1 = 1;
    rc = wide_backward_set(h, W, x, N, ma, nullptr, g[0], row0, s);
    if (!rc && mb) {
        h->seed0 = 2;
        h->seed1 = -1;
        rc = wide_backward_set(h, W, x, N, mb, nullptr, g[1], row0 + h->wide_gp, s);
    }
    h->seed0 = 0;
    h->seed1 = 1;
    *rows = mb ? 2 * h->wide_gp : h->wide_gp;
    return rc;
}

extern "C" {

int64_t hrkan_param_count(const hrkan_cfg* cfg) {
    if (check_cfg(cfg) == HRKAN_EINVAL) return 0;
    return count_params(cfg);
}

const char* hrkan_last_error(void) { return g_err.c_str(); }

int hrkan_init(hrkan_t* out, const hrkan_cfg* cfg) {
    if (!out) return fail(HRKAN_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_cfg(cfg);
    if (rc) return rc;
    const int L = cfg->n_widths - 1;
    int net_id = -1;
    bool uniform_hidden = true;
    for (int l = 1; l < L; ++l) uniform_hidden &= (cfg->widths[l] == cfg->widths[1]);
    if (uniform_hidden) net_id = narrow_net_id(L, cfg->widths[1]);
    if (cfg->flags & HRKAN_FLAG_LAYERWISE) net_id = -1;
    if (cfg->m != 4) net_id = -1;   // the fused narrow kernels are built for m = 4
    if (cfg->widths[0] == 3) {
        net_id = -1;                  // three inputs: layer-wise path, FP32, one network
        if (cfg->prec != HRKAN_FP32 || cfg->n_instances != 1)
            return fail(HRKAN_EUNSUPPORTED, "three-input networks run in FP32 with one instance");
    }
    if (cfg->prec != HRKAN_FP32 && cfg->m != 4)
        return fail(HRKAN_EUNSUPPORTED, "precision %d: the tensor-core kernels are built for m = 4 (m=%d)", cfg->prec,
                    cfg->m);
    // several instances: the fused multi-instance kernels, or the layer-wise multi-instance path
    if (cfg->prec != HRKAN_FP32 && net_id >= 0)
        return fail(HRKAN_EUNSUPPORTED, "precision %d: the fused narrow kernels are FP32 only (set HRKAN_FLAG_LAYERWISE)",
                    cfg->prec);

    hrkan_ctx* h = new (std::nothrow) hrkan_ctx();
    if (!h) return fail(HRKAN_ENOMEM, "host allocation");
    h->cfg = *cfg;
    h->L = L;
    h->n = cfg->G + cfg->k;
    h->P = count_params(cfg);
    h->net_id = net_id;
    const double hh = (cfg->grid_hi - cfg->grid_lo) / cfg->G;
    h->grid.lo = float(cfg->grid_lo);
    h->grid.h = float(hh);
    h->grid.inv_h = float(1.0 / hh);
    h->grid.inv_a = float(2.0 / ((cfg->k + 1) * hh));
    h->grid.m = cfg->m;
    h->grid.n = h->n;

    cudaError_t e;
    if ((e = cudaGetDevice(&h->device)) != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
    if ((e = cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    h->layer_off.assign(L + 1, 0);
    for (int l = 0; l < L; ++l)
        h->layer_off[l + 1] = h->layer_off[l] + int64_t(cfg->widths[l]) * cfg->widths[l + 1] * h->n;
    h->wide_gp = std::max(1, h->nsm * 2 / 8);
    // layer-wise: two point sets of wide_gp partial rows each; three inputs: two passes
    // for the interior set and one for the boundary set
    h->max_grid = net_id >= 0 ? h->nsm * 8 : (cfg->widths[0] == 3 ? 3 : 2) * h->wide_gp;
    h->max_grid_l = h->nsm * 8;
    size_t bytes_partial = size_t(h->max_grid) * size_t(h->P) * sizeof(float);
    if ((e = cudaMalloc(&h->partial, bytes_partial)) != cudaSuccess ||
        (e = cudaMalloc(&h->loss_partial, size_t(h->max_grid_l) * 2 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&h->m1, size_t(h->P) * cfg->n_instances * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&h->m2, size_t(h->P) * cfg->n_instances * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&h->t_counter, 2 * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&h->status, 4 * sizeof(int))) != cudaSuccess) {
        hrkan_destroy(h);
        return fail(HRKAN_ENOMEM, "cudaMalloc of the workspace: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMemset(h->m1, 0, size_t(h->P) * cfg->n_instances * sizeof(double))) != cudaSuccess ||
        (e = cudaMemset(h->m2, 0, size_t(h->P) * cfg->n_instances * sizeof(double))) != cudaSuccess ||
        (e = cudaMemset(h->t_counter, 0, 2 * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(h->status, 0, 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        hrkan_destroy(h);
        return cuda_fail(e, "zeroing the Adam moments");
    }
    *out = h;
    return HRKAN_OK;
}

void hrkan_destroy(hrkan_t h) {
    if (!h) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != h->device) cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    if (h->side) cudaStreamDestroy(h->side);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    cudaFree(h->partial);
    cudaFree(h->loss_partial);
    cudaFree(h->m1);
    cudaFree(h->m2);
    cudaFree(h->t_counter);
    cudaFree(h->status);
    for (auto* b : {&h->lb_train, &h->lb_fwd}) {
        cudaFree(b->mem);
        cudaFree(b->partial);
        cudaFree(b->loss_partial);
    }
    for (auto* b : {&h->train_batch, &h->fwd_batch}) {
        cudaFree(b->items); cudaFree(b->inst); cudaFree(b->item_off); cudaFree(b->counts);
        cudaFree(b->partial); cudaFree(b->loss_partial);
    }
    for (auto& w : h->ws) cudaFree(w.first);
    for (auto& ev : h->pending) { cudaEventDestroy(ev.a); cudaEventDestroy(ev.b); }
    for (auto& ev : h->pool) { cudaEventDestroy(ev.a); cudaEventDestroy(ev.b); }
    if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
    delete h;
}

int64_t hrkan_tape_floats(hrkan_t h, int64_t N, unsigned jet_mask) {
    if (!h || N <= 0 || !valid_mask(jet_mask) || h->net_id >= 0 || h->cfg.widths[0] == 3) return 0;   // recompute
    return tape_total(h, N, jets_of(jet_mask));
}

int hrkan_forward_jets(hrkan_t h, const float* W, const float* x, int64_t N, unsigned jet_mask, float* jets,
                       float* tape, hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (N < 0) return fail(HRKAN_EINVAL, "N=%lld", (long long)N);
    const bool d3 = h->cfg.widths[0] == 3;
    if (!(d3 ? valid_mask3(jet_mask) : valid_mask(jet_mask))) return fail(HRKAN_EINVAL, "jet mask 0x%x", jet_mask);
    if (N == 0) return HRKAN_OK;
    if (!W || !x || !jets) return fail(HRKAN_EINVAL, "NULL device pointer");
    if (int rc = use_device(h)) return rc;
    if (d3) {
        ProfScope ps(h, HRKAN_KERNEL_FORWARD, (cudaStream_t)stream);
        return forward3(h, W, x, N, jet_mask, jets, (cudaStream_t)stream);
    }
    if (h->net_id < 0) {
        ProfScope ps(h, HRKAN_KERNEL_FORWARD, (cudaStream_t)stream);
        return wide_forward_set(h, W, x, N, jet_mask, jets, tape, 0, (cudaStream_t)stream);
    }
    NarrowParams p = base_params(h, W);
    p.x0 = x;
    p.n0 = N;
    p.jets = jets;
    int grid = 0;
    cudaError_t e;
    {
        ProfScope ps(h, HRKAN_KERNEL_FORWARD, (cudaStream_t)stream);
        e = narrow_launch(h->net_id, MODE_FWD, jet_mask, p, &grid, 1 << 30, true, (cudaStream_t)stream);
    }
    if (e == cudaErrorNotSupported) return fail(HRKAN_EUNSUPPORTED, "jet mask 0x%x has no forward kernel", jet_mask);
    if (e != cudaSuccess) return cuda_fail(e, "forward launch");
    return HRKAN_OK;
}

int pinn_residual_loss(hrkan_t h, const pinn_problem* prob, const float* x_int, int64_t N_int, unsigned jet_mask,
                       const float* jets_int, const float* u_bnd, const float* g_bnd, int64_t N_bnd, double* loss,
                       float* dL_djets_int, float* dL_du_bnd, hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (int rc = check_problem(prob)) return rc;
    if (int rc = check_kind_inputs(prob, h->cfg.widths[0])) return rc;
    const bool d3 = h->cfg.widths[0] == 3;
    if (N_int < 0 || N_bnd < 0) return fail(HRKAN_EINVAL, "negative point count");
    if (!(d3 ? valid_mask3(jet_mask) : valid_mask(jet_mask))) return fail(HRKAN_EINVAL, "jet mask 0x%x", jet_mask);
    if (!mask_has_rows(jet_mask, prob->kind))
        return fail(HRKAN_EINVAL, "jet mask 0x%x lacks rows the residual needs", jet_mask);
    if (d3 ? jet_mask != pde_mask(HRKAN_POISSON3) : !residual_mask_supported(jet_mask))
        return fail(HRKAN_EUNSUPPORTED, "jet mask 0x%x", jet_mask);
    if (!loss) return fail(HRKAN_EINVAL, "loss is NULL");
    if (N_int > 0 && (!x_int || !jets_int)) return fail(HRKAN_EINVAL, "NULL interior pointer");
    if (N_bnd > 0 && (!u_bnd || !g_bnd)) return fail(HRKAN_EINVAL, "NULL boundary pointer");
    if (int rc = use_device(h)) return rc;
    ResidualParams r{};
    r.pde = make_pde(prob);
    r.mask = jet_mask;
    r.x = x_int;
    r.jets = jets_int;
    r.N = N_int;
    r.dL = dL_djets_int;
    r.u_bnd = u_bnd;
    r.g_bnd = g_bnd;
    r.Nb = N_bnd;
    r.dLb = dL_du_bnd;
    r.scale0 = N_int > 0 ? float(2.0 * prob->alpha / double(N_int)) : 0.0f;
    r.scale1 = N_bnd > 0 ? float(2.0 / double(N_bnd)) : 0.0f;
    r.loss_partial = h->loss_partial;
    int64_t most = N_int > N_bnd ? N_int : N_bnd;
    int64_t grid = (most + 255) / 256;
    if (grid > h->max_grid_l) grid = h->max_grid_l;
    if (grid < 1) grid = 1;
    cudaStream_t s = (cudaStream_t)stream;
    {
        ProfScope ps(h, HRKAN_KERNEL_RESIDUAL, s);
        HR_CUDA(d3 ? launch_residual3(r, (int)grid, s) : launch_residual(r, (int)grid, s), "residual launch");
    }
    ReduceParams q{};
    q.P = 0;
    q.loss_partial = h->loss_partial;
    q.Gl = (int)grid;
    q.loss = loss;
    q.status = h->status;
    q.alpha = prob->alpha;
    q.n0 = N_int;
    q.n1 = N_bnd;
    {
        ProfScope ps(h, HRKAN_KERNEL_REDUCE, s);
        HR_CUDA(launch_reduce(q, s), "loss reduce launch");
    }
    return HRKAN_OK;
}

int hrkan_backward(hrkan_t h, const float* W, const float* x, int64_t N, unsigned jet_mask, const float* tape,
                   const float* dL_djets, float* dW, int accumulate, hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (N < 0) return fail(HRKAN_EINVAL, "N=%lld", (long long)N);
    const bool d3 = h->cfg.widths[0] == 3;
    if (!(d3 ? valid_mask3(jet_mask) : valid_mask(jet_mask))) return fail(HRKAN_EINVAL, "jet mask 0x%x", jet_mask);
    if (!W || !dW) return fail(HRKAN_EINVAL, "NULL device pointer");
    if (N > 0 && (!x || !dL_djets)) return fail(HRKAN_EINVAL, "NULL device pointer");
    if (int rc = use_device(h)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (N == 0) {
        if (!accumulate) HR_CUDA(cudaMemsetAsync(dW, 0, size_t(h->P) * sizeof(float), s), "cudaMemsetAsync");
        return HRKAN_OK;
    }
    int grid = 0;
    cudaError_t e = cudaSuccess;
    if (d3) {
        if (int rc = backward3(h, W, x, N, jet_mask, dL_djets, &grid, s)) return rc;
    } else if (h->net_id < 0) {
        if (int rc = wide_backward_set(h, W, x, N, jet_mask, tape, dL_djets, 0, s)) return rc;
        grid = h->wide_gp;
    } else {
        NarrowParams p = base_params(h, W);
        p.x0 = x;
        p.n0 = N;
        p.dL = dL_djets;
        p.partial = h->partial;
        ProfScope ps(h, HRKAN_KERNEL_FUSED, s);
        e = narrow_launch(h->net_id, MODE_BWD, jet_mask, p, &grid, h->max_grid, true, s);
    }
    if (e == cudaErrorNotSupported) return fail(HRKAN_EUNSUPPORTED, "jet mask 0x%x has no backward kernel", jet_mask);
    if (e != cudaSuccess) return cuda_fail(e, "backward launch");
    ReduceParams q{};
    q.partial = h->partial;
    q.G = grid;
    q.P = h->P;
    q.dW = dW;
    q.accumulate = accumulate ? 1 : 0;
    {
        ProfScope ps(h, HRKAN_KERNEL_REDUCE, s);
        HR_CUDA(launch_reduce(q, s), "gradient reduce launch");
    }
    return HRKAN_OK;
}

int adam_step(hrkan_t h, float* W, const float* dW, double lr, double b1, double b2, double eps, int t,
              hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (!W || !dW) return fail(HRKAN_EINVAL, "NULL device pointer");
    if (t < 1) return fail(HRKAN_EINVAL, "Adam step t=%d must be >= 1", t);
    if (!(b1 >= 0.0 && b1 < 1.0 && b2 >= 0.0 && b2 < 1.0 && eps >= 0.0 && std::isfinite(lr)))
        return fail(HRKAN_EINVAL, "Adam hyper-parameters lr=%g b1=%g b2=%g eps=%g", lr, b1, b2, eps);
    if (int rc = use_device(h)) return rc;
    ReduceParams q{};
    q.partial = dW;
    q.G = 1;
    q.P = h->P;
    q.do_adam = 1;
    q.W = W;
    q.m1 = h->m1;
    q.m2 = h->m2;
    q.lr = lr; q.b1 = b1; q.b2 = b2; q.eps = eps;
    q.c1 = 1.0 - std::pow(b1, t);
    q.c2 = 1.0 - std::pow(b2, t);
    {
        ProfScope ps(h, HRKAN_KERNEL_REDUCE, (cudaStream_t)stream);
        HR_CUDA(launch_reduce(q, (cudaStream_t)stream), "Adam launch");
    }
    return HRKAN_OK;
}

int hrkan_reset_moments(hrkan_t h, hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (int rc = use_device(h)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t mb = size_t(h->P) * h->cfg.n_instances * sizeof(double);
    HR_CUDA(cudaMemsetAsync(h->m1, 0, mb, s), "cudaMemsetAsync");
    HR_CUDA(cudaMemsetAsync(h->m2, 0, mb, s), "cudaMemsetAsync");
    HR_CUDA(cudaMemsetAsync(h->t_counter, 0, 2 * sizeof(int), s), "cudaMemsetAsync");
    return HRKAN_OK;
}

int hrkan_save(hrkan_t h, const float* W, int64_t t, const char* path, hrkan_stream_t stream) {
    if (!h || !W || !path) return fail(HRKAN_EINVAL, "hrkan_save: null argument");
    if (int rc = use_device(h)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = size_t(h->P) * h->cfg.n_instances;
    std::vector<float> w;
    std::vector<double> m, v;
    try {
        w.resize(n);
        m.resize(n);
        v.resize(n);
    } catch (...) {
        return fail(HRKAN_ENOMEM, "hrkan_save: host buffers");
    }
    int tc[2] = {0, 0};
    HR_CUDA(cudaMemcpyAsync(w.data(), W, n * sizeof(float), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    HR_CUDA(cudaMemcpyAsync(m.data(), h->m1, n * sizeof(double), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    HR_CUDA(cudaMemcpyAsync(v.data(), h->m2, n * sizeof(double), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    HR_CUDA(cudaMemcpyAsync(tc, h->t_counter, sizeof tc, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    HR_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return hrkan_checkpoint_write(path, h->P, h->cfg.n_instances, t, int64_t(tc[0]), w.data(), m.data(), v.data());
}

int hrkan_load(hrkan_t h, float* W, int64_t* t, const char* path, hrkan_stream_t stream) {
    if (!h || !W || !path) return fail(HRKAN_EINVAL, "hrkan_load: null argument");
    if (int rc = use_device(h)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = size_t(h->P) * h->cfg.n_instances;
    std::vector<float> w;
    std::vector<double> m, v;
    try {
        w.resize(n);
        m.resize(n);
        v.resize(n);
    } catch (...) {
        return fail(HRKAN_ENOMEM, "hrkan_load: host buffers");
    }
    int64_t ts = 0, td = 0;
    if (int rc = hrkan_checkpoint_read(path, h->P, h->cfg.n_instances, &ts, &td, w.data(), m.data(), v.data()))
        return rc;
    if (td < 0 || td > INT32_MAX) return fail(HRKAN_EINVAL, "hrkan_load: device step count %lld", (long long)td);
    const int tc[2] = {int(td), int(td)};
    HR_CUDA(cudaMemcpyAsync(W, w.data(), n * sizeof(float), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
    HR_CUDA(cudaMemcpyAsync(h->m1, m.data(), n * sizeof(double), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
    HR_CUDA(cudaMemcpyAsync(h->m2, v.data(), n * sizeof(double), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
    HR_CUDA(cudaMemcpyAsync(h->t_counter, tc, sizeof tc, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
    HR_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");   // the host buffers die here
    if (t) *t = ts;
    return HRKAN_OK;
}

int hrkan_profile_enable(hrkan_t h, int enable) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    h->prof = enable != 0;
    return HRKAN_OK;
}

int hrkan_profile_read(hrkan_t h, int kernel_class, double* total_ms, int64_t* launches, int reset) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (kernel_class < 0 || kernel_class >= HRKAN_KERNEL_CLASSES)
        return fail(HRKAN_EINVAL, "kernel class %d", kernel_class);
    if (int rc = use_device(h)) return rc;
    size_t done = 0;
    cudaError_t e = cudaSuccess;
    for (; done < h->pending.size(); ++done) {
        const auto& ev = h->pending[done];
        float ms = 0.0f;
        if ((e = cudaEventSynchronize(ev.b)) != cudaSuccess || (e = cudaEventElapsedTime(&ms, ev.a, ev.b)) != cudaSuccess)
            break;
        h->prof_ms[ev.cls] += ms;
        h->prof_n[ev.cls] += 1;
        h->pool.push_back(ev);
    }
    // events already counted leave the pending list even when a later one fails
    h->pending.erase(h->pending.begin(), h->pending.begin() + done);
    if (e != cudaSuccess) return cuda_fail(e, "kernel timing events");
    if (total_ms) *total_ms = h->prof_ms[kernel_class];
    if (launches) *launches = h->prof_n[kernel_class];
    if (reset) {
        h->prof_ms[kernel_class] = 0.0;
        h->prof_n[kernel_class] = 0;
    }
    return HRKAN_OK;
}

namespace {
// The training step of hrkan_train_step (adam = true) and of
// hrkan_train_step_partial (adam = false: the loss contributions and the
// gradient of this shard, means over Ni_tot / Nb_tot points).
// One training step of a three-input network (the Poisson kind in three
// coordinates): the jets by the two-pass forward (directions x, y, then z),
// the residual and the boundary misfit, the two-pass backward of the interior
// set (partial rows [0, 2 GP)) and the backward of the boundary set (rows
// [2 GP, 3 GP)), then the reduction with Adam.  No tape: the backward
// recomputes the layer inputs.
int train_step3(hrkan_t h, const pinn_problem* prob, float* W, const float* x_int, int64_t N_int, const float* x_bnd,
                const float* g_bnd, int64_t N_bnd, double lr, double b1, double b2, double eps, int t, double* loss,
                float* dW, cudaStream_t s, int64_t Ni_tot, int64_t Nb_tot, bool adam) {
    const unsigned mask = pde_mask(HRKAN_POISSON3);
    const int J = __builtin_popcount(mask);
    int rc = HRKAN_OK;
    float* jets = ws_get(h, 4, size_t(J) * std::max<int64_t>(N_int, 1), &rc);
    float* dli = jets ? ws_get(h, 5, size_t(J) * std::max<int64_t>(N_int, 1), &rc) : nullptr;
    float* ub = dli ? ws_get(h, 6, size_t(std::max<int64_t>(N_bnd, 1)), &rc) : nullptr;
    float* dlb = ub ? ws_get(h, 7, size_t(std::max<int64_t>(N_bnd, 1)), &rc) : nullptr;
    if (!dlb) return rc;
    {
        ProfScope ps(h, HRKAN_KERNEL_FORWARD, s);
        if (N_int > 0 && (rc = forward3(h, W, x_int, N_int, mask, jets, s))) return rc;
        if (N_bnd > 0 && (rc = forward3(h, W, x_bnd, N_bnd, 0x1u, ub, s))) return rc;
    }
    ResidualParams r{};
    r.pde = make_pde(prob);
    r.mask = mask;
    r.x = x_int;
    r.jets = jets;
    r.N = N_int;
    r.dL = dli;
    r.u_bnd = ub;
    r.g_bnd = g_bnd;
    r.Nb = N_bnd;
    r.dLb = dlb;
    r.scale0 = Ni_tot > 0 ? float(2.0 * prob->alpha / double(Ni_tot)) : 0.0f;
    r.scale1 = Nb_tot > 0 ? float(2.0 / double(Nb_tot)) : 0.0f;
    r.loss_partial = h->loss_partial;
    r.t_counter = adam && t == 0 ? h->t_counter : nullptr;
    int64_t rg = (std::max(N_int, N_bnd) + 255) / 256;
    rg = std::min<int64_t>(std::max<int64_t>(rg, 1), h->max_grid_l);
    {
        ProfScope ps(h, HRKAN_KERNEL_RESIDUAL, s);
        HR_CUDA(launch_residual3(r, int(rg), s), "residual launch (three inputs)");
    }
    int rows_i = 0, rows_b = 0;
    if (N_int > 0 && (rc = backward3(h, W, x_int, N_int, mask, dli, &rows_i, s, 0))) return rc;
    if (N_bnd > 0 && (rc = backward3(h, W, x_bnd, N_bnd, 0x1u, dlb, &rows_b, s, rows_i))) return rc;
    ReduceParams q{};
    q.partial = h->partial;
    q.G = rows_i + rows_b;
    q.P = h->P;
    q.dW = dW;
    q.do_adam = adam ? 1 : 0;
    q.W = W;
    q.m1 = h->m1;
    q.m2 = h->m2;
    q.lr = lr; q.b1 = b1; q.b2 = b2; q.eps = eps;
    q.c1 = 1.0 - std::pow(b1, t > 0 ? t : 1);
    q.c2 = 1.0 - std::pow(b2, t > 0 ? t : 1);
    q.t_counter = adam && t == 0 ? h->t_counter : nullptr;
    q.loss_partial = h->loss_partial;
    q.Gl = int(rg);
    q.loss = loss;
    q.status = h->status;
    q.alpha = prob->alpha;
    q.n0 = Ni_tot;
    q.n1 = Nb_tot;
    {
        ProfScope ps(h, HRKAN_KERNEL_REDUCE, s);
        HR_CUDA(launch_reduce(q, s), "reduce/Adam launch (three inputs)");
    }
    return HRKAN_OK;
}

int train_step_impl(hrkan_t h, const pinn_problem* prob, float* W, const float* x_int, int64_t N_int,
                    const float* x_bnd, const float* g_bnd, int64_t N_bnd, int64_t Ni_tot, int64_t Nb_tot, bool adam,
                    double lr, double b1, double b2, double eps, int t, double* loss, float* dW,
                    hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (int rc = check_problem(prob)) return rc;
    if (int rc = check_kind_inputs(prob, h->cfg.widths[0])) return rc;
    if (N_int < 0 || N_bnd < 0) return fail(HRKAN_EINVAL, "negative point count");
    if (N_int + N_bnd == 0) return fail(HRKAN_EINVAL, "no collocation points");
    if (!W || !loss) return fail(HRKAN_EINVAL, "NULL device pointer");
    if (N_int > 0 && !x_int) return fail(HRKAN_EINVAL, "x_int is NULL");
    if (N_bnd > 0 && (!x_bnd || !g_bnd)) return fail(HRKAN_EINVAL, "boundary pointer is NULL");
    if (t < 0) return fail(HRKAN_EINVAL, "Adam step t=%d must be >= 0", t);
    if (!(b1 >= 0.0 && b1 < 1.0 && b2 >= 0.0 && b2 < 1.0 && eps >= 0.0 && std::isfinite(lr)))
        return fail(HRKAN_EINVAL, "Adam hyper-parameters lr=%g b1=%g b2=%g eps=%g", lr, b1, b2, eps);
    if (int rc = use_device(h)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned mask = pde_mask(prob->kind);
    if (h->cfg.widths[0] == 3)
        return train_step3(h, prob, W, x_int, N_int, x_bnd, g_bnd, N_bnd, lr, b1, b2, eps, t, loss, dW, s, Ni_tot,
                           Nb_tot, adam);
    if (h->net_id < 0) return wide_train_step(h, prob, W, x_int, N_int, x_bnd, g_bnd, N_bnd, lr, b1, b2, eps, t, loss,
                                              dW, s, Ni_tot, Nb_tot, adam);
    NarrowParams p = base_params(h, W);
    p.x0 = x_int;
    p.n0 = N_int;
    p.x1 = x_bnd;
    p.g1 = g_bnd;
    p.n1 = N_bnd;
    p.partial = h->partial;
    p.loss_partial = h->loss_partial;
    p.pde = make_pde(prob);
    p.scale0 = Ni_tot > 0 ? float(2.0 * prob->alpha / double(Ni_tot)) : 0.0f;
    p.scale1 = Nb_tot > 0 ? float(2.0 / double(Nb_tot)) : 0.0f;
    if (adam && t == 0) p.t_counter = h->t_counter;
    int grid = 0;
    cudaError_t e;
    {
        ProfScope ps(h, HRKAN_KERNEL_FUSED, s);
        e = narrow_launch(h->net_id, MODE_TRAIN, mask, p, &grid, h->max_grid, true, s);
    }
    if (e == cudaErrorNotSupported) return fail(HRKAN_EUNSUPPORTED, "no fused training kernel");
    if (e != cudaSuccess) return cuda_fail(e, "train launch");
    ReduceParams q{};
    q.partial = h->partial;
    q.G = grid;
    q.P = h->P;
    q.dW = dW;
    q.do_adam = adam ? 1 : 0;
    q.W = W;
    q.m1 = h->m1;
    q.m2 = h->m2;
    q.lr = lr; q.b1 = b1; q.b2 = b2; q.eps = eps;
    q.c1 = 1.0 - std::pow(b1, t > 0 ? t : 1);
    q.c2 = 1.0 - std::pow(b2, t > 0 ? t : 1);
    q.loss_partial = h->loss_partial;
    q.Gl = grid;
    q.loss = loss;
    q.status = h->status;
    q.alpha = prob->alpha;
    q.n0 = Ni_tot;
    q.n1 = Nb_tot;
    if (adam && t == 0) q.t_counter = h->t_counter;
    {
        ProfScope ps(h, HRKAN_KERNEL_REDUCE, s);
        HR_CUDA(launch_reduce(q, s), "reduce/Adam launch");
    }
    return HRKAN_OK;
}
}  // namespace

int hrkan_train_step(hrkan_t h, const pinn_problem* prob, float* W, const float* x_int, int64_t N_int,
                     const float* x_bnd, const float* g_bnd, int64_t N_bnd, double lr, double b1, double b2,
                     double eps, int t, double* loss, float* dW, hrkan_stream_t stream) {
    return train_step_impl(h, prob, W, x_int, N_int, x_bnd, g_bnd, N_bnd, N_int, N_bnd, true, lr, b1, b2, eps, t,
                           loss, dW, stream);
}

int hrkan_train_step_partial(hrkan_t h, const pinn_problem* prob, const float* W, const float* x_int, int64_t N_int,
                             const float* x_bnd, const float* g_bnd, int64_t N_bnd, int64_t N_int_total,
                             int64_t N_bnd_total, double* loss, float* dW, hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (N_int_total < N_int || N_bnd_total < N_bnd || N_int < 0 || N_bnd < 0)
        return fail(HRKAN_EINVAL, "totals %lld / %lld below this shard's %lld / %lld points", (long long)N_int_total,
                    (long long)N_bnd_total, (long long)N_int, (long long)N_bnd);
    if (N_int_total + N_bnd_total == 0) return fail(HRKAN_EINVAL, "no collocation points");
    if (!dW) return fail(HRKAN_EINVAL, "dW is NULL");
    if (N_int + N_bnd == 0) {   // an empty shard contributes nothing
        if (!loss) return fail(HRKAN_EINVAL, "NULL device pointer");
        if (int rc = check_problem(prob)) return rc;
        if (int rc = use_device(h)) return rc;
        cudaStream_t s = (cudaStream_t)stream;
        HR_CUDA(cudaMemsetAsync(dW, 0, size_t(h->P) * sizeof(float), s), "cudaMemsetAsync");
        HR_CUDA(cudaMemsetAsync(loss, 0, 3 * sizeof(double), s), "cudaMemsetAsync");
        return HRKAN_OK;
    }
    // W is read only (adam = false); the step's arguments for Adam are placeholders
    return train_step_impl(h, prob, const_cast<float*>(W), x_int, N_int, x_bnd, g_bnd, N_bnd, N_int_total,
                           N_bnd_total, false, 0.0, 0.9, 0.999, 1e-8, 1, loss, dW, stream);
}

int hrkan_set_batch_path(hrkan_t h, int path) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (path < 0 || path > 2)
        return fail(HRKAN_EINVAL, "path %d (0 fused, 1 layer-wise, 2 layer-wise with the FP32 forward)", path);
    if (path == 0 && h->net_id < 0) return fail(HRKAN_EUNSUPPORTED, "this shape has no fused multi-instance kernel");
    h->batch_layerwise = path >= 1 && h->net_id >= 0;
    h->batch_fwd_simt = path == 2;
    return HRKAN_OK;
}

int hrkan_batch_path(hrkan_t h) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (h->batch_fwd_simt) return 2;
    return (h->net_id < 0 || h->batch_layerwise) ? 1 : 0;
}

int hrkan_set_batch_items(hrkan_t h, int points_per_item) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (points_per_item < 1) return fail(HRKAN_EINVAL, "points_per_item=%d", points_per_item);
    h->batch_items_points = points_per_item;
    return HRKAN_OK;
}

int hrkan_train_step_batched(hrkan_t h, const pinn_problem* probs, float* W, const float* x_int,
                             const int64_t* off_int, const float* x_bnd, const float* g_bnd, const int64_t* off_bnd,
                             double lr, double b1, double b2, double eps, int t, double* loss, float* dW,
                             hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (h->cfg.widths[0] == 3) return fail(HRKAN_EUNSUPPORTED, "three-input networks: no multi-instance calls");
    const int n_inst = h->cfg.n_instances;
    if (!probs || !off_int || !off_bnd) return fail(HRKAN_EINVAL, "NULL host array");
    for (int i = 0; i < n_inst; ++i) {
        if (int rc = check_problem(&probs[i])) return rc;
        if (int rc = check_kind_inputs(&probs[i], h->cfg.widths[0])) return rc;
        if (probs[i].kind != probs[0].kind || probs[i].lam != probs[0].lam || probs[i].nu != probs[0].nu ||
            probs[i].alpha != probs[0].alpha)
            return fail(HRKAN_EINVAL, "instance %d: kind, lam, nu and alpha must agree across instances", i);
    }
    if (!W || !loss) return fail(HRKAN_EINVAL, "NULL device pointer");
    if (t < 0) return fail(HRKAN_EINVAL, "Adam step t=%d must be >= 0", t);
    if (!(b1 >= 0.0 && b1 < 1.0 && b2 >= 0.0 && b2 < 1.0 && eps >= 0.0 && std::isfinite(lr)))
        return fail(HRKAN_EINVAL, "Adam hyper-parameters lr=%g b1=%g b2=%g eps=%g", lr, b1, b2, eps);
    const int64_t n0 = off_int[n_inst], n1 = off_bnd[n_inst];
    if ((n0 > 0 && !x_int) || (n1 > 0 && (!x_bnd || !g_bnd))) return fail(HRKAN_EINVAL, "NULL point array");
    if (int rc = use_device(h)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->net_id < 0 || h->batch_layerwise)   // layer-wise multi-instance path
        return lb_train_step(h, probs, W, x_int, off_int, x_bnd, g_bnd, off_bnd, lr, b1, b2, eps, t, loss, dW, s);
    auto& b = h->train_batch;
    if (int rc = build_batch(h, b, n_inst, probs, off_int, off_bnd, true, s)) return rc;
    const unsigned mask = pde_mask(probs[0].kind);
    BatchParams p{};
    p.W = W;
    p.P = h->P;
    p.x0 = x_int;
    p.n0 = n0;
    p.x1 = x_bnd;
    p.g1 = g_bnd;
    p.n1 = n1;
    p.items = b.items;
    p.n_items = b.n_items;
    p.inst = b.inst;
    p.pde = make_pde(&probs[0]);
    p.partial = b.partial;
    p.loss_partial = b.loss_partial;
    p.grid = h->grid;
    p.t_counter = t == 0 ? h->t_counter : nullptr;
    if (b.n_items > 0) {
        int grid = 0;
        cudaError_t e;
        {
            ProfScope ps(h, HRKAN_KERNEL_FUSED, s);
            e = narrow_batch_launch(h->net_id, MODE_TRAIN, mask, p, &grid, 1 << 30, true, s);
        }
        if (e == cudaErrorNotSupported) return fail(HRKAN_EUNSUPPORTED, "no multi-instance training kernel");
        if (e != cudaSuccess) return cuda_fail(e, "multi-instance train launch");
    }
    BatchReduceParams q{};
    q.partial = b.partial;
    q.item_off = b.item_off;
    q.n_inst = n_inst;
    q.P = h->P;
    q.W = W;
    q.m1 = h->m1;
    q.m2 = h->m2;
    q.lr = lr; q.b1 = b1; q.b2 = b2; q.eps = eps;
    q.c1 = 1.0 - std::pow(b1, t > 0 ? t : 1);
    q.c2 = 1.0 - std::pow(b2, t > 0 ? t : 1);
    q.t_counter = t == 0 ? h->t_counter : nullptr;
    q.loss_partial = b.loss_partial;
    q.counts = b.counts;
    q.loss = loss;
    q.status = h->status;
    q.dW = dW;
    q.alpha = probs[0].alpha;
    {
        ProfScope ps(h, HRKAN_KERNEL_REDUCE, s);
        HR_CUDA(launch_batch_reduce(q, s), "multi-instance reduce launch");
    }
    return HRKAN_OK;
}

int hrkan_autotune_batch(hrkan_t h, const pinn_problem* probs, float* W, const float* x_int, const int64_t* off_int,
                         const float* x_bnd, const float* g_bnd, const int64_t* off_bnd, const int* candidates,
                         int n_candidates, int reps, int* chosen, double* ms_per_step, hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (h->cfg.widths[0] == 3) return fail(HRKAN_EUNSUPPORTED, "three-input networks: no multi-instance calls");
    static const int kDefault[] = {256, 512, 1024, 2048, 4096};
    if (!candidates) {
        candidates = kDefault;
        n_candidates = 5;
    }
    if (n_candidates < 1) return fail(HRKAN_EINVAL, "n_candidates=%d", n_candidates);
    for (int c = 0; c < n_candidates; ++c)
        if (candidates[c] < 1) return fail(HRKAN_EINVAL, "candidate %d: %d points per item", c, candidates[c]);
    if (reps < 1) reps = 3;
    if (int rc = use_device(h)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = HRKAN_OK;
    float* loss_f = ws_get(h, 13, size_t(2 * 3 * std::max(h->cfg.n_instances, 1)), &rc);
    if (!loss_f) return rc;
    double* loss = reinterpret_cast<double*>(loss_f);
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    const int saved = h->batch_items_points;
    const int saved_path = hrkan_batch_path(h);
    int best = saved, best_path = saved_path;
    bool found = false;
    float best_ms = 0.0f;
    // the paths timed: a fused shape both kernel families, the fused
    // multi-instance kernel (candidate = points per work item) and the
    // layer-wise path (candidate = points per weight-gradient chunk); a
    // tensor-core precision also the layer-wise path with every forward on the
    // FP32 SIMT kernels (path 2: narrow layers can be faster there).  A family
    // that lacks the problem's kernels (EUNSUPPORTED) is skipped
    int paths[3], n_paths = 0;
    if (h->net_id >= 0) paths[n_paths++] = 0;
    paths[n_paths++] = 1;
    if (h->cfg.prec != HRKAN_FP32) paths[n_paths++] = 2;
    for (int pi = 0; pi < n_paths && rc == HRKAN_OK; ++pi) {
        h->batch_layerwise = h->net_id >= 0 && paths[pi] >= 1;
        h->batch_fwd_simt = paths[pi] == 2;
        for (int c = 0; c < n_candidates && rc == HRKAN_OK; ++c) {
            h->batch_items_points = candidates[c];
            // lr = 0 leaves W as it is; the first call builds this candidate's work list
            auto step = [&]() {
                return hrkan_train_step_batched(h, probs, W, x_int, off_int, x_bnd, g_bnd, off_bnd, 0.0, 0.9, 0.999,
                                                1e-8, 1, loss, nullptr, stream);
            };
            if ((rc = step())) {
                if (rc == HRKAN_EUNSUPPORTED && n_paths > 1) rc = HRKAN_OK;   // try the other families
                break;
            }
            cudaEventRecord(a, s);
            for (int r = 0; r < reps && rc == HRKAN_OK; ++r) rc = step();
            cudaEventRecord(b, s);
            if (rc) break;
            cudaError_t e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "autotune timing");
                break;
            }
            ms /= float(reps);
            if (!found || ms < best_ms) {
                found = true;
                best_ms = ms;
                best = candidates[c];
                best_path = paths[pi];
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc == HRKAN_OK && !found) rc = fail(HRKAN_EUNSUPPORTED, "no multi-instance kernels for this problem");
    h->batch_items_points = rc == HRKAN_OK ? best : saved;
    const int keep = rc == HRKAN_OK ? best_path : saved_path;
    h->batch_layerwise = keep >= 1 && h->net_id >= 0;
    h->batch_fwd_simt = keep == 2;
    if (rc) return rc;
    if ((rc = hrkan_reset_moments(h, stream))) return rc;
    if (chosen) *chosen = best;
    if (ms_per_step) *ms_per_step = double(best_ms);
    return HRKAN_OK;
}

int hrkan_forward_jets_batched(hrkan_t h, const float* W, const float* x, const int64_t* offsets, unsigned jet_mask,
                               float* jets, hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (h->cfg.widths[0] == 3) return fail(HRKAN_EUNSUPPORTED, "three-input networks: no multi-instance calls");
    if (!offsets) return fail(HRKAN_EINVAL, "offsets is NULL");
    if (!valid_mask(jet_mask)) return fail(HRKAN_EINVAL, "jet mask 0x%x", jet_mask);
    const int n_inst = h->cfg.n_instances;
    const int64_t N = offsets[n_inst];
    if (N > 0 && (!W || !x || !jets)) return fail(HRKAN_EINVAL, "NULL device pointer");
    if (int rc = use_device(h)) return rc;
    if (h->net_id < 0) {   // layer-wise multi-instance path
        if (h->cfg.widths[0] != 2) return fail(HRKAN_EUNSUPPORTED, "multi-instance calls take two inputs");
        int rc = HRKAN_OK;
        {
            ProfScope ps(h, HRKAN_KERNEL_FORWARD, (cudaStream_t)stream);
            rc = lb_forward_batched(h, W, x, offsets, jet_mask, jets, (cudaStream_t)stream);
        }
        return rc;
    }
    auto& b = h->fwd_batch;
    if (int rc = build_batch(h, b, n_inst, nullptr, offsets, nullptr, false, (cudaStream_t)stream)) return rc;
    if (b.n_items == 0) return HRKAN_OK;
    BatchParams p{};
    p.W = W;
    p.P = h->P;
    p.x0 = x;
    p.n0 = N;
    p.jets = jets;
    p.items = b.items;
    p.n_items = b.n_items;
    p.grid = h->grid;
    int grid = 0;
    cudaError_t e;
    {
        ProfScope ps(h, HRKAN_KERNEL_FORWARD, (cudaStream_t)stream);
        e = narrow_batch_launch(h->net_id, MODE_FWD, jet_mask, p, &grid, 1 << 30, true, (cudaStream_t)stream);
    }
    if (e == cudaErrorNotSupported) return fail(HRKAN_EUNSUPPORTED, "jet mask 0x%x has no forward kernel", jet_mask);
    if (e != cudaSuccess) return cuda_fail(e, "multi-instance forward launch");
    return HRKAN_OK;
}

int hrkan_sync_status(hrkan_t h) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (int rc = use_device(h)) return rc;
    HR_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    int st = 0;
    HR_CUDA(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
    if (st != 0) {
        HR_CUDA(cudaMemset(h->status, 0, sizeof(int)), "status reset");
        return fail(st, st == HRKAN_ENONFINITE ? "a loss became NaN or infinite (status %d)"
                                               : "a device-side wait gave up (status %d)", st);
    }
    return HRKAN_OK;
}

int hrkan_set_wait_cycles(hrkan_t h, int64_t cycles) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (cycles < 0) return fail(HRKAN_EINVAL, "cycles=%lld", (long long)cycles);
    if (int rc = use_device(h)) return rc;
    const long long w = cycles;
    HR_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    HR_CUDA(cudaMemcpy(h->status + 2, &w, sizeof w, cudaMemcpyHostToDevice), "wait limit write");
    return HRKAN_OK;
}

int hrkan_layer_jets(hrkan_t h, int layer, const float* W, const float* z, int64_t N, unsigned jet_mask, float* y,
                     hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (h->cfg.widths[0] == 3) return fail(HRKAN_EUNSUPPORTED, "three-input networks: no single-layer calls");
    if (layer < 0 || layer >= h->L) return fail(HRKAN_EINVAL, "layer %d outside [0, %d)", layer, h->L);
    if (N < 0) return fail(HRKAN_EINVAL, "N=%lld", (long long)N);
    if (!valid_mask(jet_mask)) return fail(HRKAN_EINVAL, "jet mask 0x%x", jet_mask);
    if (N == 0) return HRKAN_OK;
    if (!W || !z || !y) return fail(HRKAN_EINVAL, "NULL device pointer");
    if (int rc = use_device(h)) return rc;
    // forward_layer takes the whole network's weights and offsets into them
    return forward_layer(h, W - h->layer_off[layer], layer, z, y, N, jet_mask, (cudaStream_t)stream);
}

int hrkan_layer_dw(hrkan_t h, int layer, const float* z, const float* gy, int64_t N, unsigned jet_mask, float* dW,
                   hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (h->cfg.widths[0] == 3) return fail(HRKAN_EUNSUPPORTED, "three-input networks: no single-layer calls");
    if (layer < 0 || layer >= h->L) return fail(HRKAN_EINVAL, "layer %d outside [0, %d)", layer, h->L);
    if (N < 0) return fail(HRKAN_EINVAL, "N=%lld", (long long)N);
    if (!valid_mask(jet_mask)) return fail(HRKAN_EINVAL, "jet mask 0x%x", jet_mask);
    if (!z || !gy || !dW) return fail(HRKAN_EINVAL, "NULL device pointer");
    if (int rc = use_device(h)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int I = h->cfg.widths[layer], O = h->cfg.widths[layer + 1];
    const int64_t cols = int64_t(O) * I * h->n;
    if (N == 0) {
        cudaError_t e = cudaMemsetAsync(dW, 0, sizeof(float) * size_t(cols), s);
        return e == cudaSuccess ? HRKAN_OK : cuda_fail(e, "memset");
    }
    WideDw d{};
    d.z = z;
    d.gy = gy;
    d.I = I;
    d.O = O;
    d.N = N;
    d.partial = h->partial;
    d.P = h->P;
    d.col0 = h->layer_off[layer];
    d.row0 = 0;
    d.GP = h->wide_gp;
    d.g = h->grid;
    if (int rc = layer_dw(h, d, layer, jet_mask, s)) return rc;
    cudaError_t e = sum_rows(h->partial + d.col0, h->wide_gp, h->P, cols, dW, s);
    return e == cudaSuccess ? HRKAN_OK : cuda_fail(e, "row sum launch");
}

int hrkan_layer_adjoint(hrkan_t h, int layer, const float* W, const float* z, const float* gy, int64_t N,
                        unsigned jet_mask, float* gz, hrkan_stream_t stream) {
    if (!h) return fail(HRKAN_EINVAL, "handle is NULL");
    if (h->cfg.widths[0] == 3) return fail(HRKAN_EUNSUPPORTED, "three-input networks: no single-layer calls");
    if (layer < 1 || layer >= h->L) return fail(HRKAN_EINVAL, "layer %d outside [1, %d)", layer, h->L);
    if (N < 0) return fail(HRKAN_EINVAL, "N=%lld", (long long)N);
    if (!valid_mask(jet_mask)) return fail(HRKAN_EINVAL, "jet mask 0x%x", jet_mask);
    if (N == 0) return HRKAN_OK;
    if (!W || !z || !gy || !gz) return fail(HRKAN_EINVAL, "NULL device pointer");
    if (int rc = use_device(h)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    WideLayer a = wide_layer(h, W - h->layer_off[layer], layer, N);
    a.z = z;
    a.gy = gy;
    a.gz = gz;
    const int J = jets_of(jet_mask);
    cudaError_t e;
    if (tc_adj_supported(h->cfg.prec, a.I, a.O, h->n, jet_mask)) {
        int rc = HRKAN_OK;
        float* gbf = ws_get(h, 11, size_t((tc_dw_gy_elems(J, a.O, N) + 1) / 2), &rc);
        float* wbf = gbf ? ws_get(h, 12, size_t((tc_adj_w_elems(a.O, a.I, h->n) + 1) / 2), &rc) : nullptr;
        if (!wbf) return rc;
        ProfScope ps(h, HRKAN_KERNEL_TENSOR, s);
        e = tc_gy_to_bf16(gy, gbf, J, a.O, N, s);
        if (e == cudaSuccess) e = tc_adj_layer(a.W, wbf, gbf, z, gz, a.I, a.O, N, h->grid, jet_mask, h->status, s);
    } else {
        e = wide_adjoint_layer(a, jet_mask, s);
    }
    if (e == cudaErrorNotSupported) return fail(HRKAN_EUNSUPPORTED, "jet mask 0x%x has no layer kernel", jet_mask);
    return e == cudaSuccess ? HRKAN_OK : cuda_fail(e, "adjoint launch");
}

}  // extern "C"
