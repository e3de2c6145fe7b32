/*
 * hrkan.h — C ABI of the GB300 (sm_103a) HRKAN physics-informed training library.
 *
 * The library evaluates Higher-order-ReLU KANs (Section 3, Eq. 2 of
 * "Higher-order-ReLU-KANs (HRKANs) for solving physics-informed neural
 * networks (PINNs) more accurately, robustly and faster") together with the
 * input-derivative jets a PDE residual needs, the residual/loss of the Poisson
 * (Eq. 3-4) and Burgers (Eq. 6-8) problems, a hand-written weight-gradient
 * backward and the Adam update (Section 4).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers named W, dW, x, jets, tape, loss, dL_* are DEVICE pointers owned by
 *   the caller; the library never frees them.  Structs passed by pointer
 *   (hrkan_cfg, pinn_problem) are HOST memory, read during the call only.
 * - A network with widths [w_0, ..., w_L] (w_0 = D = 2 input coordinates,
 *   w_L = 1 output) has L layers.  Layer l maps I = w_l units to O = w_{l+1}
 *   units with weights W_l[O][I][n], n = G + k bases per input unit (row-major,
 *   basis index fastest).  W is the concatenation of W_0 .. W_{L-1}, float32;
 *   its length P is hrkan_param_count().  Layer output o is
 *       y_o = sum_j sum_i W_l[o][j][i] v_i(z_j)
 *   with no bias, no base branch and no normalisation between layers.
 * - Supports (Sections 2.1-2.2, "the same support as the B-spline basis"):
 *   h = (grid_hi - grid_lo)/G, s_i = grid_lo + (i-k)h, e_i = grid_lo + (i+1)h,
 *   i = 0..n-1, the same for every layer.  Inputs outside [s_0, e_{n-1}] touch
 *   no basis (all contributions are exactly zero).
 * - Coordinates x are structure-of-arrays float32 [D][N] (x[d*N + p]), D = 2,
 *   or D = 3 for FP32 single networks (hrkan_forward_jets, hrkan_backward, and
 *   with the Poisson kind in three coordinates pinn_residual_loss,
 *   hrkan_train_step and hrkan_train_step_partial; their jet mask has bit 0 =
 *   u, bit 1+d = du/dx_d, bit 4+d = d2u/dx_d^2; the single-layer and
 *   multi-instance calls return HRKAN_EUNSUPPORTED).
 * - Jet rows: bit 0 of a jet mask selects u, bit 1+d selects du/dx_d, bit 1+D+d
 *   selects d2u/dx_d^2, bit 1+2D+d selects d3u/dx_d^3, bit 1+3D = 7 selects
 *   the mixed d2u/dx_0dx_1 (D = 2: 0x1F = u,u_x,u_y,u_xx,u_yy; 0x0F =
 *   u,u_x,u_t,u_xx with coordinates (x, t); 0x2F = u,u_x,u_t,u_xx,u_xxx; 0x87 =
 *   u,u_x,u_y,u_xy; 0xFF = all eight).  For D = 2, bits 8+d select
 *   d4u/dx_d^4 and bits 10+d d5u/dx_d^5 (Section 3: a fifth derivative asks for
 *   m = 6; 0x12F = u,u_x,u_t,u_xx,u_xxx,u_xxxx; 0x52F adds u_xxxxx).  A
 *   derivative bit requires the bit one order lower of the same dimension (the
 *   mixed bit: both first-order bits).  Third-derivative, mixed, fourth and
 *   fifth rows run on the layer-wise path in FP32 (masks 0x2F, 0x7F, 0x87,
 *   0xFF, 0x12F, 0x52F; the fused narrow kernels and the tensor-core kernels
 *   take 0x01, 0x0F, 0x1F and return HRKAN_EUNSUPPORTED, or fall back to the
 *   FP32 layer kernels, otherwise; other valid masks return HRKAN_EUNSUPPORTED).
 *   Jet arrays are float32 [J][N], rows in bit order, J = popcount(mask).
 * - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *   default stream).  Argument errors are detected before anything is
 *   enqueued and return HRKAN_EINVAL (or HRKAN_EUNSUPPORTED for valid but
 *   unimplemented shapes); a launch failure returns HRKAN_ECUDA.  On any
 *   non-OK status hrkan_last_error() holds a message.
 * - A handle is not thread-safe: calls on one handle must not overlap in
 *   time from several host threads.  Work enqueued on different streams for
 *   the same handle must not overlap on the GPU (they share its workspace).
 */
#ifndef HRKAN_H
#define HRKAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hrkan_ctx* hrkan_t;   /* opaque, owned by the library */
typedef void* hrkan_stream_t;        /* a cudaStream_t */

enum hrkan_status {
    HRKAN_OK = 0,
    HRKAN_EINVAL = -1,        /* bad argument (null pointer, bad size or mask) */
    HRKAN_ENOMEM = -2,        /* device or host allocation failed */
    HRKAN_ECUDA = -3,         /* a CUDA call or kernel launch failed */
    HRKAN_EUNSUPPORTED = -4,  /* valid request that this library does not implement */
    HRKAN_ETIMEOUT = -5,      /* a bounded device-side wait gave up */
    HRKAN_ENONFINITE = -6,    /* the loss became NaN or infinite */
    HRKAN_EIO = -7            /* a checkpoint file could not be written, or read back whole */
};

enum hrkan_prec { HRKAN_FP32 = 0, HRKAN_BF16 = 1, HRKAN_TF32 = 2 };
enum hrkan_pde { HRKAN_POISSON = 0, HRKAN_BURGERS = 1, HRKAN_KDV = 2, HRKAN_POISSON3 = 3 };

#define HRKAN_MAX_WIDTHS 8
/* Use the layer-wise kernels even where a fused whole-network kernel exists. */
#define HRKAN_FLAG_LAYERWISE 1

typedef struct hrkan_cfg {
    int n_widths;                    /* L + 1, in [2, HRKAN_MAX_WIDTHS] */
    int widths[HRKAN_MAX_WIDTHS];    /* widths[0] = D = 2 or 3 inputs, widths[n_widths-1] = 1, all <= 64 */
    int G;                           /* grid intervals on [grid_lo, grid_hi], >= 1 */
    int k;                           /* support width in cells minus one (B-spline order); 3 */
    int m;                           /* HR order of Eq. 2: 2..6 (FP32); the fused narrow and tensor-core kernels need 4 */
    int prec;                        /* enum hrkan_prec: arithmetic of the jet contraction.  BF16 /
                                        TF32: hidden layers with 16 <= O <= 64 (O % 16 == 0) and
                                        G + k <= 64 contract on tcgen05 tensor cores (FP32
                                        accumulation in TMEM).  BF16 forward: every input of a
                                        product carried as two bfloat16 values (x = x_hi + x_lo) and
                                        the product as a_hi w_hi + a_lo w_hi + a_hi w_lo; BF16 weight
                                        gradient and input adjoint: inputs rounded to bfloat16 once;
                                        TF32: the forward's inputs rounded to TF32 once.  The first
                                        and last layers (but for the BF16 weight gradient of the first
                                        layer) and the other hidden layers stay FP32
                                        (hrkan_profile_read(HRKAN_KERNEL_TENSOR) counts the tensor
                                        launches).  Needs the layer-wise path (a shape without a
                                        fused kernel, or HRKAN_FLAG_LAYERWISE) */
    double grid_lo, grid_hi;         /* grid_lo < grid_hi */
    int n_instances;                 /* independent networks sharing the shape (>= 1) */
    int flags;                       /* HRKAN_FLAG_*; 0 = defaults */
    size_t hbm_budget_bytes;         /* layer-wise path: the training step keeps every layer's input
                                        jets (the tape) while they fit in this many bytes, else it
                                        recomputes them in the backward; 0 = no cap */
} hrkan_cfg;

/*
 * A PINN problem (Section 4).  Residual r per interior point:
 *   HRKAN_POISSON: r = u_xx + u_yy + (a^2+b^2) pi^2 sin(a pi x) sin(b pi y)
 *                  (Eq. 3 with a = b = 1: u* = sin(pi x) sin(pi y))
 *   HRKAN_BURGERS: r = u_t + lam u u_x - nu u_xx, coordinates (x, t)
 *                  (Eq. 6 has lam = 1; the rescaled Eq. 7 has lam = 1/4, nu/16)
 *   HRKAN_KDV:     r = u_t + lam u u_x + nu u_xxx, coordinates (x, t)
 *   HRKAN_POISSON3 (three-input networks only, every other kind two-input
 *                  only; else HRKAN_EUNSUPPORTED): Eq. 3 in three coordinates,
 *                  r = u_xx + u_yy + u_zz + (a^2+b^2+c^2) pi^2 sin(a pi x)
 *                  sin(b pi y) sin(c pi z) with c = lam, interior mask 0x7F
 * Loss (Eq. 4, Eq. 8): L = alpha mean_int(r^2) + mean_bnd((u - g)^2), the
 * boundary mean pooled over every boundary and initial-condition point.
 */
typedef struct pinn_problem {
    int kind;       /* enum hrkan_pde */
    int reserved;
    double a, b;    /* Poisson source frequencies */
    double lam, nu; /* Burgers: r = u_t + lam u u_x - nu u_xx; KdV: r = u_t + lam u u_x + nu u_xxx;
                       HRKAN_POISSON3: lam = c, the third source frequency */
    double alpha;   /* weight of the PDE term */
} pinn_problem;

/* Number of float weights P of one network of this shape: sum over layers of
 * I * O * n with n = G + k bases per input unit (Sections 2.1-2.2).  0 on an
 * invalid cfg (no status: the count is the return value). */
int64_t hrkan_param_count(const hrkan_cfg* cfg);

/*
 * Create a handle for networks of shape cfg (the problem statement of
 * Section 4: widths, grid g, order k, HR order m).  Allocates the device
 * workspace and the FP64 Adam moments (zeroed) on the current device.
 * Returns HRKAN_EINVAL for an invalid cfg, HRKAN_EUNSUPPORTED for a valid
 * shape this library has no kernels for, HRKAN_ENOMEM if allocation fails.
 */
int hrkan_init(hrkan_t* out, const hrkan_cfg* cfg);

/* Release the handle and its device memory (synchronises the device). NULL is a no-op. */
void hrkan_destroy(hrkan_t h);

/* Message of the last non-OK status returned on this host thread ("" if none). */
const char* hrkan_last_error(void);

/*
 * Floats of tape that hrkan_forward_jets may fill for N points under mask so
 * that hrkan_backward can skip recomputing the forward: the input jets of
 * every layer but the first, [J][w_l][N] per layer.  0: the handle uses a
 * fused kernel, which recomputes inside the backward (pass NULL).
 */
int64_t hrkan_tape_floats(hrkan_t h, int64_t N, unsigned jet_mask);

/*
 * Network output jets at N points (Sections 1-3: the KAN layer as a matrix
 * operation, Eq. 2 bases; jets by the chain rule, Eq. 3 and Eq. 6 need them).
 *   W     [P] float32, x [2][N], jets [J][N] (written).
 *   tape  NULL, or hrkan_tape_floats(h, N, jet_mask) floats to keep the layer
 *         jets for hrkan_backward.
 * N = 0 is a valid no-op.
 * Errors: HRKAN_EINVAL for a NULL handle, N < 0, an invalid mask (a bit
 * without the bit it requires, bit 0 missing, bits above 11, or above 6 for
 * D = 3) or NULL W / x / jets with N > 0; HRKAN_EUNSUPPORTED for a mask the
 * handle's kernels lack (third-order, mixed, fourth and fifth rows on the fused
 * shapes; a mask without a layer kernel).
 */
int hrkan_forward_jets(hrkan_t h, const float* W, const float* x, int64_t N, unsigned jet_mask,
                       float* jets, float* tape, hrkan_stream_t stream);

/*
 * One layer of the network applied to given input jets (the KAN layer of
 * Sections 1-3 with its jets): layer index l, W = that layer's weights
 * [O][I][n] (a pointer into the network's W), z = input jets [J][I][N] (for
 * l = 0: the coordinates [2][N]), y = output jets [J][O][N] (written).  Runs
 * the same kernel the network forward would use for that layer under the
 * handle's precision (tensor cores for BF16/TF32 hidden layers).
 * Errors (also of hrkan_layer_dw and hrkan_layer_adjoint): HRKAN_EINVAL for a
 * NULL handle or pointer, N < 0, an invalid mask or a layer index outside
 * [0, L) ([1, L) for the adjoint); HRKAN_EUNSUPPORTED on a three-input handle.
 */
int hrkan_layer_jets(hrkan_t h, int layer, const float* W, const float* z, int64_t N, unsigned jet_mask,
                     float* y, hrkan_stream_t stream);

/*
 * Weight gradient of one layer (reverse mode of hrkan_layer_jets w.r.t. that
 * layer's weights): dW[o][j][i] = sum_p sum_r gy[r][o][p] * A_r[p][j][i] with
 * the basis-matrix entries A_r of the layer (Sections 2-3), z = input jets
 * [J][I][N] (l = 0: the coordinates [2][N]), gy = dL/d(output jets) [J][O][N],
 * dW = [O][I][n] float32 (written).  Runs the kernel the network backward uses
 * for that layer (tensor cores for BF16 hidden layers), then a fixed-order sum
 * of its partial rows.  N = 0 writes zeros.
 */
int hrkan_layer_dw(hrkan_t h, int layer, const float* z, const float* gy, int64_t N, unsigned jet_mask,
                   float* dW, hrkan_stream_t stream);

/*
 * Input adjoint of one layer l >= 1 (reverse mode of hrkan_layer_jets w.r.t.
 * its input jets, through the third basis derivative of Eq. 2, the fourth for
 * third-derivative rows):
 * gz = d/dz of sum_{r,o,p} gy[r][o][p] * y_r[o][p] for W = that layer's
 * weights [O][I][n] (a pointer into the network's W), z = input jets
 * [J][I][N], gy [J][O][N], gz [J][I][N] (written).  Runs the kernel the
 * network backward uses (tensor cores for BF16 hidden layers with masks 0x0F
 * and 0x1F).
 */
int hrkan_layer_adjoint(hrkan_t h, int layer, const float* W, const float* z, const float* gy, int64_t N,
                        unsigned jet_mask, float* gz, hrkan_stream_t stream);

/*
 * Residual and loss (Eq. 3-4 / Eq. 6-8) from precomputed jets.
 *   x_int [D][N_int], jets_int [J][N_int] under jet_mask (Poisson needs u_xx,
 *   u_yy; Burgers needs u, u_x, u_t, u_xx; the Poisson kind in three
 *   coordinates takes exactly the mask 0x7F), u_bnd / g_bnd [N_bnd] network
 *   values and targets at the boundary/initial points.
 *   loss          [3] float64 device: L, mean r^2, mean (u-g)^2 (written).
 *   dL_djets_int  [J][N_int] (written; NULL to skip), dL_du_bnd [N_bnd]
 *                 (written; NULL to skip).
 * The loss is squared per point in float32, summed per block in float64, and
 * across blocks by a fixed-order pairwise float64 tree (all terms are
 * non-negative, so the relative error stays near log2(blocks) * 2^-53).
 */
int pinn_residual_loss(hrkan_t h, const pinn_problem* prob, const float* x_int, int64_t N_int,
                       unsigned jet_mask, const float* jets_int, const float* u_bnd,
                       const float* g_bnd, int64_t N_bnd, double* loss, float* dL_djets_int,
                       float* dL_du_bnd, hrkan_stream_t stream);

/*
 * Weight gradient of sum_{r,p} dL_djets[r][p] * jets[r][p] (reverse mode of
 * hrkan_forward_jets; the training of Section 4 needs it for Adam).
 *   tape        NULL (recompute the forward) or the tape of a preceding
 *               hrkan_forward_jets on the same W, x, N, jet_mask.
 *   dW          [P] float32: overwritten (accumulate = 0) or added to (1).
 * Cross-block sums run in a fixed order; within a block float32 atomics in
 * shared memory make the last bits order-dependent.
 * Errors: as hrkan_forward_jets; W and dW are required even for N = 0, when
 * dW is zeroed (accumulate = 0) or left as it is (1).
 */
int hrkan_backward(hrkan_t h, const float* W, const float* x, int64_t N, unsigned jet_mask,
                   const float* tape, const float* dL_djets, float* dW, int accumulate,
                   hrkan_stream_t stream);

/*
 * Adam step t >= 1 on W [P] float32 with gradient dW [P] (Section 4 trains
 * every model with Adam).  The first and second moments live in the handle in
 * float64 (zeroed by hrkan_init and hrkan_reset_moments):
 *   m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
 *   W <- W - lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps)
 * Errors: HRKAN_EINVAL for a NULL handle or pointer, t < 1, b1 or b2 outside
 * [0, 1), eps < 0 or a non-finite lr.
 */
int adam_step(hrkan_t h, float* W, const float* dW, double lr, double b1, double b2, double eps,
              int t, hrkan_stream_t stream);

/*
 * Synchronise the device and report device-side failures recorded since the
 * last call: HRKAN_ETIMEOUT if a bounded wait inside a tensor-core kernel gave
 * up (the kernel then skipped its output, freed its tensor memory and
 * returned); HRKAN_ENONFINITE if a loss computed by pinn_residual_loss or a
 * training step was NaN or infinite.  The first failure is kept.  Clears the
 * record.
 */
int hrkan_sync_status(hrkan_t h);

/*
 * Limit of the tensor-core kernels' bounded waits in GPU clock cycles (0 =
 * the default, about one second).  A small value makes those waits give up
 * early, so that a test can exercise the timeout path (the kernel records
 * HRKAN_ETIMEOUT, waits with the default limit for its own copies and MMAs,
 * frees its tensor memory and returns; the handle stays usable).  Synchronises
 * the device.
 */
int hrkan_set_wait_cycles(hrkan_t h, int64_t cycles);

/* Zero the Adam moments and the device step counter of the handle (a fresh
 * start of the Adam training of Section 4).  HRKAN_EINVAL for a NULL handle. */
int hrkan_reset_moments(hrkan_t h, hrkan_stream_t stream);

/*
 * One full-batch training step (Section 4: the loss of Eq. 4 / Eq. 8
 * minimised by Adam), fused: forward jets at the interior and boundary
 * points, residual and loss, backward, cross-block reduction and Adam.  Same
 * arithmetic as hrkan_forward_jets + pinn_residual_loss + hrkan_backward +
 * adam_step; the interior mask is 0x1F for Poisson, 0x0F for Burgers, 0x2F
 * for KdV and 0x7F for the Poisson kind in three coordinates (a three-input
 * network: the two-pass forward and backward of hrkan_forward_jets /
 * hrkan_backward with the layer inputs recomputed, a residual kernel, the
 * reduction with Adam).
 *   W      [P] float32, updated in place.
 *   t      Adam step >= 1, or 0: take the step from a device-side counter of
 *          the handle (zeroed by hrkan_init / hrkan_reset_moments) and advance
 *          it on the device, so that one captured CUDA graph of this call can
 *          be replayed for successive steps.
 *   loss   [3] float64 device: the loss at W before the update (written).
 *   dW     NULL, or [P] float32 receiving the gradient.
 * No host synchronisation; capturable in a CUDA graph after one warm-up call
 * (with profiling disabled).
 * Errors: HRKAN_EINVAL for a NULL handle or pointer, a bad problem (kind,
 * non-finite coefficient), N_int + N_bnd = 0, t < 0 or bad Adam
 * hyper-parameters; HRKAN_EUNSUPPORTED for a kind that does not match the
 * network's input count (HRKAN_POISSON3 takes three inputs, the others two)
 * and for KdV on the fused shapes.
 */
int hrkan_train_step(hrkan_t h, const pinn_problem* prob, float* W, const float* x_int,
                     int64_t N_int, const float* x_bnd, const float* g_bnd, int64_t N_bnd,
                     double lr, double b1, double b2, double eps, int t, double* loss, float* dW,
                     hrkan_stream_t stream);

/*
 * One shard's part of a data-parallel training step (the loss of Eq. 4 /
 * Eq. 8 is a sum over points, so its gradient is the sum of the shards'
 * contributions): forward jets at this shard's N_int interior and N_bnd
 * boundary points, residual, backward and the fixed-order reduction, with the
 * means taken over N_int_total / N_bnd_total points (the counts of all shards
 * together), and no Adam update.
 *   W      [P] float32, read only.
 *   loss   [3] float64 device: this shard's contributions to L, mean r^2 and
 *          mean (u-g)^2 (written); summed over the shards they are the loss.
 *   dW     [P] float32 device: this shard's contribution to the gradient
 *          (written); summed over the shards it is the step's gradient.
 * A data-parallel step sums loss and dW over the shards (an all-reduce) and
 * then calls adam_step with the same arguments on every replica.  A shard with
 * no points writes zeros.
 * Errors: as hrkan_train_step, and HRKAN_EINVAL for totals below this shard's
 * counts or a NULL dW.
 */
int hrkan_train_step_partial(hrkan_t h, const pinn_problem* prob, const float* W, const float* x_int,
                             int64_t N_int, const float* x_bnd, const float* g_bnd, int64_t N_bnd,
                             int64_t N_int_total, int64_t N_bnd_total, double* loss, float* dW,
                             hrkan_stream_t stream);

/*
 * Many independent networks of the handle's shape trained together (the
 * multi-instance workload of the training experiments of Section 4, run as a
 * batch).  cfg.n_instances = I networks; W is [I][P]; instance i owns interior
 * points [off_int[i], off_int[i+1]) of x_int [2][N] and boundary points
 * [off_bnd[i], off_bnd[i+1]) of x_bnd / g_bnd.
 *   probs      host [I]: kind, lam, nu and alpha must agree; a, b may differ.
 *   off_int, off_bnd  host [I+1], non-decreasing, starting at 0.
 *   t          Adam step >= 1, or 0 for the device step counter (as in
 *              hrkan_train_step); the moments of instance i are its own.
 *   loss       device [I][3] float64 (L, mean r^2, mean (u-g)^2 per instance).
 *   dW         NULL, or device [I][P] float32 receiving each instance's gradient.
 * Kernel families (hrkan_set_batch_path): path 0, the fused shapes' persistent
 * multi-instance kernel plus one per-instance reduction/Adam launch (work
 * items of hrkan_set_batch_items points); paths 1 and 2, the layer-wise
 * kernels, each launched once over all instances (weight-gradient chunks of
 * hrkan_set_batch_items points), the boundary set's kernels on a side stream
 * of the handle that is forked from `stream` and joined back into it before
 * the reduction (in order on `stream` while hrkan_profile_enable is on).
 * The work layout is rebuilt and uploaded only when the offsets or problems
 * change (that call synchronises the stream); calls with unchanged arguments
 * only enqueue kernels, so they can be captured in a CUDA graph after one
 * warm-up call (which also creates the side stream and the scratch).
 * Errors: HRKAN_EINVAL for a NULL handle, array or (with points) pointer,
 * problems that disagree in kind, lam, nu or alpha, offsets that decrease or
 * do not start at 0, t < 0 or bad Adam hyper-parameters; HRKAN_EUNSUPPORTED
 * for a problem kind or shape without kernels on the handle's path.
 */
int hrkan_train_step_batched(hrkan_t h, const pinn_problem* probs, float* W, const float* x_int,
                             const int64_t* off_int, const float* x_bnd, const float* g_bnd,
                             const int64_t* off_bnd, double lr, double b1, double b2, double eps, int t,
                             double* loss, float* dW, hrkan_stream_t stream);

/* Output jets of every instance at its points (x [2][N], offsets host [I+1], jets [J][N]);
 * the same handle requirement as hrkan_train_step_batched.  HRKAN_EINVAL for a
 * NULL handle, offsets or (with points) pointer, decreasing offsets or an
 * invalid mask. */
int hrkan_forward_jets_batched(hrkan_t h, const float* W, const float* x, const int64_t* offsets,
                               unsigned jet_mask, float* jets, hrkan_stream_t stream);

/* Points per work item of the multi-instance calls (default 1024; on the
 * layer-wise path: points per weight-gradient chunk); a tuning knob.
 * HRKAN_EINVAL for a NULL handle or points_per_item < 1. */
int hrkan_set_batch_items(hrkan_t h, int points_per_item);

/* Kernel family of the multi-instance calls (hrkan_train_step_batched,
 * hrkan_forward_jets_batched): 0 = the fused multi-instance kernel (shapes
 * with a fused kernel), 1 = the layer-wise kernels, one launch per layer
 * kernel over all instances (every layer-wise handle; a fused shape may choose
 * it too), 2 = the layer-wise kernels with every layer's forward on the FP32
 * SIMT kernels, so that a BF16/TF32 handle uses the tensor cores for the
 * weight gradient and the input adjoint only (on narrow layers, O = 16, the
 * FP32 forward is the faster one, and it carries no rounding of the
 * contraction's inputs; for an FP32 handle 2 runs the same kernels as 1).
 * hrkan_autotune_batch may pick any of them.
 * hrkan_set_batch_path: HRKAN_EINVAL for a NULL handle or a path other than
 * 0, 1 and 2, HRKAN_EUNSUPPORTED for 0 on a shape without a fused kernel.
 * hrkan_batch_path returns the current family (0, 1 or 2), or HRKAN_EINVAL
 * for a NULL handle. */
int hrkan_set_batch_path(hrkan_t h, int path);
int hrkan_batch_path(hrkan_t h);

/*
 * Picks the points per work item of the multi-instance training step by
 * timing it: for each candidate (NULL: 256, 512, 1024, 2048, 4096) one
 * untimed call, then `reps` (< 1: 3) calls timed with CUDA events on the
 * stream, all with lr = 0 so that W keeps its values; the fastest candidate
 * becomes the handle's item size.  On a shape with a fused kernel both kernel
 * families are timed with every candidate (hrkan_set_batch_path), on a
 * BF16/TF32 handle also path 2, and the fastest pair is kept; a family without
 * kernels for the problem is skipped.  Arguments as hrkan_train_step_batched.
 * Synchronises the stream; resets the Adam moments and the device step
 * counter (call it before training).  chosen / ms_per_step (host, may be
 * NULL) receive the winner and its time per step.
 * Errors: those of hrkan_train_step_batched, and HRKAN_EINVAL for
 * n_candidates < 1 or a candidate below 1 point.
 */
int hrkan_autotune_batch(hrkan_t h, const pinn_problem* probs, float* W, const float* x_int,
                         const int64_t* off_int, const float* x_bnd, const float* g_bnd,
                         const int64_t* off_bnd, const int* candidates, int n_candidates, int reps,
                         int* chosen, double* ms_per_step, hrkan_stream_t stream);

/*
 * hrkan_backward without any allocation (the paper has no counterpart; this is
 * for callers that cannot call cudaMalloc, e.g. code running under another
 * framework's memory pool or with all device memory reserved up front, which
 * therefore cannot create a handle).  Same arguments and result as
 * hrkan_backward, but the network shape comes from cfg and no handle, tape or
 * workspace is used: the per-block gradient partials live in a file-scope
 * static device array of 1 Mi floats (4 MiB), which every GPU that loads the
 * library holds until the process exits.
 *   - Networks with more than 1 Mi weights are rejected with HRKAN_EINVAL;
 *     only the fused narrow shapes are supported (else HRKAN_EUNSUPPORTED).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current, and looks it up again
 *     whenever the current context differs from the one of the cached address
 *     (after cudaDeviceReset the module, and with it the array, is loaded
 *     anew); make the first call in each context before any stream capture.
 *   - Every call shares the one array and leaves its partials there; each
 *     call overwrites the rows it reads, so nothing needs clearing, but calls
 *     whose work overlaps on the GPU (other streams, other threads) race.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 */
int hrkan_backward_noalloc(const hrkan_cfg* cfg, const float* W, const float* x, int64_t N,
                           unsigned jet_mask, const float* dL_djets, float* dW, int accumulate,
                           hrkan_stream_t stream);

/*
 * Kernel timing.  While enabled, every kernel the handle launches is
 * bracketed by two CUDA events on its stream (do not enable it around stream
 * capture).  hrkan_profile_read waits for the recorded events, adds their
 * elapsed times to per-class totals, and returns the total milliseconds and
 * launch count of one class (optionally resetting that class).
 */
enum hrkan_kernel_class {
    HRKAN_KERNEL_FUSED = 0,     /* fused forward+residual+backward (or backward) kernel */
    HRKAN_KERNEL_REDUCE = 1,    /* cross-block gradient/loss reduction and Adam */
    HRKAN_KERNEL_FORWARD = 2,   /* forward jets */
    HRKAN_KERNEL_RESIDUAL = 3,  /* stand-alone residual */
    HRKAN_KERNEL_TENSOR = 4,    /* tcgen05 jet contraction of a hidden layer (BF16 / TF32) */
    /* Finer kinds of the layer-wise path, each launch also counted in one class above:
     * a tensor-core call includes its operand conversion kernel. */
    HRKAN_KERNEL_TC_FWD = 5,    /* tensor-core forward of a layer (tc_fwd_kernel) */
    HRKAN_KERNEL_TC_DW = 6,     /* tensor-core weight gradient of a layer (tc_dw_kernel) */
    HRKAN_KERNEL_TC_ADJ = 7,    /* tensor-core input adjoint of a layer (tc_adj_kernel) */
    HRKAN_KERNEL_LAYER_FWD = 8, /* FP32 layer forward (wide_fwd_kernel) */
    HRKAN_KERNEL_LAYER_DW = 9,  /* FP32 layer weight gradient (wide_dw_kernel) */
    HRKAN_KERNEL_LAYER_ADJ = 10, /* FP32 layer input adjoint (wide_adjoint_kernel) */
    HRKAN_KERNEL_CLASSES = 11
};
int hrkan_profile_enable(hrkan_t h, int enable);
int hrkan_profile_read(hrkan_t h, int kernel_class, double* total_ms, int64_t* launches, int reset);

/*
 * Checkpoint / resume of the training state that Section 4's Adam runs carry
 * from step to step: the weights, both Adam moments and the step counts.
 *
 * File layout (host byte order, little-endian on every supported host):
 *   bytes 0-7    magic "HRKANCK1"
 *   uint32       version (1)
 *   uint32       n_instances
 *   int64        P (weights per instance, hrkan_param_count)
 *   int64        t (the caller's Adam step count, stored as given)
 *   int64        t_device (steps taken with t = 0, the handle's device counter)
 *   float32      W [n_instances * P]
 *   float64      m [n_instances * P]  (first moment)
 *   float64      v [n_instances * P]  (second moment)
 * The file is written to "<path>.part" and renamed onto path, so a failed write
 * never leaves a partial checkpoint under path.
 *
 * hrkan_checkpoint_write / _read work on HOST buffers (W, m, v of n_instances
 * * P elements; the caller owns them); _read checks the magic, the version and
 * that P and n_instances match (HRKAN_EINVAL otherwise), and fails with
 * HRKAN_EIO on a missing, short or over-long file.
 *
 * hrkan_save / hrkan_load move the state of a handle: W is the DEVICE weight
 * buffer [n_instances * P] float32, the moments and the device step counter
 * are the handle's.  Both synchronise `stream` (file I/O is blocking) and
 * allocate temporary host buffers (HRKAN_ENOMEM if that fails).  hrkan_load
 * writes W, the moments and the counter, and returns the stored caller step
 * count in *t (may be NULL); a failed load leaves the handle and W unchanged.
 */
int hrkan_checkpoint_write(const char* path, int64_t P, int n_instances, int64_t t, int64_t t_device,
                           const float* W, const double* m, const double* v);
int hrkan_checkpoint_read(const char* path, int64_t P, int n_instances, int64_t* t, int64_t* t_device,
                          float* W, double* m, double* v);
int hrkan_save(hrkan_t h, const float* W, int64_t t, const char* path, hrkan_stream_t stream);
int hrkan_load(hrkan_t h, float* W, int64_t* t, const char* path, hrkan_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* HRKAN_H */
