"""The work counts behind bench.py's roofline fractions, against numbers
derived by hand from the layer shapes.

* Algorithmic FP32 flops per point of a fused training step: the sparse
  contraction 2 (k+1) J I O per layer and pass (forward and weight gradient
  everywhere, the input adjoint past the first layer) plus 45 flops per active
  basis and unit (20 forward, 25 backward).
* Dense tensor-core flops of a step: 2 x rows x K x N with rows = J x points,
  K = I (G + k) and N = O, for every contraction that runs on the tensor cores.
* Launches of a layer-wise step: per point set a forward per layer, a weight
  gradient per layer and an input adjoint past the first layer, plus the
  residual and the reduction/Adam."""
import bench


def test_fp32_peak_from_unit_counts():
    assert abs(bench.FP32_PEAK_TFLOPS - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert abs(bench.FP32_PEAK_TFLOPS - 80.5) < 0.1


def test_algorithmic_flops_per_point_of_the_burgers_workload():
    # [2,10,10,1], k = 3, interior J = 4:
    #   contraction 2*4*4 * (2*10*2 + 10*10*3 + 10*1*3) = 32 * 370 = 11840
    #   bases 45 * 4 * (2 + 10 + 10) = 3960
    assert bench.alg_flops_per_point([2, 10, 10, 1], 3, 4) == 11840 + 3960
    # boundary points, J = 1: 2*4*1 * 370 + 3960
    assert bench.alg_flops_per_point([2, 10, 10, 1], 3, 1) == 8 * 370 + 3960


def test_dense_tensor_core_flops_of_the_precision_workload():
    # [2,64,64,64,1] G=32 (K = 64 * 35 = 2240, N = 64), 262144 interior points x 5 rows + 16384 boundary
    rows_all, rows_int = 5 * 262144 + 16384, 5 * 262144
    fwd = 2 * rows_all * 2240 * 64            # one hidden layer's forward: 380.5 GFLOP
    adj = 2 * rows_int * 2240 * 64            # its input adjoint (interior rows): 375.8 GFLOP
    assert fwd == 380_507_258_880 and adj == 375_809_638_400
    w = ([2, 64, 64, 64, 1], 32, 3, 262144, 5, 16384)
    assert bench.dense_tc_flops(*w, False) == 2 * fwd                       # TF32: forward of 2 hidden layers
    first_dw = 2 * rows_all * (2 * 35) * 64                                # first layer's gradient, K = 2 * 35
    assert bench.dense_tc_flops(*w, True) == 2 * (fwd + fwd + adj) + first_dw   # BF16: + dW and adjoint


def test_launches_of_a_layer_wise_step():
    widths = [2, 32, 32, 1]
    none = lambda l: False
    # per point set: 3 forwards + 3 weight gradients + 2 adjoints = 8; two sets; residual; reduction
    assert bench.launches_per_step(widths, 0, none, none, False) == 2 * 8 + 2
    assert bench.launches_per_step(widths, 0, none, none, True) == 2     # fused kernel + reduction
    # BF16 on the hidden layer: its forward and gradient each add a conversion launch, and the
    # interior set's adjoint of that layer is a tensor-core launch reusing the gradient's conversion
    hid = lambda l: l == 1
    assert bench.launches_per_step(widths, 1, hid, hid, False) == 2 * (4 + 6) + 1 + 2


def test_layerwise_batched_launch_count_matches_the_launch_list():
    """The BF16 multi-instance step of [2,16,16,1] G=10 launches 21 kernels (ncu launch list of the
    bench, profiles/batched_bf16_step_poisson_batch256.md): 3 gathers, forward 3 + 3, output-layer
    kernels 2, backward 3 + 1 (interior: gradients handed over in BF16) and 3 + 2 (boundary), 1
    reduction; FP32 replaces every tensor-core call by one SIMT launch."""
    assert bench.layerwise_batched_launches([2, 16, 16, 1], 10, 3, 1, 0x1F) == 21
    # FP32: 3 gathers, 2 x 2 forwards, 2 output-layer kernels, 2 x (2 + 1) backward, 1 reduction
    assert bench.layerwise_batched_launches([2, 16, 16, 1], 10, 3, 0, 0x1F) == 3 + 2 * 2 + 2 + 2 * 3 + 1
    # path 2 (every forward on the FP32 SIMT kernels): the forward's two weight conversions go
    assert bench.layerwise_batched_launches([2, 16, 16, 1], 10, 3, 1, 0x1F, fwd_tc=False) == 19


def test_tensor_core_bytes_of_a_layer_wise_step():
    """Algorithmic bytes of the tensor-core kinds on [2,16,16,1], J = 5, 100 interior + 10 boundary
    points (510 jet rows), written out by hand: forward of the hidden layer 4*(16+16)*510; weight
    gradient of the first layer (coordinates 8 B/point, BF16 gradient 2*16*510) and of the hidden
    layer (4*16*510 + 2*16*510); adjoint of the hidden layer on the interior jet rows, input
    jets FP32, gradient BF16 in and out (the first layer's weight gradient runs on tensor cores)."""
    b = bench.layerwise_tc_bytes([2, 16, 16, 1], 10, 3, 5, 100, 10, 1)
    assert b[5] == 4 * 32 * 510
    assert b[6] == (8 * 110 + 2 * 16 * 510) + (4 * 16 * 510 + 2 * 16 * 510)
    assert b[7] == (4 * 16 + 2 * 16 + 2 * 16) * 5 * 100
    # TF32 runs only the forward on tensor cores
    b32 = bench.layerwise_tc_bytes([2, 16, 16, 1], 10, 3, 5, 100, 10, 2)
    assert b32[5] == 4 * 32 * 510 and b32[6] == 0 and b32[7] == 0
    # path 2: no tensor-core forward, the backward's bytes as before
    b2 = bench.layerwise_tc_bytes([2, 16, 16, 1], 10, 3, 5, 100, 10, 1, fwd_tc=False)
    assert b2[5] == 0 and b2[6] == b[6] and b2[7] == b[7]
