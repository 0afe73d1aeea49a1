"""FP64 pipe probes: measured DFMA and mma.sync f64 (DMMA) throughput on this GPU.

The FP64 factorization is bounded by the chip's FP64 rate; these probes measure it in the same
process as the benchmark.  GB300's FP64 is 152 SMs x 2 FMA/clk (about 1.26 TFLOP/s at
2.07 GHz): a probe far above that would mean the chains were optimised away, far below that
the probe does not fill the pipe."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_probes_measure_the_fp64_pipe():
    import torch
    assert torch.cuda.is_available()
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    fma = P.rs_fp64_probe(P.RS_PROBE_DFMA)
    mma = P.rs_fp64_probe(P.RS_PROBE_DMMA)
    print("FP64 probe: DFMA %.3f TFLOP/s, DMMA %.3f TFLOP/s" % (fma, mma))
    assert 0.5 <= fma <= 1.6, fma
    assert 0.05 <= mma <= 10.0, mma


def test_bf16_mma_probe_measures_the_tensor_pipe():
    """The bf16 mma.sync rate that the digit-slice FP64 products run on: well above the FP64
    rate (hundreds of TFLOP/s) and below the 2.25 PFLOP/s dense bf16 figure of the tensor cores."""
    import torch
    assert torch.cuda.is_available()
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    r = P.rs_fp64_probe(P.RS_PROBE_BF16_MMA)
    print("bf16 mma.sync probe: %.1f TFLOP/s" % r)
    assert 50.0 <= r <= 2300.0, r
