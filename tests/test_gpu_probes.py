"""Measurement aids (no counterpart in the paper): the FP64 issue-rate probe
and the read-bandwidth probe that give the bench its ALU and L2 roofs.

Bounds are sanity bounds from the hardware's published form (GB300: FP64
at 2 FMA per clock per SM; L2 126 MB): the probes must measure what they
claim, reject bad arguments, and leave the pool as they found it."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_01216_gb300 import build
    build.build()
    from paper_1606_01216_gb300 import airga
    airga.lib()
    return airga


def test_fp64_rate_probe(G):
    f, tflops, ms = G.probe_fp64_rate(1 << 14)
    assert 1.0 <= f <= 4.5                       # FMAs per SM clock, cycle counters
    assert tflops > 0 and ms > 0
    with pytest.raises(G.AirgaError):
        G.probe_fp64_rate(0)


def test_read_bw_probe(G):
    torch.cuda.synchronize()
    used0 = G.debug_pool_used()
    l2, ms_l2 = G.probe_read_bw(64 << 20, 20)
    dram, ms_dram = G.probe_read_bw(2 << 30, 2)
    torch.cuda.synchronize()
    assert G.debug_pool_used() == used0          # the probe's buffer went back to the pool
    assert ms_l2 > 0 and ms_dram > 0
    assert 500.0 < dram < 20000.0                # GB/s
    assert l2 > dram                             # a buffer inside L2 reads faster than DRAM
    for bad in ((1000, 1), ((1 << 20) + 8, 1), (64 << 20, 0), (64 << 20, 1001)):
        with pytest.raises(G.AirgaError):
            G.probe_read_bw(*bad)
