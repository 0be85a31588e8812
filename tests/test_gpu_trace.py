"""Call tracing (airga_trace_enable / airga_trace_read): each traced C-ABI
call leaves one record, in call order, whose device time covers the work it
enqueued; the capacity bound counts the calls it could not keep; calls under
CUDA-graph capture are not traced; turning tracing off discards records."""
import numpy as np
import pytest

from paper_1606_01216_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
AL, BE = W.ALPHA, W.BETA


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_01216_gb300 import build
    build.build()
    from paper_1606_01216_gb300 import airga
    airga.lib()
    return airga


@pytest.fixture()
def system(G):
    beam = W.beam(20000)
    M, K = G.beam_mats(beam)
    f = torch.from_numpy(np.ascontiguousarray(W.loads(beam.n)[:, 0])).cuda()
    torch.cuda.synchronize()
    return M, K, f


def test_trace_records_each_call_in_order(G, system):
    M, K, f = system
    G.trace_enable(64)
    try:
        A = G.assemble_shifted(M, K, AL, BE, 0.1)
        P = G.spai_build(A)
        r = G.pcg_solve(A, P, f, G.options(tol=1e-10, maxit=20000))
        recs, dropped = G.trace_read()
    finally:
        G.trace_enable(0)
    assert dropped == 0
    assert [x["name"] for x in recs] == ["airga_assemble_shifted", "airga_spai_build",
                                        "airga_pcg_solve"]
    assert all(x["ms"] >= 0.0 for x in recs)
    # the solve's record covers its iterations: well above one microsecond each
    assert int(r["iters"][0]) > 50 and recs[2]["ms"] > 1e-3 * int(r["iters"][0])
    # the three intervals follow one another on the stream: the solve dominates
    assert recs[2]["ms"] > recs[0]["ms"]


def test_trace_capacity_counts_dropped_calls(G, system):
    M, K, f = system
    G.trace_enable(2)
    try:
        for s in (1.0, 2.0, 3.0, 4.0):
            G.assemble_shifted(M, K, AL, BE, s)
        recs, dropped = G.trace_read()
        assert [x["name"] for x in recs] == ["airga_assemble_shifted"] * 2
        assert dropped == 2
        recs, dropped = G.trace_read()
        assert recs == [] and dropped == 0
    finally:
        G.trace_enable(0)


def test_trace_skips_graph_capture_and_off_discards(G, system):
    M, K, f = system
    A = G.assemble_shifted(M, K, AL, BE, 5.0)
    P = G.spai_build(A)
    systems = [(A, P, f, torch.zeros_like(f))]
    B = G.Batch(systems)
    torch.cuda.synchronize()
    G.trace_enable(16)
    try:
        g = torch.cuda.CUDAGraph()
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            with torch.cuda.graph(g, stream=st):
                B.solve(stream=st)
        g.replay()
        torch.cuda.synchronize()
        recs, dropped = G.trace_read()
        assert recs == [] and dropped == 0          # the captured call left no record
        B.solve()                                   # an eager call does
        torch.cuda.synchronize()
        G.trace_enable(0)                           # off: the unread record is discarded
        G.trace_enable(16)
        recs, dropped = G.trace_read()
        assert recs == [] and dropped == 0
    finally:
        G.trace_enable(0)
    assert int(B.status[0]) == G.OK
