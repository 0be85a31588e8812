"""Batched persistent PCG (airga_batch_*) against the CPU oracle: uneven
beams x shifts x right-hand sides in one launch, graph capture and replay,
and re-planning with measured costs (the autotuner's hook)."""
import numpy as np
import pytest

import oracle as O
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


def make_systems(G, spec, seed=3):
    """spec: list of (n_e, shifts, m).  Returns systems, oracle data."""
    systems, ref = [], []
    keep = []
    for (n_e, shifts, m) in spec:
        beam = W.beam(n_e)
        M, K = G.beam_mats(beam)
        F = W.loads(beam.n, m, seed=seed)
        keep.append((M, K))
        for s in shifts:
            A = G.assemble_shifted(M, K, AL, BE, s)
            P = G.spai_build(A)
            for c in range(m):
                f = torch.from_numpy(np.ascontiguousarray(F[:, c])).cuda()
                x = torch.zeros(beam.n, dtype=torch.float64, device="cuda")
                systems.append((A, P, f, x))
                ref.append((beam, s, F[:, c]))
    return systems, ref, keep


SPEC = [(37, [0.3, 20.0], 1), (900, [0.1, 2.0, 500.0], 2), (5000, [1.0], 3), (12, [5.0], 1)]


@pytest.mark.parametrize("share", [1, 2], ids=["cta_per_sm", "two_ctas_per_sm"])
@pytest.mark.parametrize("grouped", [False, True], ids=["single", "rhs_grouped"])
@pytest.mark.parametrize("rows", [0, 64, 700])
def test_batch_matches_oracle(G, rows, grouped, share):
    from paper_1606_01216_gb300 import autotune
    systems, ref, keep = make_systems(G, SPEC)
    group = autotune.rhs_groups(systems) if grouped else None
    B = G.Batch(systems, G.options(sm_share=share), rows_per_cta=rows, group=group)
    info = B.info()
    assert info["grid"] >= 1 and info["rows_max"] % 2 == 0
    B.solve()
    torch.cuda.synchronize()
    cache = {}
    for k, ((A, P, f, x), (beam, s, F)) in enumerate(zip(systems, ref)):
        key = (beam.n_e, s)
        if key not in cache:
            Ao = O.shifted_csr(beam, AL, BE, s)
            cache[key] = (Ao, O.spai(Ao))
        Ao, Po = cache[key]
        xd = O.chol_solve(Ao, F)[:, 0]
        x_o, it_o, st_o, _ = O.pcg(Ao, F, [Po], tol=1e-10, maxit=20000)
        xg = x.cpu().numpy()
        assert int(B.status[k]) == G.OK
        assert np.linalg.norm(xg - xd) <= 1e-8 * np.linalg.norm(xd)
        assert abs(int(B.iters[k]) - it_o) <= max(2, it_o // 20)
        true = np.linalg.norm(F - O.spmv(Ao, xg)) / np.linalg.norm(F)
        assert float(B.relres[k]) <= 2e-10
        assert abs(true - float(B.relres[k])) <= 1e-3 * true + 1e-12


def test_batch_graph_replay_and_cost_replan(G):
    systems, ref, keep = make_systems(G, SPEC, seed=8)
    B = G.Batch(systems, rows_per_cta=256)
    B.solve()
    torch.cuda.synchronize()
    x_first = [s[3].clone() for s in systems]
    it_first = B.iters.clone()
    # capture one solve in a CUDA graph and replay it twice
    for s in systems:
        s[3].zero_()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            B.solve(stream=stream)
    for _ in range(2):
        for s in systems:
            s[3].zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(B.iters, it_first)
        for s, x0 in zip(systems, x_first):
            assert torch.equal(s[3], x0)
    # re-plan with measured costs (rows x iterations): same answers
    cost = [float(s[0].n * max(1, int(it))) for s, it in zip(systems, it_first.cpu())]
    for s in systems:
        s[3].zero_()
    B2 = G.Batch(systems, cost=cost, rows_per_cta=512)
    B2.solve()
    torch.cuda.synchronize()
    # another row partition sums in another order: equal to the CG tolerance
    for s, x0 in zip(systems, x_first):
        assert float((s[3] - x0).norm()) <= 1e-8 * float(x0.norm())


@pytest.mark.parametrize("share", [1, 2], ids=["cta_per_sm", "two_lanes"])
def test_batch_groups_sit_on_distinct_sms(G, share):
    """A system's CTA group never puts two of its CTAs on one SM: with one
    CTA per SM trivially, with two lanes (sm_share = 2) because a CTA takes
    its lane from its arrival order on its SM (one CTA of each lane per SM)
    and a group stays within one lane.  rows_per_cta = 64 gives the
    n = 10,002 systems the largest group a lane allows (one CTA per SM).  The
    placement hook records each system's CTA ranks on every solve."""
    systems, ref, keep = make_systems(G, [(5000, [1.0, 20.0], 2), (900, [0.1], 1), (12, [5.0], 1)])
    nsys = len(systems)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    place = torch.full((nsys * 1024,), -1, dtype=torch.int32, device="cuda")
    G.debug_record_placement(place)
    try:
        B = G.Batch(systems, G.options(sm_share=share), rows_per_cta=64)
    finally:
        G.debug_record_placement(None)
    B.solve()
    torch.cuda.synchronize()
    pl = place.view(nsys, 1024).cpu().numpy()
    sizes = []
    for s in range(nsys):
        row = pl[s]
        g = int((row >= 0).sum())
        assert 1 <= g <= sms
        assert np.all(row[:g] >= 0) and np.all(row[:g] < 1024) and np.all(row[g:] == -1)
        assert len(set(row[:g].tolist())) == g, s          # distinct SMs within the group
        assert int(B.status[s]) == G.OK
        sizes.append(g)
    assert max(sizes) == sms                               # the n = 10,002 systems span every SM


def test_batch_rejects(G):
    beam = W.beam(10)
    M, K = G.beam_mats(beam)
    A = G.assemble_shifted(M, K, AL, BE, 1.0)
    P = G.spai_build(A)
    f = torch.ones(beam.n, dtype=torch.float64, device="cuda")
    x = torch.zeros(beam.n, dtype=torch.float64, device="cuda")
    with pytest.raises(G.AirgaError):
        G.Batch([(A, P, f, x), (A, None, f, x)])      # mixed preconditioning


def test_batch_barrier_timeout_is_per_system(G):
    """A host-injected missing arrival in system 0 expires that system's
    bounded barrier waits only: it reports AIRGA_E_TIMEOUT (relres NaN), every
    other system of the launch still solves, and the next solve of the same
    batch is clean."""
    systems, ref, keep = make_systems(G, SPEC)
    B = G.Batch(systems, G.options(tol=1e-10, maxit=20000, barrier_timeout_ms=100))
    G.debug_set_fault(G.FAULT_SKIP_ARRIVAL)
    B.solve()
    torch.cuda.synchronize()
    assert int(B.status[0]) == G.E_TIMEOUT
    assert np.isnan(float(B.relres[0]))
    assert all(int(v) == G.OK for v in B.status[1:])
    assert float(B.relres[1:].max()) <= 2e-10
    B.solve()
    torch.cuda.synchronize()
    assert all(int(v) == G.OK for v in B.status)
