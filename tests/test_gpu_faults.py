"""Failure detection without a GPU fault: host-side injection of a failed
device allocation and of a failed kernel launch.

Each injected failure must come back as a clean status code from the call
that met it (AIRGA_E_OOM for the allocation, AIRGA_E_CUDA for the launch),
release everything that call had allocated (the library pool's bytes in use
are unchanged after a synchronise), and leave later calls working: the
same solve afterwards gives the same result, bit for bit, as before.
"""
import numpy as np
import pytest

from paper_1606_01216_gb300 import workloads as W

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
    yield airga
    airga.debug_set_fault(airga.FAULT_NONE)


def _problem(G, storage):
    if storage == "band":
        beam = W.beam(3000)
        M, K = G.beam_mats(beam)
        n = beam.n
    else:
        w = W.membrane(60, 50, seed=31)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        M = G.mat_from_csr(w.n, dev(w.m_rowptr), dev(w.m_col), dev(w.m_val))
        K = G.mat_from_csr(w.n, dev(w.k_rowptr), dev(w.k_col), dev(w.k_val))
        n = w.n
    A = G.assemble_shifted(M, K, W.ALPHA, W.BETA, 2.0)
    F = torch.from_numpy(np.random.default_rng(5).standard_normal(n)).cuda()
    return A, F


def _used(G):
    torch.cuda.synchronize()
    return G.debug_pool_used()


@pytest.mark.parametrize("storage", ["band", "csr"])
@pytest.mark.parametrize("fault", ["alloc", "launch"])
def test_injected_failure_is_clean(G, storage, fault):
    A, F = _problem(G, storage)
    P = G.spai_build(A)
    ref = G.pcg_solve(A, P, F)
    torch.cuda.synchronize()
    code = G.E_OOM if fault == "alloc" else G.E_CUDA
    kind = G.FAULT_ALLOC if fault == "alloc" else G.FAULT_LAUNCH
    base = _used(G)
    # a SPAI build that meets the fault
    G.debug_set_fault(kind)
    with pytest.raises(G.AirgaError) as e:
        G.spai_build(A)
    assert e.value.code == code, str(e.value)
    assert _used(G) == base
    # a PCG solve that meets the fault
    G.debug_set_fault(kind)
    with pytest.raises(G.AirgaError) as e:
        G.pcg_solve(A, P, F)
    assert e.value.code == code, str(e.value)
    assert _used(G) == base
    # the fault was consumed: the same calls work and give the same result
    P2 = G.spai_build(A)
    out = G.pcg_solve(A, P2, F)
    torch.cuda.synchronize()
    assert int(out["status"][0]) == G.OK
    assert torch.equal(out["X"], ref["X"])


def test_unknown_fault_rejected(G):
    with pytest.raises(G.AirgaError) as e:
        G.debug_set_fault(99)
    assert e.value.code == G.E_INVALID_ARG
