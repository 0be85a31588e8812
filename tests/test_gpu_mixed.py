"""FP32-inner / FP64-refinement solve (airga_pcg_solve_mixed) against the
FP64 oracle.  The refinement stops on the FP64 true residual, so the same
targets as the plain FP64 PCG apply: X within 1e-8 relative of the oracle's
direct solution, ||f - A x|| / ||f|| <= tol = 1e-10."""
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


def solve(G, beam, s, F, precond=True, **kw):
    M, K = G.beam_mats(beam)
    A = G.assemble_shifted(M, K, AL, BE, s)
    P = G.spai_build(A) if precond else None
    Fd = torch.from_numpy(np.ascontiguousarray(np.atleast_2d(F.T))).cuda()
    res = G.pcg_solve_mixed(A, P, Fd.t() if F.ndim == 2 else Fd.reshape(-1), G.options(**kw))
    torch.cuda.synchronize()
    return res


@pytest.mark.parametrize("s", [0.1, 1.0, 13.9, 100.0, 1e4])
def test_mixed_matches_fp64_oracle(G, s):
    beam = W.beam(1237)
    F = W.loads(beam.n)[:, 0]
    res = solve(G, beam, s, F)
    Ao = O.shifted_csr(beam, AL, BE, s)
    xd = O.chol_solve(Ao, F)[:, 0]
    x = res["X"].cpu().numpy()
    assert int(res["status"][0]) == G.OK
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    true = np.linalg.norm(F - O.spmv(Ao, x)) / np.linalg.norm(F)
    assert true <= 1e-10 and float(res["true_relres"][0]) <= 1e-10
    # both residuals are evaluated in FP64 with different summation orders;
    # near 1e-13 they agree only up to that evaluation noise
    assert abs(true - float(res["true_relres"][0])) <= 1e-3 * true + 1e-11
    assert int(res["outer_iters"][0]) >= 1 and int(res["inner_iters"][0]) >= int(res["outer_iters"][0])


def test_mixed_multi_rhs_and_identity(G):
    beam = W.beam(2000)
    F = W.loads(beam.n, 3, seed=9)
    Ao = O.shifted_csr(beam, AL, BE, 50.0)
    Xd = O.chol_solve(Ao, F)
    for pre in (True, False):
        res = solve(G, beam, 50.0, F, precond=pre)
        X = res["X"].cpu().numpy()
        for c in range(3):
            assert int(res["status"][c]) == G.OK
            assert np.linalg.norm(X[:, c] - Xd[:, c]) <= 1e-8 * np.linalg.norm(Xd[:, c])


def test_mixed_outer_cap(G):
    beam = W.beam(1500)
    F = W.loads(beam.n)[:, 0]
    res = solve(G, beam, 0.1, F, max_outer=1, inner_tol=1e-2)
    assert int(res["status"][0]) == G.E_MAXIT and int(res["outer_iters"][0]) == 1
    assert 1e-10 < float(res["true_relres"][0]) < 1.0


def test_mixed_zero_rhs(G):
    beam = W.beam(300)
    res = solve(G, beam, 1.0, np.zeros(beam.n))
    assert int(res["status"][0]) == G.OK and int(res["outer_iters"][0]) == 0
    assert not res["X"].any()


@pytest.mark.parametrize("s", [0.1, 1e4])
def test_mixed_full_size_two_million(G, s):
    """The precision workload's size: 1,000,000 elements (n = 2e6)."""
    beam = W.beam(1_000_000)
    F = W.loads(beam.n, 2, seed=4)
    res = solve(G, beam, s, F)
    Ao = O.shifted_csr(beam, AL, BE, s)
    Xd = O.chol_solve(Ao, F)
    X = res["X"].cpu().numpy()
    for c in range(2):
        assert int(res["status"][c]) == G.OK
        assert np.linalg.norm(X[:, c] - Xd[:, c]) <= 1e-8 * np.linalg.norm(Xd[:, c])
        assert float(res["true_relres"][c]) <= 1e-10


def test_mixed_barrier_timeout_reports_status(G):
    """A CTA that never arrives at the first inner barrier (host-injected)
    makes every bounded wait expire: the column ends with AIRGA_E_TIMEOUT,
    x keeps its last refined value (here 0), later columns and later calls
    solve normally."""
    beam = W.beam(5000)
    F = W.loads(beam.n, 2, seed=3)
    G.debug_set_fault(G.FAULT_SKIP_ARRIVAL)
    res = solve(G, beam, 1.0, F, barrier_timeout_ms=100)
    assert int(res["status"][0]) == G.E_TIMEOUT
    assert not res["X"][:, 0].any()
    assert int(res["status"][1]) == G.OK
    assert float(res["true_relres"][1]) <= 1e-10
    res = solve(G, beam, 1.0, F)
    assert all(int(v) == G.OK for v in res["status"])


def _psym_band(band, n):
    """(P + P^T) / 2 of a band-7 factor, in the same band layout."""
    B = band.reshape(7, n)
    S = np.zeros_like(B)
    for d in range(-3, 4):
        i = np.arange(max(0, -d), min(n, n - d))
        S[d + 3, i] = 0.5 * (B[d + 3, i] + B[3 - d, i + d])
    return S.reshape(-1)


def test_mixed_symmetric_read_is_bit_identical_to_full_band(G):
    """The FP32 copy of P_sym keeps only its upper diagonals and reads the
    lower entries from earlier rows, summing in the band order.  The same
    matrix handed over as a plain band factor (symmetrize = 0, full 7-diagonal
    FP32 copy) must give the same solve bit for bit."""
    beam = W.beam(1237)
    M, K = G.beam_mats(beam)
    A = G.assemble_shifted(M, K, AL, BE, 0.5)
    P = G.spai_build(A)
    S = _psym_band(G.precond_factor(P, 0).cpu().numpy(), beam.n)
    P2 = G.precond_from_bands([torch.from_numpy(S).cuda()])
    F = torch.from_numpy(W.loads(beam.n)[:, 0]).cuda()
    r1 = G.pcg_solve_mixed(A, P, F, G.options())
    r2 = G.pcg_solve_mixed(A, P2, F, G.options(symmetrize=0))
    torch.cuda.synchronize()
    assert int(r1["status"][0]) == G.OK and int(r2["status"][0]) == G.OK
    assert int(r1["inner_iters"][0]) == int(r2["inner_iters"][0])
    assert torch.equal(r1["X"], r2["X"])
