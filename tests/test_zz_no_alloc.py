"""The allocation-free PCG entry point, against the regular one and the oracle.

airga_pcg_solve_noalloc is for callers that cannot let a library allocate
device memory: their own allocator owns the GPU's memory, or their loop cannot
absorb the synchronisation and possible failure of an allocation call.  It
works out of one fixed scratch array that every call shares and that keeps
the previous call's contents, so every case here makes two calls in a row
through the C ABI.  Tolerances are those of the PCG parity tests: X within
1e-8 relative, true residual within 2e-10, iteration counts within
max(2, 5 %).

Cases:
  * two shifts against airga_pcg_solve on the same problem, with the device's
    free memory unchanged by the second call (nothing allocated);
  * a NONSYMMETRIC band M (z = M r applied as given) against the oracle's PCG
    with the same factor and no symmetrisation, at even n (row-pair kernel)
    and odd n (generic kernel), residual histories included;
  * the largest n the scratch accepts, 2^20 (even: the split-state plan);
  * a size above the limit is rejected.

Collected last on purpose: it must pass alone in a fresh process and after
the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1606_01216_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_ROWS = 1 << 20


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_01216_gb300 import build
    build.build()
    from paper_1606_01216_gb300 import airga
    airga.lib()
    return airga


def sym_band(P: torch.Tensor, n: int) -> torch.Tensor:
    """1/2 (P + P^T) on band-7 storage, computed with torch on the device."""
    B = P.reshape(7, n)
    S = torch.zeros_like(B)
    for d in range(-3, 4):
        lo, hi = max(0, -d), min(n, n - d)
        i = torch.arange(lo, hi, device=P.device)
        S[d + 3, i] = 0.5 * (B[d + 3, i] + B[3 - d, i + d])
    return S.reshape(-1).contiguous()


def csr_to_band(A: O.CSR) -> np.ndarray:
    """band[(d+3) n + i] = A(i, i+d) for a CSR matrix inside the band |i-j| <= 3."""
    n = A.n
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    d = A.col - rows
    assert np.all(np.abs(d) <= 3)
    band = np.zeros((7, n))
    band[d + 3, rows] = A.val
    return band.reshape(-1)


def trim(A: O.CSR, n: int) -> O.CSR:
    """Leading n x n principal block of a CSR matrix (SPD stays SPD)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    keep = (rows < n) & (A.col < n)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows[keep], minlength=n), out=rp[1:])
    return O.CSR(n, rp, A.col[keep], A.val[keep])


def noalloc(G, n, A_band, M_band, F, m, opts, X, hist, iters, status, relres):
    L = G.lib()
    p = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    return L.airga_pcg_solve_noalloc(n, p(A_band), p(M_band), p(F), m, C.byref(opts), p(X),
                                     p(hist), p(iters), p(status), p(relres),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_pcg_solve_on_two_calls(G):
    beam = W.beam(60_011)                       # n = 120,022: 152 CTAs, ragged last block
    n = beam.n
    M, K = G.beam_mats(beam)
    F = np.asfortranarray(W.loads(n, 2, seed=17))
    Fd = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()      # (m, n) = column-major n x m
    opts = G.options()
    shifts = (0.518, 13.9)
    refs, bands = [], []
    for s in shifts:
        A = G.assemble_shifted(M, K, W.ALPHA, W.BETA, s)
        P = G.spai_build(A)
        refs.append(G.pcg_solve(A, P, Fd.t(), opts))
        bands.append((G.mat_to_band(A), sym_band(G.precond_factor(P, 0), n)))
    # every buffer exists before the first call, so the free-memory reading
    # after the second call can only move if the entry point allocated
    outs = [dict(X=torch.zeros(2, n, dtype=torch.float64, device="cuda"),
                 iters=torch.zeros(2, dtype=torch.int32, device="cuda"),
                 status=torch.zeros(2, dtype=torch.int32, device="cuda"),
                 relres=torch.zeros(2, dtype=torch.float64, device="cuda")) for _ in shifts]
    free = []
    for (A_band, M_band), o in zip(bands, outs):   # two calls in a row on the shared scratch
        rc = noalloc(G, n, A_band, M_band, Fd, 2, opts, o["X"], None, o["iters"], o["status"],
                     o["relres"])
        assert rc == G.OK, G.last_error()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    assert free[1] == free[0], "device free memory changed across a call: %d -> %d" % tuple(free)
    for ref, o in zip(refs, outs):
        Xr = ref["X"].t().cpu().numpy()
        Xn = o["X"].cpu().numpy()
        for c in range(2):
            assert int(o["status"][c]) == G.OK and int(ref["status"][c]) == G.OK
            # the raw band runs the full 7-point stencil, the handle path the
            # packed beam stencil, so rounding moves the step that crosses tol
            it_ref = int(ref["iters"][c])
            assert abs(int(o["iters"][c]) - it_ref) <= max(2, it_ref // 20)
            assert np.linalg.norm(Xn[c] - Xr[c]) <= 1e-8 * np.linalg.norm(Xr[c])
            assert float(o["relres"][c]) <= 2e-10


def _nonsym_case(beam, n, s, w=0.6):
    """Oracle operands: A(s) trimmed to n rows, and the nonsymmetric band
    M = w P + (1 - w) P^T from the oracle's SPAI P of that matrix."""
    A = trim(O.shifted_csr(beam, W.ALPHA, W.BETA, s), n)
    P = O.spai(A)
    PT = P.transpose()
    assert np.array_equal(P.col, PT.col)         # band pattern: P and P^T share it
    Mo = O.CSR(n, P.rowptr, P.col, w * P.val + (1.0 - w) * PT.val)
    return A, Mo


def _check_against_oracle(G, A, Mo, F, maxit=3000):
    n = A.n
    m = F.shape[1]
    A_band = torch.from_numpy(csr_to_band(A)).cuda()
    M_band = torch.from_numpy(csr_to_band(Mo)).cuda()
    Fd = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
    opts = G.options(maxit=maxit)
    X = torch.zeros(m, n, dtype=torch.float64, device="cuda")
    hist = torch.full((m, maxit + 1), float("nan"), dtype=torch.float64, device="cuda")
    iters = torch.zeros(m, dtype=torch.int32, device="cuda")
    status = torch.zeros(m, dtype=torch.int32, device="cuda")
    relres = torch.zeros(m, dtype=torch.float64, device="cuda")
    rc = noalloc(G, n, A_band, M_band, Fd, m, opts, X, hist, iters, status, relres)
    assert rc == G.OK, G.last_error()
    torch.cuda.synchronize()
    Xn, Hn = X.cpu().numpy(), hist.cpu().numpy()
    for c in range(m):
        xo, ito, sto, ho = O.pcg(A, F[:, c], factors=(Mo,), symmetrize=False, maxit=maxit)
        assert sto == O.OK, "oracle status %d" % sto
        assert int(status[c]) == G.OK, G.status_string(int(status[c]))
        it = int(iters[c])
        assert abs(it - ito) <= max(2, ito // 20), (it, ito)
        # the early residual history fixes the operator: a preconditioner read
        # as its symmetric part would move ||r_1|| by percent, not by rounding
        k = min(8, it, ito)
        np.testing.assert_allclose(Hn[c, :k + 1], ho[:k + 1], rtol=1e-8, atol=0)
        assert np.linalg.norm(Xn[c] - xo) <= 1e-8 * np.linalg.norm(xo)
        assert float(relres[c]) <= 2e-10


@pytest.mark.parametrize("odd", [False, True], ids=["even_n", "odd_n"])
def test_noalloc_nonsymmetric_band_vs_oracle(G, odd):
    beam = W.beam(60_011)
    n = beam.n - (1 if odd else 0)              # odd n runs the generic kernel
    F = W.loads(n, 2, seed=23)
    for s in (13.9, 373.0):                      # two calls in a row
        A, Mo = _nonsym_case(beam, n, s)
        _check_against_oracle(G, A, Mo, F)


def test_noalloc_largest_size(G):
    beam = W.beam(MAX_ROWS // 2)                 # n = 2^20, even: split-state row-pair plan
    n = beam.n
    assert n == MAX_ROWS
    A, Mo = _nonsym_case(beam, n, 13.9)
    F = W.loads(n, 1, seed=29)
    _check_against_oracle(G, A, Mo, F)
    _check_against_oracle(G, A, Mo, F)           # again on the scratch the first call left


def test_noalloc_rejects_oversize(G):
    n = MAX_ROWS + 1
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    i32 = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = noalloc(G, n, dummy, None, dummy, 1, G.options(), dummy, None, i32, i32, dummy)
    assert rc == G.E_INVALID_ARG
    assert "1048576" in G.last_error()
