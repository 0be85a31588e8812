"""Two CG solves side by side (options.sm_share = 2 for the lead, 3 for the
partner): each solve takes half of every SM (the node-pair split-state kernel
at 256 threads), so two solves issued on different streams run concurrently.  Each must still be the
CG solve of its own system: checked against the oracle's direct solve and
iteration count (the parity tests' bars), with the other solve in flight."""
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


def _solve_pair(G, beam, shifts, share):
    M, K = G.beam_mats(beam)
    F = W.loads(beam.n, 2, seed=9)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    out = []
    for s, st, c, sh in zip(shifts, streams, (0, 1), share):
        with torch.cuda.stream(st):
            f = torch.from_numpy(np.ascontiguousarray(F[:, c])).cuda()
            A = G.assemble_shifted(M, K, AL, BE, s, stream=st)
            P = G.spai_build(A, G.options(spai_mode=G.SPAI_NE), stream=st)
            if c == 0:                        # the second stream starts after the lead's
                ready = torch.cuda.Event()    # inputs, then after a short hold
                ready.record(st)
                streams[1].wait_event(ready)
                G.stream_hold(50, streams[1])
            r = G.pcg_solve(A, P, f, G.options(tol=1e-10, maxit=20000, sm_share=sh), stream=st)
            out.append((r, A, P, f))
    torch.cuda.synchronize()
    return out, F


def band_of(D):
    n = D.shape[0]
    band = np.zeros((7, n))
    for d in range(-3, 4):
        i = np.arange(max(0, -d), min(n, n - d))
        band[d + 3, i] = D[i, i + d]
    return band


def test_two_odd_band_solves_share(G):
    """Odd n: the half-SM plan does not apply and the generic kernel runs;
    sm_share = 2 still gives each system's CG solve."""
    n = 4001
    rp, ci = W.band_pattern(n, 3)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    cases = []
    for seed, st, sh in zip((31, 32), streams, (2, 3)):
        opts = G.options(tol=1e-10, maxit=20000, sm_share=sh)
        rng = np.random.default_rng(seed)
        D = np.zeros((n, n))
        for d in range(1, 4):
            i = np.arange(n - d)
            v = rng.uniform(-1, 1, i.size)
            D[i, i + d] = v
            D[i + d, i] = v
        D += np.diag(7.0 + rng.uniform(0, 1, n))
        f = rng.standard_normal(n)
        with torch.cuda.stream(st):
            A = G.mat_from_band(torch.from_numpy(band_of(D).ravel()).cuda(), stream=st)
            P = G.spai_build(A, stream=st)
            r = G.pcg_solve(A, P, torch.from_numpy(f).cuda(), opts, stream=st)
        cases.append((D, f, r, A, P))
    torch.cuda.synchronize()
    for D, f, r, _, _ in cases:
        Ao = O.dense_to_csr(D, O.CSR(n, rp, ci, np.ones(ci.size)))
        xd = O.chol_solve(Ao, f)[:, 0]
        assert int(r["status"][0]) == G.OK
        assert np.linalg.norm(r["X"].cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)


@pytest.mark.parametrize("share", [(2, 3), (3, 3), (2, 2)], ids=["lead+partner", "two partners", "two leads"])
def test_two_solves_share_the_sms(G, share):
    # two leads cannot share an SM (their second launch waits for SMs): still
    # each its own solve
    beam = W.beam(20000)
    shifts = (0.1, 2.6827)
    out, F = _solve_pair(G, beam, shifts, share)
    for (r, _, _, _), s, c in zip(out, shifts, (0, 1)):
        Ao = O.shifted_csr(beam, AL, BE, s)
        xd = O.chol_solve(Ao, F[:, c])[:, 0]
        _, it_o, st_o, _ = O.pcg(Ao, F[:, c], [O.spai(Ao)], tol=1e-10, maxit=20000)
        assert int(r["status"][0]) == G.OK and st_o == O.OK
        assert np.linalg.norm(r["X"].cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
        assert abs(int(r["iters"][0]) - it_o) <= max(2, it_o // 20)
        assert float(r["true_relres"][0]) <= 2e-10


@pytest.mark.parametrize("share", [2, 3])
def test_sm_share_matches_whole_sm_solve(G, share):
    """The same system with sm_share 1 and 2 or 3: the same iteration count
    and solutions equal to the CG tolerance (the half-SM kernel sums its
    reductions over 256-thread blocks, so the rounding order differs)."""
    beam = W.beam(30000)
    M, K = G.beam_mats(beam)
    A = G.assemble_shifted(M, K, AL, BE, 0.5179)
    P = G.spai_build(A)
    f = torch.from_numpy(np.ascontiguousarray(W.loads(beam.n)[:, 0])).cuda()
    r1 = G.pcg_solve(A, P, f, G.options(sm_share=1))
    r2 = G.pcg_solve(A, P, f, G.options(sm_share=share))
    torch.cuda.synchronize()
    assert int(r1["status"][0]) == G.OK and int(r2["status"][0]) == G.OK
    assert abs(int(r1["iters"][0]) - int(r2["iters"][0])) <= 1
    x1, x2 = r1["X"], r2["X"]
    assert float((x1 - x2).norm()) <= 1e-8 * float(x1.norm())


def test_stream_hold(G):
    st = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    G.stream_hold(300, st)
    e1.record(st)
    torch.cuda.synchronize()
    assert 0.3 <= e0.elapsed_time(e1) < 50.0        # ms: at least the hold, and bounded
    G.stream_hold(0, st)                             # nothing queued
    for bad in (-1, 1001):
        with pytest.raises(G.AirgaError):
            G.stream_hold(bad, st)


def test_sm_share_rejects_other_values(G):
    beam = W.beam(10)
    M, K = G.beam_mats(beam)
    A = G.assemble_shifted(M, K, AL, BE, 1.0)
    f = torch.ones(beam.n, dtype=torch.float64, device="cuda")
    for bad in (0, 4):
        with pytest.raises(G.AirgaError):
            G.pcg_solve(A, None, f, G.options(sm_share=bad))


def test_lead_ctas_never_share_an_sm(G):
    """A lead solve (sm_share = 2) reserves just over half an SM's shared
    memory, so no two of its CTAs can sit on one SM: the placement hook must
    show every CTA on its own SM, whatever else runs.  A partner launched
    beside it on another stream still solves its own system."""
    beam = W.beam(500000)                       # n = 1e6: 152 CTAs of 6580 rows
    M, K = G.beam_mats(beam)
    f = torch.from_numpy(np.ascontiguousarray(W.loads(beam.n)[:, 0])).cuda()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    place_a = torch.full((1024,), -1, dtype=torch.int32, device="cuda")
    place_b = torch.full((1024,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(sa):
        Aa = G.assemble_shifted(M, K, AL, BE, 2.6827, stream=sa)
        Pa = G.spai_build(Aa, G.options(spai_mode=G.SPAI_NE), stream=sa)
        ready = torch.cuda.Event()
        ready.record(sa)
        G.debug_record_placement(place_a)
        ra = G.pcg_solve(Aa, Pa, f, G.options(sm_share=2), stream=sa)
    sb.wait_event(ready)
    G.stream_hold(50, sb)
    with torch.cuda.stream(sb):
        Ab = G.assemble_shifted(M, K, AL, BE, 13.895, stream=sb)
        Pb = G.spai_build(Ab, G.options(spai_mode=G.SPAI_NE), stream=sb)
        G.debug_record_placement(place_b)
        rb = G.pcg_solve(Ab, Pb, f, G.options(sm_share=3), stream=sb)
    G.debug_record_placement(None)
    torch.cuda.synchronize()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    pa = place_a.cpu().numpy()
    grid = int((pa >= 0).sum())
    assert 1 <= grid <= sms
    assert np.all(pa[:grid] >= 0) and np.all(pa[:grid] < 1024) and np.all(pa[grid:] == -1)
    assert len(set(pa[:grid].tolist())) == grid          # one lead CTA per SM
    pb = place_b.cpu().numpy()
    assert int((pb >= 0).sum()) == grid
    for r in (ra, rb):
        assert int(r["status"][0]) == G.OK and float(r["true_relres"][0]) <= 2e-10


def _band_from_csr(C):
    """(7, n) band of a CSR factor on the band-7 pattern: band[d + 3, i] = C[i, i + d]."""
    rows = np.repeat(np.arange(C.n), np.diff(C.rowptr))
    band = np.zeros((7, C.n))
    band[C.col - rows + 3, rows] = C.val
    return band


def _band_col_errors(bg, bo):
    """max_j ||f_gpu(:, j) - f_ora(:, j)|| / ||f_ora(:, j)|| on two (7, n) bands."""
    n = bo.shape[1]
    num, den = np.zeros(n), np.zeros(n)
    for d in range(-3, 4):
        i = np.arange(max(0, -d), min(n, n - d))
        num[i + d] += (bg[d + 3, i] - bo[d + 3, i]) ** 2
        den[i + d] += bo[d + 3, i] ** 2
    return np.sqrt(num) / np.where(den > 0, np.sqrt(den), 1.0)


def test_full_size_step_configuration(G):
    """The measured configuration at full size: the n = 1e6 beam, SPAI by the
    normal equations without per-column residuals, the s = 0.1 solve as a
    lead (sm_share = 2) and the s = 0.518 solve as a partner (sm_share = 3)
    on a second stream that starts 50 us after the lead's inputs, both solves
    in flight together.  Every SPAI column against the oracle's Householder
    solve, each solution against the oracle's banded Cholesky solve, each
    iteration count against the oracle's PCG."""
    beam = W.beam(500000)
    M, K = G.beam_mats(beam)
    F = W.loads(beam.n)[:, 0]
    f = torch.from_numpy(np.ascontiguousarray(F)).cuda()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    so = G.options(spai_mode=G.SPAI_NE, want_colres=0)
    torch.cuda.synchronize()
    out = []
    for s, st, share in ((0.1, sa, 2), (0.5179474679231212, sb, 3)):
        with torch.cuda.stream(st):
            A = G.assemble_shifted(M, K, AL, BE, s, stream=st)
            P = G.spai_build(A, so, stream=st)
            if st is sa:
                ready = torch.cuda.Event()
                ready.record(sa)
                sb.wait_event(ready)
                G.stream_hold(50, sb)
            r = G.pcg_solve(A, P, f, G.options(tol=1e-10, maxit=20000, sm_share=share), stream=st)
            out.append((s, A, P, r))
    torch.cuda.synchronize()
    for s, A, P, r in out:
        Ao = O.shifted_csr(beam, AL, BE, s)
        Po = O.spai(Ao)
        err = _band_col_errors(G.precond_factor(P, 0).cpu().numpy().reshape(7, -1),
                               _band_from_csr(Po))
        assert err.max() <= 1e-10, (s, float(err.max()))
        x = r["X"].cpu().numpy().reshape(-1)
        xd = O.chol_solve(Ao, F)[:, 0]
        assert int(r["status"][0]) == G.OK
        assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
        true = np.linalg.norm(F - O.spmv(Ao, x)) / np.linalg.norm(F)
        assert true <= 2e-10
        assert abs(true - float(r["true_relres"][0])) <= 1e-3 * true + 1e-12
        _, it_o, _, _ = O.pcg(Ao, F, [Po], tol=1e-10, maxit=20000)
        assert abs(int(r["iters"][0]) - it_o) <= max(2, it_o // 20), (s, int(r["iters"][0]), it_o)
