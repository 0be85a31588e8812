"""General sparse (CSR) storage: the CUDA path against the CPU oracle.

Matrices whose entries leave the band |i - j| <= 3 are kept as CSR; the SPAI
pattern S of Eq. 3.1 is an operand.  Inputs are the seeded membrane family of
workloads.membrane (bilinear quadrilaterals, random element coefficients and
node numbering: a 9-point pattern with no band structure), with consistent or
lumped mass.  Tolerances are those of the band parity tests:
  assembly            |a_gpu - a_ora| <= 4 eps (|c_m m| + |c_k k|) per entry
  SpMV                |y_gpu - y_ora| <= 8 eps sum_k |a_ik x_k| per row
  SPAI / update       ||m_gpu - m_ora|| / ||m_ora|| <= 1e-10 per column
  MR mode             equal step counts and 1e-10 columns except columns whose
                      final residual is within 1e-12 of the threshold
  PCG                 ||x_gpu - x_ora|| / ||x_ora|| <= 1e-8, true residual <= 2 tol,
                      iteration counts within max(2, 5 %)
"""
import numpy as np
import pytest

import oracle as O
from paper_1606_01216_gb300 import workloads as W

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps
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


# ---------------------------------------------------------------------------
# helpers (host side, numpy / scipy only)
# ---------------------------------------------------------------------------

def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def upload(G, n, rowptr, col, val):
    return G.mat_from_csr(n, dev(rowptr.astype(np.int64)), dev(col.astype(np.int32)),
                          dev(val.astype(np.float64)))


def mats(G, w):
    M = upload(G, w.n, w.m_rowptr, w.m_col, w.m_val)
    K = upload(G, w.n, w.k_rowptr, w.k_col, w.k_val)
    return M, K


def scipy_of(rowptr, col, val, n):
    return sp.csr_matrix((val, col, rowptr), shape=(n, n))


def ora_of(S):
    S = sp.csr_matrix(S)
    S.sort_indices()
    return O.CSR(S.shape[0], S.indptr, S.indices, S.data)


def stored_pattern(rowptr, col, val, n):
    """Pattern a matrix takes part in the general kernels with: its CSR
    pattern, or, when every entry lies in |i - j| <= 3 (band storage), the
    pattern of its nonzero entries."""
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    if col.size == 0 or np.abs(col.astype(np.int64) - rows).max() <= 3:
        nz = val != 0
        return sp.csr_matrix((np.ones(int(nz.sum())), (rows[nz], col[nz])), shape=(n, n))
    return scipy_of(rowptr, col, np.ones(col.size), n)


def ora_shifted(w, s):
    """A(s) on the union pattern of M and K, by the oracle's entrywise formula
    (M and K read as 0 where they store nothing)."""
    M = scipy_of(w.m_rowptr, w.m_col, w.m_val, w.n)
    K = scipy_of(w.k_rowptr, w.k_col, w.k_val, w.n)
    pm = stored_pattern(w.m_rowptr, w.m_col, w.m_val, w.n)
    pk = stored_pattern(w.k_rowptr, w.k_col, w.k_val, w.n)
    U = (pm + pk).tocsr()
    U.sort_indices()
    r = np.repeat(np.arange(w.n), np.diff(U.indptr))
    mu = np.asarray(M[r, U.indices]).ravel()
    ku = np.asarray(K[r, U.indices]).ravel()
    return O.CSR(w.n, U.indptr, U.indices, O.shifted(mu, ku, AL, BE, s)), mu, ku


def gpu_csr(G, A):
    rp, ci, va = G.mat_to_csr(A)
    return rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy()


def factor_scipy(G, P, k):
    rp, ci, va = G.precond_factor_csr(P, k)
    n = P.n
    return scipy_of(rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy(), n)


def column_errors(Fg, Fo: O.CSR):
    """max_j ||f_gpu(:,j) - f_ora(:,j)|| / ||f_ora(:,j)||, plus the pattern check."""
    Fo_s = scipy_of(Fo.rowptr, Fo.col, Fo.val, Fo.n)
    D = (Fg - Fo_s).tocsc()
    num = np.sqrt(np.asarray(D.multiply(D).sum(axis=0)).ravel())
    den = np.sqrt(np.asarray(Fo_s.multiply(Fo_s).sum(axis=0)).ravel())
    return num / np.where(den > 0, den, 1.0)


def pattern_cols(S):
    """Oracle form of a pattern given by its columns: the CSR of S^T."""
    T = sp.csr_matrix(S.T)
    T.sort_indices()
    return O.CSR(T.shape[0], T.indptr, T.indices, np.ones(T.nnz))


def pattern_handle(G, S):
    S = sp.csr_matrix(S)
    S.sort_indices()
    return upload(G, S.shape[0], S.indptr, S.indices, np.ones(S.nnz))


def run_pcg(G, A, P, F, **kw):
    opts = G.options(**kw)
    Fd = dev(np.ascontiguousarray(np.atleast_2d(F.T)))
    return G.pcg_solve(A, P, Fd.t() if F.ndim == 2 else Fd.reshape(-1), opts, want_hist=True)


# ---------------------------------------------------------------------------
# storage, assembly, SpMV
# ---------------------------------------------------------------------------

def test_csr_import_canonical(G):
    w = W.membrane(12, 9, seed=1)
    n = w.n
    rng = np.random.default_rng(4)
    rows = np.repeat(np.arange(n), np.diff(w.k_rowptr))
    cols, vals = w.k_col.astype(np.int64), w.k_val.copy()
    # split every third entry into two duplicates, then shuffle within rows
    dup = np.flatnonzero(np.arange(cols.size) % 3 == 0)
    first = vals.copy()
    first[dup] = vals[dup] * rng.uniform(0.2, 0.8, dup.size)
    r2 = np.concatenate([rows, rows[dup]])
    c2 = np.concatenate([cols, cols[dup]])
    v2 = np.concatenate([first, vals[dup] - first[dup]])
    order = np.lexsort((rng.permutation(r2.size), r2))
    r2, c2, v2 = r2[order], c2[order], v2[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r2, minlength=n), out=rp[1:])
    A = upload(G, n, rp, c2, v2)
    assert not G.mat_is_banded(A)
    grp, gci, gva = gpu_csr(G, A)
    ref = scipy_of(rp, c2, v2, n)       # scipy sums the two halves of each pair: a + b
    ref.sum_duplicates()
    ref.sort_indices()
    assert np.array_equal(grp, ref.indptr) and np.array_equal(gci, ref.indices)
    assert np.array_equal(gva, ref.data)           # each duplicate pair summed once: exact
    # a banded CSR input keeps the band storage
    beam = W.beam(20)
    B = upload(G, beam.n, beam.rowptr, beam.col, beam.m_val)
    assert G.mat_is_banded(B)
    # malformed inputs
    with pytest.raises(G.AirgaError) as e:
        upload(G, n, rp, np.where(np.arange(c2.size) == 5, n + 3, c2), v2)
    assert e.value.code == G.E_INVALID_ARG
    bad = rp.copy()
    bad[-1] -= 1
    with pytest.raises(G.AirgaError) as e:
        G.mat_from_csr(n, dev(bad), dev(c2.astype(np.int32)), dev(v2))
    assert e.value.code == G.E_INVALID_ARG


@pytest.mark.parametrize("lumped", [False, True], ids=["consistent", "lumped"])
@pytest.mark.parametrize("s", [0.0, 0.3, 17.0, 1e4])
def test_csr_assemble_shifted(G, lumped, s):
    w = W.membrane(23, 17, seed=2, lumped_mass=lumped)
    M, K = mats(G, w)
    A = G.assemble_shifted(M, K, AL, BE, s)
    assert not G.mat_is_banded(A)
    Ao, mu, ku = ora_shifted(w, s)
    rp, ci, va = gpu_csr(G, A)
    assert np.array_equal(rp, Ao.rowptr) and np.array_equal(ci, Ao.col)
    scale = np.abs((s * s + AL * s) * mu) + np.abs((1 + BE * s) * ku)
    assert np.all(np.abs(va - Ao.val) <= 4 * EPS * scale)


def test_csr_assembly_shares_pattern_across_shifts(G):
    w = W.membrane(15, 11, seed=5, lumped_mass=True)
    M, K = mats(G, w)
    A1 = G.assemble_shifted(M, K, AL, BE, 1.0)
    A2 = G.assemble_shifted(M, K, AL, BE, 2.0)
    P1 = G.spai_build(A1)
    # the update requires A_prev and A_next on one pattern: assembled pairs are
    Q = G.spai_update(P1, A1, A2)
    assert len(Q) == 2


@pytest.mark.parametrize("nx,ny", [(9, 7), (61, 40)])
def test_csr_spmv_and_residual(G, nx, ny):
    w = W.membrane(nx, ny, seed=6)
    M, K = mats(G, w)
    A = G.assemble_shifted(M, K, AL, BE, 2.5)
    Ao, _, _ = ora_shifted(w, 2.5)
    X = np.random.default_rng(nx).standard_normal((w.n, 3))
    Xd = dev(X.T.copy()).t()
    Y = G.spmv(A, Xd).cpu().numpy()
    absA = O.CSR(Ao.n, Ao.rowptr, Ao.col, np.abs(Ao.val))
    for c in range(3):
        ref = O.spmv(Ao, X[:, c])
        assert np.all(np.abs(Y[:, c] - ref) <= 8 * EPS * O.spmv(absA, np.abs(X[:, c])) + 1e-300)
    F = np.random.default_rng(1).standard_normal((w.n, 3))
    rr = G.true_residual(A, Xd, dev(F.T.copy()).t()).cpu().numpy()
    for c in range(3):
        ref = np.linalg.norm(F[:, c] - O.spmv(Ao, X[:, c])) / np.linalg.norm(F[:, c])
        assert abs(rr[c] - ref) <= 1e-12 * ref


# ---------------------------------------------------------------------------
# SPAI on a general pattern (Eq. 3.1) and the update (Sec. 3.2), QR mode
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("s", [0.1, 3.0, 1e3])
def test_csr_spai_build_and_update_qr(G, s):
    w = W.membrane(37, 29, seed=7)
    M, K = mats(G, w)
    A0 = G.assemble_shifted(M, K, AL, BE, s / 5.18)
    A1 = G.assemble_shifted(M, K, AL, BE, s)
    Ao0, _, _ = ora_shifted(w, s / 5.18)
    Ao1, _, _ = ora_shifted(w, s)
    P = G.spai_build(A1)
    assert not G.precond_is_banded(P)
    Po, colres_o = O.spai(Ao1, want_colres=True)
    assert column_errors(factor_scipy(G, P, 0), Po).max() <= 1e-10
    steps, colres, st = G.precond_status(P)
    assert st == G.OK and int(steps.abs().max()) == 0
    np.testing.assert_allclose(colres.cpu().numpy(), colres_o, rtol=1e-8, atol=1e-14)
    Q = G.spai_update(G.spai_build(A0), A0, A1)
    Qo = O.spai(Ao1, A_old=Ao0)
    assert column_errors(factor_scipy(G, Q, 1), Qo).max() <= 1e-10


def test_csr_spai_pattern_operand(G):
    """S as an input of Eq. 3.1: a nonsymmetric pattern (the upper triangle of
    A's pattern), the pattern of A^2 (wide blocks: up to 25 unknowns and 49
    rows), and the band pattern of a band-stored handle."""
    w = W.membrane(19, 14, seed=8)
    M, K = mats(G, w)
    A = G.assemble_shifted(M, K, AL, BE, 1.7)
    Ao, _, _ = ora_shifted(w, 1.7)
    As = scipy_of(Ao.rowptr, Ao.col, Ao.val, Ao.n)
    upper = sp.triu(As, format="csr")
    square = (abs(As) @ abs(As)).tocsr()
    for S in (upper, square):
        P = G.spai_build(A, pattern=pattern_handle(G, S))
        Po = O.spai(Ao, pattern=pattern_cols(S))
        assert column_errors(factor_scipy(G, P, 0), Po).max() <= 1e-10
    # a band-stored pattern handle stands for the band |i - j| <= 3
    band = sp.diags([np.ones(w.n - abs(d)) for d in range(-3, 4)], list(range(-3, 4)), format="csr")
    Pb = G.spai_build(A, pattern=upload(G, w.n, band.indptr, band.indices, band.data))
    Pbo = O.spai(Ao, pattern=pattern_cols(band))
    assert column_errors(factor_scipy(G, Pb, 0), Pbo).max() <= 1e-10


def test_csr_pattern_on_band_matrix(G):
    """A band-stored beam matrix with a wider CSR pattern (|i - j| <= 6): the
    general kernels read the band on its full pattern."""
    beam = W.beam(300)
    Mb, Kb = G.beam_mats(beam)
    A = G.assemble_shifted(Mb, Kb, AL, BE, 2.0)
    Ao = O.shifted_csr(beam, AL, BE, 2.0)
    wide = sp.diags([np.ones(beam.n - abs(d)) for d in range(-6, 7)], list(range(-6, 7)),
                    format="csr")
    P = G.spai_build(A, pattern=pattern_handle(G, wide))
    assert not G.precond_is_banded(P)
    Po = O.spai(Ao, pattern=pattern_cols(wide))
    assert column_errors(factor_scipy(G, P, 0), Po).max() <= 1e-10
    F = W.loads(beam.n)[:, 0]
    res = run_pcg(G, A, P, F)
    xo, ito, sto, _ = O.pcg(Ao, F, factors=(Po,), symmetrize=True)
    x = res["X"].cpu().numpy()
    assert int(res["status"][0]) == G.OK and sto == O.OK
    assert abs(int(res["iters"][0]) - ito) <= max(2, ito // 20)
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)


# ---------------------------------------------------------------------------
# MR mode (Algorithms 2 / 4) on a general pattern
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("relative", [False, True], ids=["absolute", "relative"])
def test_csr_spai_mr(G, relative):
    tol, kmax = 0.01, 50
    w = W.membrane(31, 22, seed=9)
    M, K = mats(G, w)
    A0 = G.assemble_shifted(M, K, AL, BE, 0.9)
    A1 = G.assemble_shifted(M, K, AL, BE, 2.0)
    Ao0, _, _ = ora_shifted(w, 0.9)
    Ao1, _, _ = ora_shifted(w, 2.0)
    opts = G.options(spai_mode=G.SPAI_MR, mr_tol=tol, mr_kmax=kmax, mr_relative=int(relative))
    n = w.n
    A0s = scipy_of(Ao0.rowptr, Ao0.col, Ao0.val, n)
    cnorm = np.sqrt(np.asarray(A0s.multiply(A0s).sum(axis=0)).ravel())
    cases = [(G.spai_build(A1, opts), 0, None, np.full(n, tol)),
             (G.spai_update(G.spai_build(A0, opts), A0, A1, opts), 1, Ao0,
              tol * cnorm if relative else np.full(n, tol))]
    for P, k, A_old, thr in cases:
        Fo, steps_o, res_o, _ = O.spai_mr(Ao1, tol=tol, kmax=kmax, A_old=A_old, relative=relative)
        steps, colres, _ = G.precond_status(P)
        steps, colres = steps.cpu().numpy(), colres.cpu().numpy()
        near = (np.abs(res_o - thr) <= 1e-12 * thr) | (np.abs(colres - thr) <= 1e-12 * thr)
        ok = ~near
        assert np.array_equal(steps[ok], steps_o[ok])
        err = column_errors(factor_scipy(G, P, k), Fo)
        assert err[ok].max() <= 1e-10
        np.testing.assert_allclose(colres[ok], res_o[ok], rtol=1e-9, atol=1e-14)


# ---------------------------------------------------------------------------
# PCG
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("s", [0.1, 1.0, 100.0])
def test_csr_pcg_matches_oracle(G, s):
    w = W.membrane(43, 31, seed=10, lumped_mass=(s == 1.0))
    M, K = mats(G, w)
    A = G.assemble_shifted(M, K, AL, BE, s)
    Ao, _, _ = ora_shifted(w, s)
    P = G.spai_build(A)
    Po = O.spai(Ao)
    F = np.asfortranarray(np.random.default_rng(11).standard_normal((w.n, 2)))
    res = run_pcg(G, A, P, F)
    X = res["X"].t().cpu().numpy() if res["X"].dim() == 2 else res["X"].cpu().numpy()[None]
    H = res["res_hist"]
    Xd = np.linalg.solve(scipy_of(Ao.rowptr, Ao.col, Ao.val, w.n).toarray(), F)
    for c in range(2):
        xo, ito, sto, ho = O.pcg(Ao, F[:, c], factors=(Po,), symmetrize=True)
        assert sto == O.OK and int(res["status"][c]) == G.OK
        it = int(res["iters"][c])
        assert abs(it - ito) <= max(2, ito // 20)
        assert np.linalg.norm(X[c] - xo) <= 1e-8 * np.linalg.norm(xo)
        assert np.linalg.norm(X[c] - Xd[:, c]) <= 1e-8 * np.linalg.norm(Xd[:, c])
        assert float(res["true_relres"][c]) <= 2e-10
        h = H[c].cpu().numpy() if H.dim() == 2 else H.cpu().numpy()
        k = min(6, it, ito)
        np.testing.assert_allclose(h[:k + 1], ho[:k + 1], rtol=1e-8)


def test_csr_pcg_update_chain_and_apply(G):
    w = W.membrane(29, 21, seed=12)
    M, K = mats(G, w)
    shifts = (1.0, 1.6, 2.5)
    As = [G.assemble_shifted(M, K, AL, BE, s) for s in shifts]
    Aos = [ora_shifted(w, s)[0] for s in shifts]
    P = G.spai_build(As[0])
    for k in (1, 2):
        P = G.spai_update(P, As[k - 1], As[k])
    assert len(P) == 3
    facs = (O.spai(Aos[0]), O.spai(Aos[1], A_old=Aos[0]), O.spai(Aos[2], A_old=Aos[1]))
    for k in range(3):
        assert column_errors(factor_scipy(G, P, k), facs[k]).max() <= 1e-10
    # chain apply: z = 1/2 (C + C^T) r and z = C r against dense products
    r = np.random.default_rng(13).standard_normal(w.n)
    Cd = np.eye(w.n)
    for f in facs:
        Cd = f.dense() @ Cd
    for sym in (True, False):
        z = G.precond_apply(P, dev(r), symmetrize=sym).cpu().numpy()
        ref = 0.5 * (Cd @ r + Cd.T @ r) if sym else Cd @ r
        assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)
    F = np.random.default_rng(14).standard_normal(w.n)
    res = run_pcg(G, As[2], P, F)
    xo, ito, sto, _ = O.pcg(Aos[2], F, factors=facs, symmetrize=True)
    x = res["X"].cpu().numpy()
    assert int(res["status"][0]) == G.OK and sto == O.OK
    assert abs(int(res["iters"][0]) - ito) <= max(2, ito // 20)
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
    assert float(res["true_relres"][0]) <= 2e-10


def test_csr_precond_export_import(G):
    w = W.membrane(17, 13, seed=15)
    M, K = mats(G, w)
    A = G.assemble_shifted(M, K, AL, BE, 0.7)
    P = G.spai_build(A)
    P2 = G.precond_from_csr(w.n, [G.precond_factor_csr(P, 0)])
    F = np.random.default_rng(16).standard_normal(w.n)
    r1, r2 = run_pcg(G, A, P, F), run_pcg(G, A, P2, F)
    assert torch.equal(r1["X"], r2["X"]) and int(r1["iters"][0]) == int(r2["iters"][0])


def test_csr_edge_cases(G):
    # smallest non-banded matrix: n = 5 with a corner coupling
    n = 5
    D = np.diag([4.0, 5.0, 6.0, 5.0, 4.0]) + np.diag(np.full(4, -1.0), 1) + np.diag(np.full(4, -1.0), -1)
    D[0, 4] = D[4, 0] = 0.5
    S = sp.csr_matrix(D)
    A = upload(G, n, S.indptr, S.indices, S.data)
    assert not G.mat_is_banded(A)
    Ao = ora_of(S)
    P = G.spai_build(A)
    assert column_errors(factor_scipy(G, P, 0), O.spai(Ao)).max() <= 1e-10
    b = np.arange(1.0, 6.0)
    res = run_pcg(G, A, P, b)
    assert int(res["status"][0]) == G.OK
    assert np.allclose(res["X"].cpu().numpy(), np.linalg.solve(D, b), rtol=1e-9)
    # zero right-hand side: x = 0, no iteration
    z = run_pcg(G, A, P, np.zeros(n))
    assert int(z["iters"][0]) == 0 and int(z["status"][0]) == G.OK
    assert float(z["true_relres"][0]) == 0.0 and not z["X"].abs().max().item()
    # warm start from the solution: no iteration needed
    opts = G.options(warm_start=1)
    X = res["X"].clone()
    out = G.pcg_solve(A, P, dev(b), opts, X=X)
    assert int(out["iters"][0]) <= 1 and int(out["status"][0]) == G.OK


def test_csr_barrier_timeout_reports_status(G):
    w = W.membrane(21, 15, seed=17)
    M, K = mats(G, w)
    A = G.assemble_shifted(M, K, AL, BE, 1.0)
    P = G.spai_build(A)
    F = np.random.default_rng(18).standard_normal(w.n)
    G.debug_set_fault(G.FAULT_SKIP_ARRIVAL)
    res = run_pcg(G, A, P, F, barrier_timeout_ms=100)
    assert int(res["status"][0]) == G.E_TIMEOUT
    res = run_pcg(G, A, P, F)
    assert int(res["status"][0]) == G.OK


def test_csr_band_only_calls_refuse(G):
    w = W.membrane(9, 8, seed=19)
    M, K = mats(G, w)
    A = G.assemble_shifted(M, K, AL, BE, 1.0)
    P = G.spai_build(A)
    F = dev(np.ones(w.n))
    with pytest.raises(G.AirgaError) as e:
        G.pcg_solve_mixed(A, P, F)
    assert e.value.code == G.E_UNSUPPORTED
    with pytest.raises(G.AirgaError) as e:
        G.mat_to_band(A)
    assert e.value.code == G.E_UNSUPPORTED
    with pytest.raises(G.AirgaError) as e:
        G.precond_factor(P, 0)
    assert e.value.code == G.E_UNSUPPORTED


def test_csr_full_size(G):
    """n = 490,700 (a 700 x 700 membrane): every SPAI column against the
    oracle, then PCG against the oracle's PCG."""
    w = W.membrane(700, 700, seed=20)
    M, K = mats(G, w)
    A = G.assemble_shifted(M, K, AL, BE, 1.0)
    Ao, _, _ = ora_shifted(w, 1.0)
    P = G.spai_build(A)
    Po = O.spai(Ao)
    assert column_errors(factor_scipy(G, P, 0), Po).max() <= 1e-10
    F = np.random.default_rng(21).standard_normal(w.n)
    res = run_pcg(G, A, P, F)
    xo, ito, sto, _ = O.pcg(Ao, F, factors=(Po,), symmetrize=True)
    x = res["X"].cpu().numpy()
    assert int(res["status"][0]) == G.OK and sto == O.OK
    assert abs(int(res["iters"][0]) - ito) <= max(2, ito // 20)
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
    assert float(res["true_relres"][0]) <= 2e-10
