"""SPAI by the normal equations (spai_mode AIRGA_SPAI_NE) against the CPU
oracle's Householder solve of the same least-squares problems (Eq. 3.1,
Sec. 3.2).

The normal equations give the same minimiser; only rounding differs.  The
bars are those of the QR parity tests:
  factor columns   max_j ||m_gpu - m_ora|| / ||m_ora|| <= 1e-10
  column residual  ||b_j - A m_j|| within rtol 1e-8 of the oracle's
Columns whose Gram block is ill-conditioned go to the Householder kernel
(steps[j] = 1); on the unit-element beam none do, and a beam with two
columns scaled by 1e-3 sends exactly the 8 columns whose pattern holds them.
"""
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


def column_errors(band_gpu, F_ora):
    """max_j ||f_gpu(:,j) - f_ora(:,j)|| / ||f_ora(:,j)|| over the band."""
    n = F_ora.n
    Fg = np.zeros((n, n))
    b = band_gpu.reshape(7, n)
    for d in range(-3, 4):
        i = np.arange(max(0, -d), min(n, n - d))
        Fg[i, i + d] = b[d + 3, i]
    Fo = F_ora.dense()
    num = np.linalg.norm(Fg - Fo, axis=0)
    den = np.linalg.norm(Fo, axis=0)
    return num / np.where(den > 0, den, 1.0)


def band_of(D):
    n = D.shape[0]
    band = np.zeros((7, n))
    for d in range(-3, 4):
        i = np.arange(max(0, -d), min(n, n - d))
        band[d + 3, i] = D[i, i + d]
    return band


def ne(G):
    return G.options(spai_mode=G.SPAI_NE)


@pytest.mark.parametrize("n_e", [7, 8, 9, 35, 500, 1237])
@pytest.mark.parametrize("s", [0.1, 2.6827, 13.895, 1e4])
def test_ne_build_matches_householder_oracle(G, n_e, s):
    beam = W.beam(n_e)
    M, K = G.beam_mats(beam)
    A = G.assemble_shifted(M, K, AL, BE, s)
    P = G.spai_build(A, ne(G))
    Ao = O.shifted_csr(beam, AL, BE, s)
    Po, colres_o = O.spai(Ao, want_colres=True)
    err = column_errors(G.precond_factor(P, 0).cpu().numpy(), Po)
    assert err.max() <= 1e-10, err.max()
    steps, colres, st = G.precond_status(P)
    assert st == G.OK
    assert int(steps.abs().max()) == 0               # no column needed the Householder pass
    np.testing.assert_allclose(colres.cpu().numpy(), colres_o, rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("n_e", [9, 300])
@pytest.mark.parametrize("shifts", [(2.0, 7.0), (372.76, 1930.7), (1930.7, 1e4)])
def test_ne_update_matches_householder_oracle(G, n_e, shifts):
    # update residuals are 1e-6 .. 1e-3 of ||b_j|| at the large shifts: the
    # column residual is formed explicitly, not as ||b||^2 - g.m
    beam = W.beam(n_e)
    M, K = G.beam_mats(beam)
    s0, s1 = shifts
    A0 = G.assemble_shifted(M, K, AL, BE, s0)
    A1 = G.assemble_shifted(M, K, AL, BE, s1)
    P1 = G.spai_update(G.spai_build(A0, ne(G)), A0, A1, ne(G))
    Ao0, Ao1 = O.shifted_csr(beam, AL, BE, s0), O.shifted_csr(beam, AL, BE, s1)
    Qo, colres_o = O.spai(Ao1, A_old=Ao0, want_colres=True)
    err = column_errors(G.precond_factor(P1, 1).cpu().numpy(), Qo)
    assert err.max() <= 1e-10, err.max()
    steps, colres, st = G.precond_status(P1)
    assert st == G.OK and int(steps.abs().max()) == 0
    np.testing.assert_allclose(colres.cpu().numpy(), colres_o, rtol=1e-8, atol=1e-14)


def test_ne_ill_conditioned_columns_take_householder(G):
    """Columns 40 and 41 of a beam scaled by 1e-3: every Gram block that holds
    them has a pivot below 1e-6 of its largest diagonal entry, so columns
    37..44 (J_j within 3 of them) are solved by the Householder kernel and
    marked; all columns match the oracle."""
    beam = W.beam(200)
    D = O.shifted_csr(beam, AL, BE, 1.0).dense()
    D[:, 40:42] *= 1e-3
    n = beam.n
    A = G.mat_from_band(torch.from_numpy(band_of(D).ravel()).cuda())
    rp, ci = W.band_pattern(n, 3)
    Ao = O.dense_to_csr(D, O.CSR(n, rp, ci, np.ones(ci.size)))
    P = G.spai_build(A, ne(G))
    Po, colres_o = O.spai(Ao, want_colres=True)
    assert column_errors(G.precond_factor(P, 0).cpu().numpy(), Po).max() <= 1e-10
    steps, colres, st = G.precond_status(P)
    assert st == G.OK
    assert np.flatnonzero(steps.cpu().numpy()).tolist() == list(range(37, 45))
    np.testing.assert_allclose(colres.cpu().numpy(), colres_o, rtol=1e-8, atol=1e-14)


def test_ne_random_band_and_pcg(G):
    # nonsymmetric random diagonally dominant band (odd n), then a PCG with
    # the NE factor reaches the tolerance like the QR factor does
    rng = np.random.default_rng(23)
    n = 777
    D = np.zeros((n, n))
    for d in range(-3, 4):
        i = np.arange(max(0, -d), min(n, n - d))
        D[i, i + d] = rng.uniform(-1, 1, i.size)
    D = D + np.diag(12.0 + rng.uniform(0, 1, n))
    A = G.mat_from_band(torch.from_numpy(band_of(D).ravel()).cuda())
    rp, ci = W.band_pattern(n, 3)
    Ao = O.dense_to_csr(D, O.CSR(n, rp, ci, np.ones(ci.size)))
    P = G.spai_build(A, ne(G))
    assert column_errors(G.precond_factor(P, 0).cpu().numpy(), O.spai(Ao)).max() <= 1e-10
    beam = W.beam(2000)
    M, K = G.beam_mats(beam)
    As = G.assemble_shifted(M, K, AL, BE, 0.5)
    F = torch.from_numpy(np.ascontiguousarray(W.loads(beam.n)[:, 0])).cuda()
    r_ne = G.pcg_solve(As, G.spai_build(As, ne(G)), F)
    r_qr = G.pcg_solve(As, G.spai_build(As), F)
    assert int(r_ne["status"][0]) == G.OK
    it_qr = int(r_qr["iters"][0])                    # the parity tests' iteration bar
    assert abs(int(r_ne["iters"][0]) - it_qr) <= max(2, it_qr // 20)
    assert float(r_ne["true_relres"][0]) <= 2e-10
    Fo = W.loads(beam.n)[:, :1]
    xd = O.chol_solve(O.shifted_csr(beam, AL, BE, 0.5), Fo)[:, 0]
    assert np.linalg.norm(r_ne["X"].cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)


def test_ne_narrow_patterns_fall_back_to_qr(G):
    # the NE solver is for half-width 3 on band storage; narrower patterns
    # run the Householder solver: the same factor as spai_mode QR, bit for bit
    beam = W.beam(300)
    M, K = G.beam_mats(beam)
    A = G.assemble_shifted(M, K, AL, BE, 3.0)
    for hbw in (1, 2):
        a = G.precond_factor(G.spai_build(A, G.options(spai_mode=G.SPAI_NE, pattern_hbw=hbw)), 0)
        b = G.precond_factor(G.spai_build(A, G.options(pattern_hbw=hbw)), 0)
        assert torch.equal(a, b)


def test_ne_without_column_residuals(G):
    """want_colres = 0 skips only the residual pass: the factor is the same
    bit for bit, the NE columns' residual entries read NaN and the columns
    the Householder kernel took keep theirs."""
    beam = W.beam(200)
    D = O.shifted_csr(beam, AL, BE, 1.0).dense()
    D[:, 40:42] *= 1e-3                              # columns 37..44 take the Householder pass
    A = G.mat_from_band(torch.from_numpy(band_of(D).ravel()).cuda())
    P1 = G.spai_build(A, G.options(spai_mode=G.SPAI_NE))
    P0 = G.spai_build(A, G.options(spai_mode=G.SPAI_NE, want_colres=0))
    assert torch.equal(G.precond_factor(P0, 0), G.precond_factor(P1, 0))
    r = torch.from_numpy(np.random.default_rng(5).standard_normal(beam.n)).cuda()
    assert torch.equal(G.precond_apply(P0, r), G.precond_apply(P1, r))      # P_sym r
    c0, c1 = G.precond_status(P0)[1].cpu().numpy(), G.precond_status(P1)[1].cpu().numpy()
    fb = np.zeros(c0.size, dtype=bool)
    fb[37:45] = True
    assert np.all(np.isnan(c0[~fb]))
    assert np.array_equal(c0[fb], c1[fb])
    # the Householder solver keeps its by-product residuals either way
    Pq = G.spai_build(A, G.options(want_colres=0))
    assert not np.any(np.isnan(G.precond_status(Pq)[1].cpu().numpy()))


@pytest.mark.parametrize("s", [0.1, 4.0, 1e4])
def test_ne_update_same_matrix_is_identity(G, s):
    """Sec. 3.2 with A_prev = A_next: the update's least-squares problem is
    solved exactly by Q = I.  Through the normal equations m = G^{-1} G e_c,
    so the error is the Gram block's rounding (cond(G) <= 4.6e5 on the beam)."""
    beam = W.beam(300)
    M, K = G.beam_mats(beam)
    A = G.assemble_shifted(M, K, AL, BE, s)
    Q = G.precond_factor(G.spai_update(G.spai_build(A, ne(G)), A, A, ne(G)), 1).cpu().numpy()
    Q = Q.reshape(7, -1)
    assert np.abs(Q[3] - 1.0).max() <= 1e-9
    assert np.abs(np.delete(Q, 3, axis=0)).max() <= 1e-9
