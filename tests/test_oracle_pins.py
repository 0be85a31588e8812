"""Pins of the CPU oracle to things other than itself.

Each test checks an oracle routine against a closed form, a library routine
(numpy/scipy LAPACK), a special case with a known answer, or an invariant the
mathematics fixes.  Chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import numpy as np
import pytest
import scipy.linalg as la

from paper_1606_01216_gb300 import workloads as W

AL, BE = W.ALPHA, W.BETA


def _beamA(ora, n_e, s, scaling="unit", al=AL, be=BE):
    b = W.beam(n_e, scaling)
    return b, ora.shifted_csr(b, al, be, s)


def _dense(ora, b, which):
    return ora.from_beam(b, which).dense()


# ---------------------------------------------------------------------------
# shifted coefficient matrix, Eq. (1.1) / Sec. 3.1
# ---------------------------------------------------------------------------

def test_shifted_special_values(ora):
    b = W.beam(6)
    M, K = _dense(ora, b, "m"), _dense(ora, b, "k")
    # s = 0 gives K exactly, whatever the damping
    assert np.array_equal(ora.shifted_csr(b, 0.7, 0.3, 0.0).dense(), K)
    # undamped: s^2 M + K
    A = ora.shifted_csr(b, 0.0, 0.0, 3.0).dense()
    assert np.allclose(A, 9.0 * M + K, rtol=1e-15, atol=0)


def test_shifted_matches_first_moment(ora):
    """X(s) = A(s)^{-1} F; the paper's first moment (Sec. 2) is
    X^(1)(s0) = -A(s0)^{-1} (2 s0 M + D) X^(0)(s0) = dX/ds.  A central finite
    difference of direct solves of the oracle's A(s) must reproduce it (this
    pins the s-dependence: a wrong power of s or a missing damping term
    breaks it)."""
    b = W.beam(8)
    M, K = _dense(ora, b, "m"), _dense(ora, b, "k")
    D = AL * M + BE * K
    F = W.loads(b.n)[:, 0]
    s0, h = 2.0, 1e-5
    X = lambda s: np.linalg.solve(ora.shifted_csr(b, AL, BE, s).dense(), F)
    x0 = X(s0)
    dX = (X(s0 + h) - X(s0 - h)) / (2 * h)
    A0 = ora.shifted_csr(b, AL, BE, s0).dense()
    x1 = -np.linalg.solve(A0, (2 * s0 * M + D) @ x0)
    assert np.linalg.norm(dX - x1) <= 1e-7 * np.linalg.norm(x1)


def test_shifted_is_quadratic_in_s(ora):
    b = W.beam(5)
    M = _dense(ora, b, "m")
    A = lambda s: ora.shifted_csr(b, AL, BE, s).dense()
    second = A(3.0) - 2 * A(2.0) + A(1.0)          # = 2 M for a quadratic
    assert np.allclose(second, 2 * M, rtol=1e-10, atol=1e-12 * np.abs(M).max())


# ---------------------------------------------------------------------------
# sparse mat-vec
# ---------------------------------------------------------------------------

def test_spmv_against_dense(ora):
    b, A = _beamA(ora, 9, 1.3)
    x = np.random.default_rng(0).standard_normal(A.n)
    assert np.allclose(ora.spmv(A, x), A.dense() @ x, rtol=1e-14, atol=1e-14)
    assert np.allclose(ora.spmv_t(A, x), A.dense().T @ x, rtol=1e-14, atol=1e-14)
    R = ora.CSR(3, [0, 1, 2, 3], [2, 0, 1], [1.0, 2.0, 3.0])   # nonsymmetric
    assert np.array_equal(ora.spmv(R, [1.0, 2.0, 3.0]), [3.0, 2.0, 6.0])
    assert np.array_equal(ora.spmv_t(R, [1.0, 2.0, 3.0]), [4.0, 9.0, 1.0])


# ---------------------------------------------------------------------------
# dense Householder least squares
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(1, 1), (4, 4), (13, 7), (12, 7), (40, 9)])
def test_lsq_qr_against_lapack(ora, shape):
    rng = np.random.default_rng(sum(shape))
    A = rng.standard_normal(shape)
    b = rng.standard_normal(shape[0])
    x, st = ora.lsq_qr(A, b)
    assert st == ora.OK
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.allclose(x, ref, rtol=1e-12, atol=1e-12)


def test_lsq_qr_ill_conditioned_and_rank(ora):
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((13, 7)))
    V, _ = np.linalg.qr(rng.standard_normal((7, 7)))
    A = U @ np.diag(np.logspace(0, -8, 7)) @ V.T
    b = rng.standard_normal(13)
    x, st = ora.lsq_qr(A, b)
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert st == ora.OK
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref)   # kappa 1e8
    A[:, 3] = A[:, 1]
    assert ora.lsq_qr(A, b)[1] == ora.ERANK


def test_lsq_qr_exact_system(ora):
    A = np.array([[2.0, 1.0], [1.0, 3.0], [0.0, 0.0]])
    x, st = ora.lsq_qr(A, np.array([3.0, 5.0, 0.0]))
    assert np.allclose(x, [0.8, 1.4], rtol=1e-15)


# ---------------------------------------------------------------------------
# SPAI (Eq. 3.1) and SPAI update (Sec. 3.2), exact LS on a fixed pattern
# ---------------------------------------------------------------------------

def test_spai_full_pattern_is_inverse(ora):
    """n = 4 (two elements): the band-7 pattern covers the whole matrix, so
    min ||I - A P||_F over it is attained at P = A^{-1}."""
    b, A = _beamA(ora, 2, 0.7)
    P = ora.spai(A).dense()
    assert np.allclose(P, np.linalg.inv(A.dense()), rtol=1e-11, atol=1e-13)


def test_update_full_pattern(ora):
    """Full pattern: min ||A_old - A_new Q||_F is attained at Q = A_new^{-1} A_old."""
    b = W.beam(2)
    Ao, An = ora.shifted_csr(b, AL, BE, 0.7), ora.shifted_csr(b, AL, BE, 1.9)
    Q = ora.spai(An, A_old=Ao).dense()
    ref = np.linalg.solve(An.dense(), Ao.dense())
    assert np.allclose(Q, ref, rtol=1e-11, atol=1e-12)


def test_update_same_matrix_is_identity(ora):
    b, A = _beamA(ora, 40, 5.0)
    Q = ora.spai(A, A_old=A).dense()
    assert np.allclose(Q, np.eye(A.n), rtol=0, atol=1e-12)


def test_spai_diagonal_pattern_closed_form(ora):
    """Pattern = diagonal: m_j = A_jj / ||A(:, j)||^2 (one-variable LS)."""
    b, A = _beamA(ora, 30, 2.0)
    I = ora.CSR(A.n, np.arange(A.n + 1), np.arange(A.n), np.ones(A.n))
    P = ora.spai(A, pattern=I).dense()
    Ad = A.dense()
    ref = np.diag(Ad) / np.sum(Ad * Ad, axis=0)
    assert np.allclose(np.diag(P), ref, rtol=1e-14)
    assert np.count_nonzero(P - np.diag(np.diag(P))) == 0


@pytest.mark.parametrize("s", [0.1, 3.0, 1e3])
def test_spai_columns_against_lstsq(ora, s):
    """Brute force: every column of P (and of an update Q) against LAPACK
    lstsq on the full n-row problem restricted to the column's band."""
    b, A = _beamA(ora, 25, s)
    Ad = A.dense()
    Ao = ora.shifted_csr(b, AL, BE, s * 0.5)
    P = ora.spai(A).dense()
    Q = ora.spai(A, A_old=Ao).dense()
    Aod = Ao.dense()
    n = A.n
    for j in range(n):
        J = np.arange(max(0, j - 3), min(n, j + 4))
        e = np.zeros(n); e[j] = 1
        ref = np.linalg.lstsq(Ad[:, J], e, rcond=None)[0]
        assert np.linalg.norm(P[J, j] - ref) <= 1e-11 * np.linalg.norm(ref)
        refq = np.linalg.lstsq(Ad[:, J], Aod[:, j], rcond=None)[0]
        assert np.linalg.norm(Q[J, j] - refq) <= 1e-11 * np.linalg.norm(refq)
        outside = np.setdiff1d(np.arange(n), J)
        assert np.all(P[outside, j] == 0) and np.all(Q[outside, j] == 0)


def test_spai_normal_equations_invariant(ora):
    """First-order optimality of each column LS: A(:,J)^T (e_j - A m_j) = 0."""
    b, A = _beamA(ora, 400, 0.5)
    P = ora.spai(A)
    n = A.n
    R = np.eye(n) - A.dense() @ P.dense()
    G = A.dense().T @ R
    for j in range(0, n, 37):
        J = np.arange(max(0, j - 3), min(n, j + 4))
        assert np.abs(G[J, j]).max() <= 1e-11 * max(1.0, np.abs(A.dense()).max())


def test_spai_colres_is_frobenius_split(ora):
    """Eq. (3.1): ||I - A P||_F^2 = sum_j ||e_j - A p_j||^2."""
    b, A = _beamA(ora, 60, 1.0)
    P, colres = ora.spai(A, want_colres=True)
    fro = np.linalg.norm(np.eye(A.n) - A.dense() @ P.dense(), "fro")
    assert abs(fro ** 2 - np.sum(colres ** 2)) <= 1e-12 * fro ** 2


# ---------------------------------------------------------------------------
# MR iteration (Algorithms 2 and 4) — pinned only through limits
# ---------------------------------------------------------------------------

def test_alpha_formulas(ora):
    b, A = _beamA(ora, 10, 1.0)
    c = 3.5
    I = ora.CSR(4, np.arange(5), np.arange(4), np.full(4, c))
    assert ora.alpha_build(I) == pytest.approx(1.0 / c, rel=1e-15)
    assert ora.alpha_update(A, A) == pytest.approx(1.0, rel=1e-15)
    A2 = ora.CSR(A.n, A.rowptr, A.col, 2.0 * A.val)
    assert ora.alpha_update(A, A2) == pytest.approx(0.5, rel=1e-15)
    # alpha minimises ||A_old - alpha A_new||_F over alpha
    Ao = ora.shifted_csr(b, AL, BE, 0.8)
    a = ora.alpha_update(Ao, A)
    f = lambda t: np.linalg.norm(Ao.dense() - t * A.dense())
    assert f(a) <= min(f(a * (1 + 1e-6)), f(a * (1 - 1e-6)))
    Ad = A.dense()
    assert ora.alpha_build(A) == pytest.approx(np.trace(Ad) / np.trace(Ad @ Ad.T), rel=1e-13)


def test_mr_identity_and_same_matrix(ora):
    n = 12
    I = ora.CSR(n, np.arange(n + 1), np.arange(n), np.ones(n))
    P, steps, res, a0 = ora.spai_mr(I)
    assert np.array_equal(P.dense(), np.eye(n)) and np.all(steps == 0)
    b, A = _beamA(ora, 20, 2.0)
    Q, steps, res, a0 = ora.spai_mr(A, A_old=A)
    assert a0 == pytest.approx(1.0) and np.all(steps == 0)
    assert np.allclose(Q.dense(), np.eye(A.n), atol=1e-15)


def test_mr_diagonal_pattern_one_step_is_exact(ora):
    """Pattern = diagonal: d = r_j e_j spans the whole search space, so one MR
    step lands on the LS minimiser A_jj / ||A(:, j)||^2."""
    b, A = _beamA(ora, 15, 2.0)
    D = ora.CSR(A.n, np.arange(A.n + 1), np.arange(A.n), np.ones(A.n))
    P, steps, res, a0 = ora.spai_mr(A, tol=1e-14, kmax=1, pattern=D)
    Ad = A.dense()
    ref = np.diag(Ad) / np.sum(Ad * Ad, axis=0)
    assert np.all(steps == 1)
    assert np.allclose(np.diag(P.dense()), ref, rtol=1e-13)


def test_mr_residual_monotone_and_bounded_by_ls(ora):
    """Each MR step minimises ||r - a w|| over a, so the final column
    residual never exceeds the initial one, and no pattern-restricted
    iterate can beat the exact LS minimum."""
    b, A = _beamA(ora, 30, 1.0)
    _, colres_ls = ora.spai(A, want_colres=True)
    a0 = ora.alpha_build(A)
    Ad = A.dense()
    r0 = np.linalg.norm(np.eye(A.n) - a0 * Ad, axis=0)
    for k in (1, 3, 10):
        P, steps, res, _ = ora.spai_mr(A, tol=0.01, kmax=k)
        assert np.all(res <= r0 * (1 + 1e-12))
        assert np.all(res >= colres_ls * (1 - 1e-9))
        true = np.linalg.norm(np.eye(A.n) - Ad @ P.dense(), axis=0)
        assert np.allclose(true, res, rtol=1e-9)


def _mr_threshold(ora, A, A_old, tol, relative):
    """tol (Algorithms 2/4 as written) or tol ||b_j|| per column."""
    n = A.n
    B = A_old.dense() if A_old is not None else np.eye(n)
    return tol * np.linalg.norm(B, axis=0) if relative else np.full(n, tol)


@pytest.mark.parametrize("update,relative,tol", [(False, False, 0.5), (False, True, 0.5),
                                                 (True, False, 0.02), (True, True, 0.003)])
def test_mr_stop_test_is_the_first_crossing(ora, update, relative, tol):
    """Algorithms 2 and 4 loop while ||r|| > tol.  A column's step count must
    therefore be the first k at which its residual reaches the threshold:
    the final residual is at or below it (unless the cap kmax ended the
    column), and rerunning with kmax = steps - 1 leaves the residual above
    it.  Checked against thresholds computed here from the definition (tol,
    or tol ||b_j|| for the relative reading), not from the oracle."""
    b, A = _beamA(ora, 30, 1.0)
    A_old = ora.shifted_csr(b, AL, BE, 0.8) if update else None
    kmax = 50
    thr = _mr_threshold(ora, A, A_old, tol, relative)
    P, steps, res, _ = ora.spai_mr(A, tol=tol, kmax=kmax, A_old=A_old, relative=relative)
    done = steps < kmax
    assert done.any() and (steps > 0).any(), "the case must exercise the stop test"
    assert np.all(res[done] <= thr[done])
    for k in np.unique(steps[(steps > 0)]):
        _, st_k, res_k, _ = ora.spai_mr(A, tol=tol, kmax=int(k) - 1, A_old=A_old,
                                        relative=relative)
        sel = steps == k
        assert np.all(res_k[sel] > thr[sel])


def test_mr_absolute_and_relative_readings(ora):
    """The paper's absolute test ||r|| <= tol and the relative reading
    ||r|| <= tol ||b_j|| agree whenever ||b_j|| = 1, i.e. for every column of
    the build (b_j = e_j): identical steps and entries.  For the update the
    relative reading is invariant under scaling A_old and A_new by a power of
    two (every operation scales exactly in FP64), while the absolute one is
    not: scaled residuals cross a fixed tol later."""
    b, A = _beamA(ora, 30, 1.0)
    Ao = ora.shifted_csr(b, AL, BE, 0.8)
    P1, s1, r1, _ = ora.spai_mr(A, tol=0.5, kmax=50, relative=False)
    P2, s2, r2, _ = ora.spai_mr(A, tol=0.5, kmax=50, relative=True)
    assert np.array_equal(s1, s2) and np.array_equal(P1.val, P2.val) and (s1 < 50).any()
    c = 2.0 ** 10
    As = ora.CSR(A.n, A.rowptr, A.col, c * A.val)
    Aos = ora.CSR(A.n, Ao.rowptr, Ao.col, c * Ao.val)
    Q1, q1, _, _ = ora.spai_mr(A, tol=0.003, A_old=Ao, relative=True)
    Q2, q2, _, _ = ora.spai_mr(As, tol=0.003, A_old=Aos, relative=True)
    assert np.array_equal(q1, q2) and np.array_equal(Q1.val, Q2.val)
    Q3, q3, _, _ = ora.spai_mr(A, tol=0.02, A_old=Ao, relative=False)
    Q4, q4, _, _ = ora.spai_mr(As, tol=0.02, A_old=Aos, relative=False)
    assert np.all(q4 >= q3) and q4.sum() > q3.sum()


def _random_band(ora, n, seed):
    """Nonsymmetric, diagonally dominant band-7 CSR (structurally symmetric)."""
    rng = np.random.default_rng(seed)
    rp, ci = W.band_pattern(n)
    rows = np.repeat(np.arange(n), np.diff(rp))
    val = rng.uniform(-1.0, 1.0, ci.size)
    val[ci == rows] = 8.0 + rng.uniform(0.0, 1.0, n)
    return ora.CSR(n, rp, ci, val)


@pytest.mark.parametrize("nonsym", [False, True])
@pytest.mark.parametrize("update", [False, True])
def test_mr_steps_are_minimal_residual_along_projected_residual(ora, update, nonsym):
    """Each MR step of Algorithms 2/4 is fixed by two properties that do not
    restate its formula.  The change m_{k+1} - m_k is parallel to Pi_J(r_k),
    the current residual restricted to the column's pattern.  The new
    residual is orthogonal to A Pi_J(r_k), i.e. minimal along that direction.
    Both are checked on every column for the first two steps from
    m_0 = alpha_0 e_j; the right-hand side is e_j (build) or A_old(:, j)
    (update)."""
    if nonsym:       # A != A^T: a transposed operand would break the pins
        A = _random_band(ora, 24, 5)
        A_old = _random_band(ora, 24, 6) if update else None
    else:
        b, A = _beamA(ora, 12, 1.3)
        A_old = ora.shifted_csr(b, AL, BE, 0.9) if update else None
    n = A.n
    Ad = A.dense()
    Bd = A_old.dense() if update else np.eye(n)
    a0 = ora.alpha_update(A_old, A) if update else ora.alpha_build(A)
    iters = [a0 * np.eye(n)]
    for k in (1, 2):
        P, steps, _, a0k = ora.spai_mr(A, tol=0.0, kmax=k, A_old=A_old)
        assert a0k == a0 and np.all(steps == k)
        iters.append(P.dense())
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    mask = np.zeros((n, n), dtype=bool)
    mask[rows, A.col] = True                      # column j's pattern: rows i with A(i, j) stored
    for k in (0, 1):
        R = Bd - Ad @ iters[k]
        D = np.where(mask, R, 0.0)
        W = Ad @ D
        delta = iters[k + 1] - iters[k]
        Rn = Bd - Ad @ iters[k + 1]
        for j in range(n):
            d, dj = D[:, j], delta[:, j]
            a = (dj @ d) / (d @ d)
            assert np.linalg.norm(dj - a * d) <= 1e-12 * np.linalg.norm(dj)
            assert abs(Rn[:, j] @ W[:, j]) <= 1e-10 * np.linalg.norm(Rn[:, j]) * np.linalg.norm(W[:, j])
            assert a * (R[:, j] @ W[:, j]) > 0        # the step decreases the residual


# ---------------------------------------------------------------------------
# PCG and the direct solve
# ---------------------------------------------------------------------------

def test_chol_against_lapack(ora):
    b, A = _beamA(ora, 50, 0.3)
    F = W.loads(A.n, 3, seed=1)
    X = ora.chol_solve(A, F)
    ref = la.solve(A.dense(), F, assume_a="pos")
    assert np.allclose(X, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n_e", [5, 20, 60])
def test_static_closed_form(ora, n_e):
    """s = 0: K x = tip force.  Hermite-cubic elements are nodally exact, so
    w(x) = x^2 (3L - x) / 6 and theta(x) = x (2L - x) / 2 at the nodes (EI = 1,
    unit load).  Checked for the direct solve and for SPAI-preconditioned CG."""
    b = W.beam(n_e)
    A = ora.shifted_csr(b, AL, BE, 0.0)
    F = W.loads(b.n)[:, 0]
    L = n_e * b.h
    xk = b.h * np.arange(1, n_e + 1)
    ref = np.empty(b.n)
    ref[0::2] = xk ** 2 * (3 * L - xk) / 6
    ref[1::2] = xk * (2 * L - xk) / 2
    X = ora.chol_solve(A, F)[:, 0]
    # backward-stable direct solve: forward error within kappa(K) * eps
    bound = np.linalg.cond(A.dense()) * np.finfo(float).eps
    assert np.linalg.norm(X - ref) <= bound * np.linalg.norm(ref)
    P = ora.spai(A)
    x, it, st, hist = ora.pcg(A, F, [P], tol=1e-13, maxit=5000)
    assert st == ora.OK
    assert np.linalg.norm(x - ref) <= 1e-7 * np.linalg.norm(ref)


def test_pcg_exact_preconditioner_one_step(ora):
    b, A = _beamA(ora, 6, 1.0)
    Ainv = np.linalg.inv(A.dense())
    Pinv = ora.dense_to_csr(Ainv, pattern=ora.CSR(A.n, np.arange(0, A.n * A.n + 1, A.n),
                                                   np.tile(np.arange(A.n), A.n),
                                                   np.ones(A.n * A.n)))
    F = W.loads(A.n, 2, seed=3)[:, 1]
    x, it, st, hist = ora.pcg(A, F, [Pinv], tol=1e-12)
    assert st == ora.OK and it == 1
    assert np.allclose(x, Ainv @ F, rtol=1e-12)


def test_pcg_terminates_within_n_and_energy_monotone(ora):
    """Unpreconditioned CG on a small SPD system: exact arithmetic ends in at
    most n steps; the A-norm error decreases at every step."""
    rng = np.random.default_rng(7)
    n = 12
    G = rng.standard_normal((n, n))
    Ad = G @ G.T + n * np.eye(n)
    A = ora.dense_to_csr(Ad)
    F = rng.standard_normal(n)
    xs = np.linalg.solve(Ad, F)
    x, it, st, hist = ora.pcg(A, F, [], tol=1e-13, maxit=n + 2)
    assert st == ora.OK and it <= n
    assert np.allclose(x, xs, rtol=1e-11)
    errs = []
    for k in range(1, it + 1):
        xk = ora.pcg(A, F, [], tol=0.0, maxit=k)[0]
        e = xk - xs
        errs.append(e @ Ad @ e)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:]))


@pytest.mark.parametrize("s", [0.1, 1.0, 100.0, 1e4])
def test_pcg_matches_direct_and_history(ora, s):
    b, A = _beamA(ora, 500, s)
    F = W.loads(A.n)[:, 0]
    P = ora.spai(A)
    x, it, st, hist = ora.pcg(A, F, [P], tol=1e-10, maxit=5000)
    xd = ora.chol_solve(A, F)[:, 0]
    assert st == ora.OK
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    true = np.linalg.norm(F - A.dense() @ x) / np.linalg.norm(F)
    assert hist[-1] <= 1e-10 and true <= 2e-10
    assert hist[0] == pytest.approx(1.0)


def test_pcg_zero_rhs_and_warm_start(ora):
    b, A = _beamA(ora, 20, 1.0)
    x, it, st, hist = ora.pcg(A, np.zeros(A.n), [ora.spai(A)])
    assert st == ora.OK and it == 0 and not np.any(x)
    F = W.loads(A.n)[:, 0]
    xd = ora.chol_solve(A, F)[:, 0]
    x, it, st, hist = ora.pcg(A, F, [ora.spai(A)], x0=xd)
    assert st == ora.OK and it == 0


def test_pcg_chain_symmetrised_is_spd_operator(ora):
    """z = 1/2 (C + C^T) r is symmetric in r for a chain; with one factor it is
    P_sym r.  Checked against dense products."""
    b = W.beam(12)
    A1, A2, A3 = (ora.shifted_csr(b, AL, BE, s) for s in (1.0, 1.5, 2.2))
    P1 = ora.spai(A1)
    Q2 = ora.spai(A2, A_old=A1)
    Q3 = ora.spai(A3, A_old=A2)
    Cd = Q3.dense() @ Q2.dense() @ P1.dense()
    Sym = 0.5 * (Cd + Cd.T)
    F = W.loads(b.n)[:, 0]
    # one PCG step from x0 = 0 with maxit=1 exposes z0 through x1 = a z0
    x1 = ora.pcg(A3, F, [P1, Q2, Q3], tol=0.0, maxit=1)[0]
    z0 = Sym @ F
    a = (F @ z0) / (z0 @ A3.dense() @ z0)
    assert np.allclose(x1, a * z0, rtol=1e-12, atol=1e-15)
