"""Pins of the synthetic beam inputs (Sec. 5 beam model) to closed forms."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as la

from paper_1606_01216_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "cantilever_roots.txt")


def _roots():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    return [(int(k), float(a), float(b)) for k, a, b in rows]


def _dense(b, which):
    A = np.zeros((b.n, b.n))
    rows = np.repeat(np.arange(b.n), np.diff(b.rowptr))
    A[rows, b.col] = b.m_val if which == "m" else b.k_val
    return A


def test_bisection_matches_tabulated_roots():
    for k, r5, r10 in _roots():
        x = W.cantilever_beta_l(k)
        assert abs(x - r10) < 1e-9
        assert abs(x - r5) < 6e-5
        assert abs(1 + math.cos(x) * math.cosh(x)) < 1e-9 * math.cosh(x)


@pytest.mark.parametrize("scaling", ["unit", "literal"])
@pytest.mark.parametrize("n_e", [10, 20, 50])
def test_eigenfrequencies(n_e, scaling):
    """Generalised eigenvalues of (K, M) give omega_k = (beta_k L)^2 / L^2
    (EI = rho A = 1).  The Hermite-cubic FE error in beta_k L falls like h^4:
    bound 2e-4 (k=3, n_e=10) scaled by (10/n_e)^4, with headroom; a floor of
    2e-8 covers the dense eigensolver's own eps * kappa error at n_e = 50."""
    b = W.beam(n_e, scaling)
    L = n_e * b.h
    ev = la.eigh(_dense(b, "k"), _dense(b, "m"), eigvals_only=True)[:3]
    for (k, r5, r10), lam in zip(_roots(), ev):
        bl = math.sqrt(math.sqrt(lam)) * L
        tol = max({1: 1e-6, 2: 3e-5, 3: 3e-4}[k] * (10.0 / n_e) ** 4, 2e-8)
        assert abs(bl - r10) / r10 < tol, (k, bl, r10)
        if n_e >= 20:
            assert abs(bl - r5) / r5 < 5e-5


def test_h4_convergence():
    errs = []
    for n_e in (10, 20):
        b = W.beam(n_e, "unit")
        lam = la.eigh(_dense(b, "k"), _dense(b, "m"), eigvals_only=True)[2]
        errs.append(abs(math.sqrt(math.sqrt(lam)) * n_e - _roots()[2][2]))
    assert 12 < errs[0] / errs[1] < 20   # h halves -> error / 16


def test_structure():
    b = W.beam(7)
    assert b.n == 14 and b.nnz == 7 * b.n - 12
    for A in (_dense(b, "m"), _dense(b, "k")):
        assert np.array_equal(A, A.T)
        assert np.all(np.linalg.eigvalsh(A) > 0)
        i, j = np.nonzero(A)
        assert np.max(np.abs(i - j)) == 3


def test_loads_and_shifts():
    F = W.loads(10, 3, seed=4)
    assert F.flags.f_contiguous and F.shape == (10, 3)
    assert F[8, 0] == 1.0 and np.count_nonzero(F[:, 0]) == 1
    assert np.array_equal(F, W.loads(10, 3, seed=4))
    s = W.log_shifts(-1, 4, 8)
    assert s[0] == pytest.approx(0.1) and s[-1] == pytest.approx(1e4)
    assert np.allclose(np.diff(np.log10(s)), 5 / 7)
    mid = W.midpoint_shifts(-1, 4, 16)
    assert len(mid) == 16 and mid[0] > 0.1 and mid[-1] < 1e4
    batch = W.batched_beams()
    assert len(batch) == 32
    assert all(5000 <= c["n_e"] <= 500000 and 4 <= len(c["shifts"]) <= 16 and c["m"] in (1, 4)
               for c in batch)


# ---------------------------------------------------------------------------
# general sparse inputs (membrane family)
# ---------------------------------------------------------------------------

def test_membrane_matrices_are_spd_and_not_banded():
    w = W.membrane(6, 5, seed=3)
    assert w.n == 6 * 6
    Kd = np.zeros((w.n, w.n))
    Md = np.zeros((w.n, w.n))
    Kd[np.repeat(np.arange(w.n), np.diff(w.k_rowptr)), w.k_col] = w.k_val
    Md[np.repeat(np.arange(w.n), np.diff(w.m_rowptr)), w.m_col] = w.m_val
    assert np.array_equal(Kd, Kd.T) and np.array_equal(Md, Md.T)
    assert np.linalg.eigvalsh(Kd)[0] > 0 and np.linalg.eigvalsh(Md)[0] > 0
    rows = np.repeat(np.arange(w.n), np.diff(w.k_rowptr))
    assert np.abs(w.k_col - rows).max() > 3                    # leaves every narrow band
    assert np.diff(w.k_rowptr).max() <= 9                      # bilinear quads: 9-point rows


def test_membrane_element_sums():
    """Unpermuted grid: each stiffness row of a node away from the clamped
    edge sums to zero (the Laplace operator annihilates constants), and the
    consistent mass of the free nodes plus their coupling to the clamp adds
    up to the element masses (sum of M_e entries = rho_e for a unit square)."""
    w = W.membrane(5, 4, seed=7, permute=False)
    rows = np.repeat(np.arange(w.n), np.diff(w.k_rowptr))
    rsum = np.bincount(rows, weights=w.k_val, minlength=w.n)
    ny1 = 4 + 1
    away = np.arange(w.n) >= ny1                                 # nodes with i >= 2
    assert np.allclose(rsum[away], 0.0, atol=1e-14)
    lumped = W.membrane(5, 4, seed=7, permute=False, lumped_mass=True)
    mrows = np.repeat(np.arange(w.n), np.diff(w.m_rowptr))
    assert np.allclose(lumped.m_val, np.bincount(mrows, weights=w.m_val, minlength=w.n))
    rng = np.random.default_rng(7)                               # unpermuted: E, then rho
    rng.uniform(0.5, 2.0, (5, 4))
    rho = rng.uniform(0.5, 2.0, (5, 4))
    # elements off the clamp keep all four nodes (entries of M_e sum to 1);
    # the clamp-side column keeps nodes 1 and 2 of each element: 12/36 of it
    expected = rho[1:].sum() + rho[0].sum() * 12.0 / 36.0
    assert abs(w.m_val.sum() - expected) <= 1e-13 * expected


def _membrane_by_loops(nx, ny, seed, lumped_mass=False, permute=True):
    """The membrane's assembly written element by element with dense
    accumulation, as a reference for the vectorised generator (small sizes)."""
    rng = np.random.default_rng(seed)
    ke = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    me = np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]]) / 36.0
    n = nx * (ny + 1)
    perm = rng.permutation(n) if permute else np.arange(n)
    E = rng.uniform(0.5, 2.0, (nx, ny))
    rho = rng.uniform(0.5, 2.0, (nx, ny))
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    present = np.zeros((n, n), dtype=bool)
    for ex in range(nx):
        for ey in range(ny):
            corners = [(ex, ey), (ex + 1, ey), (ex + 1, ey + 1), (ex, ey + 1)]
            nodes = [perm[(i - 1) * (ny + 1) + j] if i > 0 else -1 for i, j in corners]
            for a in range(4):
                for b in range(4):
                    if nodes[a] >= 0 and nodes[b] >= 0:
                        K[nodes[a], nodes[b]] += E[ex, ey] * ke[a, b]
                        M[nodes[a], nodes[b]] += rho[ex, ey] * me[a, b]
                        present[nodes[a], nodes[b]] = True
    if lumped_mass:
        M = np.diag(M.sum(axis=1))
    return K, M, present


@pytest.mark.parametrize("args", [(3, 2, 0, False, True), (7, 5, 4, False, True),
                                  (6, 4, 9, True, True), (5, 6, 2, False, False)])
def test_membrane_matches_element_loop(args):
    nx, ny, seed, lumped, permute = args
    w = W.membrane(nx, ny, seed=seed, lumped_mass=lumped, permute=permute)
    K, M, present = _membrane_by_loops(nx, ny, seed, lumped, permute)
    for rowptr, col, val, ref, pat in ((w.k_rowptr, w.k_col, w.k_val, K, present),
                                       (w.m_rowptr, w.m_col, w.m_val, M, np.diag(np.diag(M)) != 0
                                        if lumped else present)):
        rows = np.repeat(np.arange(w.n), np.diff(rowptr))
        got = np.zeros_like(ref)
        got[rows, col] = val
        assert np.allclose(got, ref, rtol=1e-14, atol=1e-15)
        stored = np.zeros_like(pat)
        stored[rows, col] = True
        assert np.array_equal(stored, pat)                      # the pattern, explicit zeros kept
        for r in range(w.n):                                     # sorted, no duplicates
            c = col[rowptr[r]:rowptr[r + 1]]
            assert np.all(np.diff(c) > 0)
