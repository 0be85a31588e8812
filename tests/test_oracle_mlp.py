"""Pins of the learned-SPAI oracle (oracle/mlp.py) against closed forms,
finite differences and an independent rounding construction.  CPU only."""
import math

import numpy as np
import pytest

from oracle import mlp as om
from paper_1606_01216_gb300 import workloads as W


def _rand_band(n, seed, spd=True):
    rng = np.random.default_rng(seed)
    b = np.zeros((7, n))
    for d in range(-3, 4):
        i = np.arange(max(0, -d), min(n, n - d))
        b[d + 3, i] = rng.uniform(-1, 1, i.size)
    if spd:   # symmetric, diagonally dominant
        for d in range(1, 4):
            i = np.arange(0, n - d)
            b[3 - d, i + d] = b[3 + d, i]
        b[3] = 8.0 + rng.uniform(0, 1, n)
    return b


def test_sizes():
    assert om.NPARAM == W.MLP_NPARAM == 6288
    p = np.arange(om.NPARAM, dtype=np.float64)
    assert np.array_equal(om.pack(om.unpack(p)), p)
    assert om.unpack(p)["W2"][1, 0] == 1024 + 64 + 64


def test_bf16_rounding():
    # independent construction: 8 significant bits by frexp + round-half-even
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.uniform(-6, 6, 2000),
                        [1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, 1.0]])
    x = x.astype(np.float32).astype(np.float64)
    m, e = np.frexp(x)
    ref = np.ldexp(np.round(m * 256.0) / 256.0, e)
    assert np.array_equal(om.bf16(x), ref)
    assert om.bf16(np.array([1 + 2 ** -8]))[0] == 1.0            # tie -> even
    assert om.bf16(np.array([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6  # tie -> even (up)


def test_gradient_finite_differences():
    p = W.mlp_random_params(11).astype(np.float64)
    X, T, mask = W.mlp_random_samples(12, 40)
    L0, g = om.loss_grad(p, X, T, mask, emulate_bf16=False)
    rng = np.random.default_rng(5)
    idx = []
    for name, (o, s) in om.OFFSETS.items():
        size = int(np.prod(s))
        idx += list(o + rng.choice(size, min(size, 12), replace=False))
    for k in idx:
        h = 1e-6 * max(1.0, abs(p[k]))
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (om.loss_grad(pp, X, T, mask, False)[0] - om.loss_grad(pm, X, T, mask, False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_gradient_closed_form_zero_weights():
    p = W.mlp_random_params(21).astype(np.float64)
    d = om.unpack(p)
    d["W1"][:] = 0
    d["W2"][:] = 0
    d["W3"][:] = 0
    p = om.pack(d)
    X, T, mask = W.mlp_random_samples(22, 30)
    M = om.mask_matrix(mask)[:, :7]
    e = (d["b3"][None, :7] - T[:, :7]) * M          # y = b3 exactly
    L, g = om.loss_grad(p, X, T, mask, emulate_bf16=False)
    gd = om.unpack(g)
    assert L == pytest.approx(0.5 * (e ** 2).sum() / 30, rel=1e-14)
    assert np.allclose(gd["b3"][:7], e.sum(0) / 30, rtol=1e-13, atol=0)
    assert np.allclose(gd["W3"][:7], np.outer(e.sum(0) / 30, np.maximum(d["b2"], 0)), rtol=1e-12, atol=1e-15)
    for k in ("W1", "b1", "W2", "b2"):
        assert not gd[k].any()
    assert not gd["W3"][7:].any() and not gd["b3"][7:].any()


def test_emulated_gradient_close_to_exact():
    p = W.mlp_random_params(31).astype(np.float64)
    X, T, mask = W.mlp_random_samples(32, 200)
    _, ge = om.loss_grad(p, X, T, mask, emulate_bf16=True)
    _, gx = om.loss_grad(p, X, T, mask, emulate_bf16=False)
    assert np.linalg.norm(ge - gx) <= 2e-2 * np.linalg.norm(gx)
    assert np.linalg.norm(ge - gx) > 0


def test_adam_closed_forms():
    rng = np.random.default_rng(41)
    p0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    g[0] = 0.0
    lr, eps = 1e-3, 1e-8
    p1, m, v = om.adam(p0, np.zeros(50), np.zeros(50), g, 1, lr, eps=eps)
    # bias correction makes step 1 exactly lr * g / (|g| + eps)
    assert np.allclose(p0 - p1, lr * g / (np.abs(g) + eps), rtol=1e-9, atol=0)
    # a constant gradient keeps mhat = g, vhat = g^2 at every step
    p = p1
    for t in range(2, 7):
        pn, m, v = om.adam(p, m, v, g, t, lr, eps=eps)
        assert np.allclose(p - pn, lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-18)
        p = pn
    assert om.cosine_lr(2.0, 0, 100) == 2.0 and om.cosine_lr(2.0, 100, 100) == pytest.approx(0.0)
    assert om.cosine_lr(2.0, 50, 100) == pytest.approx(1.0) and om.cosine_lr(2.0, 7, 0) == 2.0


def test_features_hand_computed():
    # tridiagonal 4x4: diag 4, 9, 16, 25; off-diagonal A(i, i+1) = A(i+1, i) = 2
    n = 4
    b = np.zeros((7, n))
    b[3] = [4.0, 9.0, 16.0, 25.0]
    b[4, :3] = 2.0
    b[2, 1:] = 2.0
    X = om.features(b, 100.0, 0.1, 1e-4)
    assert X[0, 0] == pytest.approx(0.5) and X[0, 1] == 0.1 and X[0, 2] == 1e-4
    assert X[1, 3] == pytest.approx(math.log10(9.0) / 8)
    # column 1: A(0,1) / sqrt(4*9) at d = -1 (slot 6), A(2,1) / sqrt(16*9) at d = +1 (slot 7)
    assert X[1, 6] == pytest.approx(2 / 6) and X[1, 7] == pytest.approx(2 / 12)
    assert X[1, 4] == 0 and X[1, 5] == 0 and X[1, 8] == 0
    assert X[0, 10] == 0 and X[3, 11] == 0 and X[2, 10] == pytest.approx(2 / 8)
    assert list(X[:, 12]) == [0, 1, 0, 1]
    assert not X[:, 13:].any()


def test_targets_decode_round_trip_and_masks():
    n = 37
    A = _rand_band(n, 51)
    P = _rand_band(n, 52, spd=False)
    T, mask = om.targets(A, P)
    assert mask[0] == 0b1111000 and mask[n - 1] == 0b0001111 and mask[10] == 127
    assert not T[:, 7].any()
    Y = np.zeros((n, 16))
    Y[:, :8] = T
    assert np.allclose(om.decode(A, Y), P, rtol=1e-14, atol=0)
    # subset of columns gives the same rows
    cols = np.array([0, 5, 36])
    T2, m2 = om.targets(A, P, cols)
    assert np.array_equal(T2, T[cols]) and np.array_equal(m2, mask[cols])
    assert np.array_equal(om.features(A, 3.0, 0.1, 1e-4, cols), om.features(A, 3.0, 0.1, 1e-4)[cols])


def test_scale_invariance(ora):
    # SPAI of cA is P/c (Eq. 3.1 is homogeneous): features move only in the
    # log-diagonal slot and the scaled targets do not move at all
    beam = W.beam(20)
    A = ora.shifted_csr(beam, W.ALPHA, W.BETA, 3.0)
    from oracle import CSR
    c = 7.5
    Ac = CSR(A.n, A.rowptr, A.col, c * A.val)
    bA = _band(A)
    bAc = _band(Ac)
    P = _band(ora.spai(A))
    Pc = _band(ora.spai(Ac))
    assert np.allclose(Pc, P / c, rtol=1e-10, atol=1e-14)
    X, Xc = om.features(bA, 3.0, 0.1, 1e-4), om.features(bAc, 3.0, 0.1, 1e-4)
    assert np.allclose(Xc[:, 3] - X[:, 3], math.log10(c) / 8, rtol=0, atol=1e-14)
    keep = [k for k in range(16) if k != 3]
    assert np.allclose(Xc[:, keep], X[:, keep], rtol=1e-13, atol=1e-15)
    assert np.allclose(om.targets(bAc, Pc)[0], om.targets(bA, P)[0], rtol=1e-9, atol=1e-12)


def test_learned_spai_jacobi_closed_form():
    # W3 = 0 and b3 = e_3 make the network output the unit diagonal target,
    # i.e. P(j, j) = 1 / A_jj (Jacobi), whatever the features
    p = W.mlp_random_params(61).astype(np.float64)
    d = om.unpack(p)
    d["W3"][:] = 0
    d["b3"][:] = 0
    d["b3"][3] = 1.0
    A = _rand_band(25, 62)
    for emu in (False, True):
        P = om.learned_spai(om.pack(d), A, 10.0, 0.1, 1e-4, emulate_bf16=emu)
        assert np.allclose(P[3], 1.0 / A[3], rtol=1e-15)
        assert not np.delete(P, 3, axis=0).any()


def _band(csr):
    n = csr.n
    b = np.zeros((7, n))
    rows = np.repeat(np.arange(n), np.diff(csr.rowptr))
    b[csr.col - rows + 3, rows] = csr.val
    return b
