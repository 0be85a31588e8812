"""CPU oracle of the learned SPAI-column predictor — TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and bench.py's CPU legs use this module; the
product never imports it.  Plain numpy, FP64.

What it computes (all written from the definitions, no blocking or fusion):

* Training pairs for column j of a shifted matrix A = s^2 M + s D + K
  (Eq. 1.1) and its SPAI P (Sec. 3.1, Eq. 3.1; column j of P is supported on
  J_j = {j-3..j+3}):
    features  x_j = ( log10(s)/4, alpha, beta, log10(A_jj)/8,
                      A(j+d, j) / sqrt(A(j+d, j+d) A_jj)  for d = -3,-2,-1,1,2,3
                      (0 where j+d is outside the matrix),
                      min(j, 8)/8, min(n-1-j, 8)/8, j mod 2, 0, 0, 0 )
    targets   t_j[o] = P(j+d, j) sqrt(A(j+d, j+d) A_jj),  d = o - 3, o = 0..6
    mask      bit o set when 0 <= j+d < n.
  The symmetric diagonal scaling makes the targets O(1) at every shift and is
  undone exactly by `decode`.
* A three-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3,
  relu(z) = max(z, 0) (16 -> 64 -> 64 -> 16; outputs 7..15 unused), and the loss
  L = 1/(2B) sum_samples sum_{o in mask} (y_o - t_o)^2 with its gradient by
  the chain rule (back-propagation).
* The Adam update of Kingma and Ba (ICLR 2015, Algorithm 1) with bias
  correction.
* The learned SPAI: features of A, forward pass, `decode` to a band-7 P.

Two arithmetic modes.  emulate_bf16=False is the exact FP64 function and its
exact gradient (pinned by finite differences).  emulate_bf16=True applies the
rounding the tensor-core kernels apply — every GEMM operand (inputs, weights,
hidden activations, output errors, hidden deltas) rounded to bfloat16 with
round-to-nearest-even, products accumulated exactly (FP64 here, FP32 on the
GPU), biases and activations in full precision — so GPU results can be
compared tightly.  relu'(0) is taken as 0.

Parameter vector layout (FP32 on the GPU, 6288 values):
  W1[64][16] | b1[64] | W2[64][64] | b2[64] | W3[16][64] | b3[16]
with W[out][in] row-major.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT, N_USED = 16, 64, 16, 7
OFFSETS = {}
_o = 0
for _name, _shape in (("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)),
                      ("b2", (N_HID,)), ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))):
    OFFSETS[_name] = (_o, _shape)
    _o += int(np.prod(_shape))
NPARAM = _o   # 6288
DIST_CAP = 8


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    assert p.size == NPARAM
    return {k: p[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in OFFSETS.items()}


def pack(d):
    out = np.zeros(NPARAM)
    for k, (o, s) in OFFSETS.items():
        out[o:o + int(np.prod(s))] = np.asarray(d[k], dtype=np.float64).ravel()
    return out


def bf16(x):
    """Round to bfloat16 (8 significant bits, round to nearest, ties to even)
    after rounding to FP32; returned as float64 holding the exact value."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# training pairs from (A, P) bands; band[(d+3), i] = A(i, i+d)
# ---------------------------------------------------------------------------

def _entry(band, i, d):
    """A(i, i+d) for index arrays i (all in range)."""
    return band[d + 3, i]


def features(band_A, s, alpha, beta, cols=None):
    """Feature rows (FP64) for columns `cols` (default all) of A."""
    band_A = np.asarray(band_A, dtype=np.float64)
    n = band_A.shape[1]
    j = np.arange(n) if cols is None else np.asarray(cols, dtype=np.int64)
    diag = band_A[3]
    X = np.zeros((j.size, N_IN))
    X[:, 0] = np.log10(s) / 4.0
    X[:, 1] = alpha
    X[:, 2] = beta
    X[:, 3] = np.log10(diag[j]) / 8.0
    for c, d in enumerate((-3, -2, -1, 1, 2, 3)):
        ok = (j + d >= 0) & (j + d < n)
        i = j[ok] + d                       # row of the entry A(j+d, j)
        X[ok, 4 + c] = _entry(band_A, i, -d) / np.sqrt(diag[i] * diag[j[ok]])
    X[:, 10] = np.minimum(j, DIST_CAP) / DIST_CAP
    X[:, 11] = np.minimum(n - 1 - j, DIST_CAP) / DIST_CAP
    X[:, 12] = j % 2
    return X


def targets(band_A, band_P, cols=None):
    """Scaled SPAI column entries T[N, 8] (slot 7 = 0) and mask bytes."""
    band_A = np.asarray(band_A, dtype=np.float64)
    band_P = np.asarray(band_P, dtype=np.float64)
    n = band_A.shape[1]
    j = np.arange(n) if cols is None else np.asarray(cols, dtype=np.int64)
    diag = band_A[3]
    T = np.zeros((j.size, 8))
    mask = np.zeros(j.size, dtype=np.uint8)
    for o in range(N_USED):
        d = o - 3
        ok = (j + d >= 0) & (j + d < n)
        i = j[ok] + d
        T[ok, o] = _entry(band_P, i, -d) * np.sqrt(diag[i] * diag[j[ok]])
        mask[ok] |= np.uint8(1 << o)
    return T, mask


def decode(band_A, Y):
    """Band-7 P from network outputs Y[n, >=7] for every column of A."""
    band_A = np.asarray(band_A, dtype=np.float64)
    n = band_A.shape[1]
    j = np.arange(n)
    diag = band_A[3]
    P = np.zeros((7, n))
    for o in range(N_USED):
        d = o - 3
        ok = (j + d >= 0) & (j + d < n)
        i = j[ok] + d
        P[-d + 3, i] = Y[ok, o] / np.sqrt(diag[i] * diag[j[ok]])
    return P


# ---------------------------------------------------------------------------
# the network
# ---------------------------------------------------------------------------

def forward(params, X, emulate_bf16=True):
    """Outputs y[N, 16] and the intermediate values needed by backward."""
    p = unpack(params)
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Xq = r(X)
    W1, W2, W3 = r(p["W1"]), r(p["W2"]), r(p["W3"])
    z1 = Xq @ W1.T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    H1 = r(h1)
    z2 = H1 @ W2.T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    H2 = r(h2)
    y = H2 @ W3.T + p["b3"]
    return y, dict(Xq=Xq, W1=W1, W2=W2, W3=W3, z1=z1, H1=H1, z2=z2, H2=H2)


def mask_matrix(mask, cols=N_OUT):
    m = np.asarray(mask, dtype=np.uint8)
    M = np.zeros((m.size, cols))
    for o in range(N_USED):
        M[:, o] = (m >> o) & 1
    return M


def loss_grad(params, X, T, mask, emulate_bf16=True):
    """Loss L = 1/(2B) sum masked (y - t)^2 and dL/dparams (vector, NPARAM)."""
    X = np.asarray(X, dtype=np.float64)
    B = X.shape[0]
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, c = forward(params, X, emulate_bf16)
    Tm = np.zeros((B, N_OUT))
    Tm[:, :8] = np.asarray(T, dtype=np.float64)[:, :8]
    e = (y - Tm) * mask_matrix(mask)
    loss = 0.5 * float((e * e).sum()) / B
    E = r(e)
    dz2 = (E @ c["W3"]) * (c["z2"] > 0.0)          # relu'(z) = 1 for z > 0, else 0
    Dz2 = r(dz2)
    dz1 = (Dz2 @ c["W2"]) * (c["z1"] > 0.0)
    Dz1 = r(dz1)
    g = dict(W3=E.T @ c["H2"], b3=E.sum(0), W2=Dz2.T @ c["H1"], b2=Dz2.sum(0),
             W1=Dz1.T @ c["Xq"], b1=Dz1.sum(0))
    return loss, pack(g) / B


def adam(params, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, Algorithm 1) at step number t >= 1."""
    m = beta1 * np.asarray(m) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return np.asarray(params) - lr * mhat / (np.sqrt(vhat) + eps), m, v


def cosine_lr(lr, t, total):
    """Learning rate of step t (1-based) under a half-cosine decay over
    `total` steps (total <= 0: constant)."""
    if total <= 0:
        return lr
    return lr * 0.5 * (1.0 + np.cos(np.pi * min(t, total) / total))


def learned_spai(params, band_A, s, alpha, beta, emulate_bf16=True):
    """Band-7 P predicted by the network for every column of A."""
    X = features(band_A, s, alpha, beta)
    if emulate_bf16:
        X = X.astype(np.float32).astype(np.float64)   # features are stored in FP32
    y, _ = forward(params, X, emulate_bf16)
    return decode(band_A, y)
