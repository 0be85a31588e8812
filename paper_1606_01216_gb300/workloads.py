"""Seeded synthetic inputs for the shifted-system solve path.

This module builds the *inputs* of the method and nothing else: the mass and
stiffness matrices M, K of a clamped Euler-Bernoulli cantilever discretised
with Hermite-cubic beam elements (the one-dimensional beam model of Sec. 5),
the load matrix F, and the lists of real expansion points (shifts).  It holds
none of the method's arithmetic: no shifted matrix, no SPAI, no CG.  Both the
CUDA path and the CPU oracle are fed from here.

Conventions
-----------
* Nodes 0..n_e along the beam, node 0 clamped (its two DOFs removed), so
  n = 2 n_e and the DOF order is (w_1, theta_1, w_2, theta_2, ..., w_ne,
  theta_ne), 0-based row 2(k-1) = w_k, row 2(k-1)+1 = theta_k.
* Element matrices are the textbook consistent Hermite-cubic ones
  (E I / h^3 and rho A h / 420 scalings).  E = I = rho = A = 1.
* Two scalings of the same FE family:
    "unit"    element length h = 1, beam length L = n_e (well conditioned in
              FP64 at every size; the graded workload);
    "literal" L = 1, h = 1 / n_e (kappa grows like n_e^4).
* M and K are returned in CSR on the full band-7 pattern (|i - j| <= 3),
  explicit zeros kept, sorted column indices: 7 n - 12 stored entries.
* Loads: column 0 is a unit force on the free-end deflection DOF (row n - 2);
  further columns are i.i.d. N(0, 1) from numpy's default_rng(seed).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ALPHA = 0.1    # proportional damping D = alpha M + beta K, Eq. (1.1)
BETA = 1e-4
HALF_BW = 3    # band-7 pattern: offsets -3..+3


@dataclass
class BeamCSR:
    """Band-7 CSR pair (M, K) sharing one pattern."""
    n: int
    n_e: int
    h: float
    rowptr: np.ndarray   # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    m_val: np.ndarray    # float64 [nnz]
    k_val: np.ndarray    # float64 [nnz]
    scaling: str = "unit"
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def element_matrices(h: float) -> tuple[np.ndarray, np.ndarray]:
    """Consistent Hermite-cubic beam element (DOFs w_a, theta_a, w_b, theta_b)."""
    ke = np.array([[12.0, 6 * h, -12.0, 6 * h],
                   [6 * h, 4 * h * h, -6 * h, 2 * h * h],
                   [-12.0, -6 * h, 12.0, -6 * h],
                   [6 * h, 2 * h * h, -6 * h, 4 * h * h]]) / h ** 3
    me = np.array([[156.0, 22 * h, 54.0, -13 * h],
                   [22 * h, 4 * h * h, 13 * h, -3 * h * h],
                   [54.0, 13 * h, 156.0, -22 * h],
                   [-13 * h, -3 * h * h, -22 * h, 4 * h * h]]) * (h / 420.0)
    return ke, me


def band_pattern(n: int, w: int = HALF_BW) -> tuple[np.ndarray, np.ndarray]:
    """CSR rowptr/col of the full band |i-j| <= w of an n x n matrix."""
    rows = np.arange(n, dtype=np.int64)
    lo = np.maximum(rows - w, 0)
    hi = np.minimum(rows + w, n - 1)
    counts = hi - lo + 1
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    # column index = lo[row] + position within the row
    row_of = np.repeat(rows, counts)
    pos = np.arange(nnz, dtype=np.int64) - rowptr[row_of]
    col = (lo[row_of] + pos).astype(np.int32)
    return rowptr, col


def beam(n_e: int, scaling: str = "unit") -> BeamCSR:
    """Clamped cantilever with n_e Hermite-cubic elements, band-7 CSR."""
    if n_e < 1:
        raise ValueError("n_e must be >= 1")
    if scaling == "unit":
        h = 1.0
    elif scaling == "literal":
        h = 1.0 / n_e
    else:
        raise ValueError("scaling must be 'unit' or 'literal'")
    n = 2 * n_e
    ke, me = element_matrices(h)
    # dense-band accumulation: band[d+3, i] = entry (i, i+d) of the full
    # (clamped-node-included) matrix of size N = 2 (n_e + 1)
    N = 2 * (n_e + 1)
    kb = np.zeros((7, N))
    mb = np.zeros((7, N))
    first = 2 * np.arange(n_e)                    # first DOF of each element
    for a in range(4):
        for b in range(4):
            d = b - a
            np.add.at(kb[d + 3], first + a, ke[a, b])
            np.add.at(mb[d + 3], first + a, me[a, b])
    kb = kb[:, 2:]   # drop clamped node rows (w_0, theta_0)
    mb = mb[:, 2:]
    rowptr, col = band_pattern(n)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    d = col.astype(np.int64) - rows
    k_val = np.ascontiguousarray(kb[d + 3, rows])
    m_val = np.ascontiguousarray(mb[d + 3, rows])
    return BeamCSR(n=n, n_e=n_e, h=h, rowptr=rowptr, col=col, m_val=m_val,
                   k_val=k_val, scaling=scaling)


def loads(n: int, m: int = 1, seed: int | None = None) -> np.ndarray:
    """F in R^{n x m}, column-major (Fortran order): tip force + N(0,1) columns."""
    if m < 1:
        raise ValueError("m must be >= 1")
    F = np.zeros((n, m), order="F")
    F[n - 2, 0] = 1.0
    if m > 1:
        rng = np.random.default_rng(seed)
        F[:, 1:] = rng.standard_normal((n, m - 1))
    return F


def log_shifts(lo_exp: float, hi_exp: float, count: int) -> np.ndarray:
    """count real shifts log-spaced over [10^lo_exp, 10^hi_exp], both ends kept."""
    return np.logspace(lo_exp, hi_exp, count)


def midpoint_shifts(lo_exp: float, hi_exp: float, count: int) -> np.ndarray:
    """count shifts at the geometric midpoints of a (count+1)-point logspace."""
    g = np.logspace(lo_exp, hi_exp, count + 1)
    return np.sqrt(g[:-1] * g[1:])


# ---------------------------------------------------------------------------
# workloads with the sizes and structure of the paper's beam experiments
# ---------------------------------------------------------------------------

def small_beam_case():
    """500 elements (n = 1000), tip force, 4 shifts log-spaced in [1, 1e3]."""
    return dict(n_e=500, m=1, shifts=log_shifts(0, 3, 4), seed=None)


def scale_beam_case(n_e: int = 50_000):
    """n = 2 n_e, tip force, 8 shifts log-spaced in [1e-1, 1e4]."""
    return dict(n_e=n_e, m=1, shifts=log_shifts(-1, 4, 8), seed=None)


def headline_case():
    """500,000 elements (n = 1e6), tip force, 8 shifts in [1e-1, 1e4]."""
    return scale_beam_case(500_000)


def batched_beams(seed: int = 20261203, count: int = 32,
                  ne_lo: int = 5_000, ne_hi: int = 500_000):
    """Uneven batch: element counts log-uniform in [ne_lo, ne_hi], 4..16 shifts
    log-spaced in [1e-1, 1e4] per beam, m in {1, 4} RHS per beam."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n_e = int(round(math.exp(rng.uniform(math.log(ne_lo), math.log(ne_hi)))))
        ns = int(rng.integers(4, 17))
        m = int(rng.choice([1, 4]))
        out.append(dict(n_e=n_e, shifts=log_shifts(-1, 4, ns), m=m,
                        seed=int(rng.integers(0, 2 ** 31 - 1))))
    return out


@dataclass
class SparseCSR:
    """A general sparse (M, K) pair, each with its own CSR pattern."""
    n: int
    m_rowptr: np.ndarray
    m_col: np.ndarray
    m_val: np.ndarray
    k_rowptr: np.ndarray
    k_col: np.ndarray
    k_val: np.ndarray
    meta: dict = field(default_factory=dict)


def _coo_to_csr(n, rows, cols, *vals):
    """Sorted CSR with duplicates summed (input assembly, no method arithmetic),
    one value array per matrix on the same (rows, cols) list: returns rowptr,
    col and the summed values of each.  Entries are ordered by (row, col),
    stably, and duplicates are summed in their input order."""
    key = rows.astype(np.int64) * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    idx = np.cumsum(first) - 1
    nu = int(idx[-1]) + 1 if idx.size else 0
    r = rows[order][first]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rowptr[1:])
    col = cols[order][first].astype(np.int32)
    # bincount adds the weights in index order, as a sequential sum would
    summed = [np.bincount(idx, weights=v[order], minlength=nu) for v in vals]
    return (rowptr, col, *summed)


def membrane(nx: int, ny: int, seed: int = 0, lumped_mass: bool = False,
             permute: bool = True) -> SparseCSR:
    """A second-order system whose matrices leave every narrow band: a square
    membrane of nx x ny bilinear quadrilateral elements (unit size), clamped
    along the edge x = 0, with per-element stiffness and density drawn from
    U(0.5, 2) (seed).  Textbook element matrices of the Laplace operator,
    K_e = [[4,-1,-2,-1],[-1,4,-1,-2],[-2,-1,4,-1],[-1,-2,-1,4]] / 6 and
    M_e = [[4,2,1,2],[2,4,2,1],[1,2,4,2],[2,1,2,4]] / 36 (nodes counter-
    clockwise); a 9-point pattern per free node.  lumped_mass replaces M by
    the diagonal of its row sums (a different pattern from K).  permute
    renumbers the free nodes by a seeded random permutation, so the
    pattern has no band structure.  n = nx * (ny + 1)."""
    rng = np.random.default_rng(seed)
    ke = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    me = np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]]) / 36.0
    # grid nodes (i, j), i = 0..nx along x, j = 0..ny; nodes with i = 0 clamped
    free = np.arange(nx * (ny + 1))
    perm = rng.permutation(free.size) if permute else free
    E = rng.uniform(0.5, 2.0, (nx, ny))
    rho = rng.uniform(0.5, 2.0, (nx, ny))
    # element (ex, ey) has nodes (ex, ey), (ex+1, ey), (ex+1, ey+1), (ex, ey+1);
    # entries in element order, then a, then b (the order duplicates are summed in)
    ex, ey = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    ni = np.stack([ex, ex + 1, ex + 1, ex], axis=-1)          # (nx, ny, 4) node i
    nj = np.stack([ey, ey, ey + 1, ey + 1], axis=-1)
    nodes = np.where(ni > 0, perm[np.maximum(ni - 1, 0) * (ny + 1) + nj], -1)
    ra = np.broadcast_to(nodes[:, :, :, None], (nx, ny, 4, 4))
    cb = np.broadcast_to(nodes[:, :, None, :], (nx, ny, 4, 4))
    keep = (ra >= 0) & (cb >= 0)
    rows = ra[keep].astype(np.int64)
    cols = cb[keep].astype(np.int64)
    kv = (E[:, :, None, None] * ke[None, None])[keep]
    mv = (rho[:, :, None, None] * me[None, None])[keep]
    n = free.size
    krp, kci, kva, mva = _coo_to_csr(n, rows, cols, kv, mv)
    mrp, mci = krp, kci
    if lumped_mass:
        diag = np.zeros(n)
        np.add.at(diag, np.repeat(np.arange(n), np.diff(mrp)), mva)
        mrp, mci, mva = np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), diag
    return SparseCSR(n, mrp, mci, mva, krp, kci, kva,
                     meta=dict(nx=nx, ny=ny, seed=seed, lumped_mass=lumped_mass))


def cantilever_beta_l(k: int) -> float:
    """k-th root (1-based) of 1 + cos x cosh x = 0 by bisection (closed form
    used to pin the assembled M, K; not part of the method)."""
    f = lambda x: 1.0 + math.cos(x) * math.cosh(x)
    lo = (k - 0.5) * math.pi - 1.0 if k > 1 else 1.0
    hi = (k - 0.5) * math.pi + 1.0 if k > 1 else 2.5
    flo = f(lo)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if (fm < 0) == (flo < 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


# ---------------------------------------------------------------------------
# inputs of the learned SPAI-column predictor (network shapes, seeded draws)
# ---------------------------------------------------------------------------

MLP_IN, MLP_HID, MLP_OUT = 16, 64, 16
MLP_NPARAM = MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_OUT * MLP_HID + MLP_OUT


def mlp_random_params(seed: int, bias_scale: float = 0.5) -> np.ndarray:
    """FP32 parameter vector W1|b1|W2|b2|W3|b3 (W[out][in]) with Glorot-uniform
    weights and uniform biases, for parity tests."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in ((MLP_HID, MLP_IN), (MLP_HID, MLP_HID), (MLP_OUT, MLP_HID)):
        lim = math.sqrt(6.0 / (o + i))
        parts.append(rng.uniform(-lim, lim, o * i))
        parts.append(rng.uniform(-bias_scale, bias_scale, o))
    return np.concatenate(parts).astype(np.float32)


def mlp_random_samples(seed: int, count: int):
    """Feature rows X[count, 16] (FP32, U(-1, 1)), targets T[count, 8] (FP32,
    U(-2, 2)) and 7-bit output masks (uint8; every fourth row all ones)."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, (count, MLP_IN)).astype(np.float32)
    T = rng.uniform(-2.0, 2.0, (count, 8)).astype(np.float32)
    mask = rng.integers(0, 128, count).astype(np.uint8)
    mask[::4] = 127
    return X, T, mask


def mlp_training_columns(n: int, n_interior: int, seed: int, edge: int = 16) -> np.ndarray:
    """Columns of an n-row beam matrix that enter the training set: the
    `edge` columns at each end (clamped and free) and n_interior columns
    drawn uniformly from the rest, sorted (int64)."""
    rng = np.random.default_rng(seed)
    e = min(edge, n // 2)
    inner = np.arange(e, n - e)
    pick = rng.choice(inner, size=min(n_interior, inner.size), replace=False) if inner.size else inner
    return np.unique(np.concatenate([np.arange(e), np.arange(n - e, n), pick])).astype(np.int64)
