"""The all-cores (OpenMP) build of the oracle against the serial one.

The OpenMP build is the bench's all-cores CPU baseline; it must compute the
same thing.  SPAI columns are independent, so they agree bit for bit; the
PCG iterates differ only by the order in which dot products are summed
(thread chunks added in thread order), so solutions agree to rounding and
iteration counts exactly on this well-conditioned case."""
import numpy as np
import pytest

from paper_1606_01216_gb300 import workloads as W

AL, BE = W.ALPHA, W.BETA


@pytest.fixture()
def both(ora):
    yield ora
    ora.use_openmp(False)


def _run(ora, openmp, A, F):
    ora.use_openmp(openmp)
    P = ora.spai(A)
    Pm, steps, res, _ = ora.spai_mr(A, tol=0.01, kmax=20)
    x, it, st, _ = ora.pcg(A, F, factors=(P,), symmetrize=True)
    return P, Pm, steps, x, it, st


def test_openmp_build_matches_serial(both):
    ora = both
    b = W.beam(40_000)                       # n = 80,000: dot products above the split size
    A = ora.shifted_csr(b, AL, BE, 3.0)
    F = W.loads(b.n, 2, seed=3)[:, 1]
    P1, M1, s1, x1, it1, st1 = _run(ora, False, A, F)
    P2, M2, s2, x2, it2, st2 = _run(ora, True, A, F)
    assert ora.threads() >= 1
    assert np.array_equal(P1.val, P2.val) and np.array_equal(M1.val, M2.val)
    assert np.array_equal(s1, s2)
    assert st1 == st2 == ora.OK and it1 == it2
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)
