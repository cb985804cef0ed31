"""Pins of the input generators (host logic, no GPU): the quaternion-orthonormal factors are
orthonormal, and the matrices have the spectra their recipes state (the quaternion singular
values are every other singular value of the complex representation, Sec. 2)."""
import numpy as np
import pytest

import oracle as O
import workloads as WL


def _qsv(A):
    return np.linalg.svd(O.chi(A), compute_uv=False)[::2]


@pytest.mark.parametrize("m,R", [(40, 40), (60, 25)])
def test_fast_orthonormal_factor(m, R):
    U = WL.random_orthonormal_fast(np.random.default_rng(m), m, R)
    np.testing.assert_allclose(O.qmatmul(O.qconjT(U), U), O.qeye(R), atol=1e-13)
    assert np.abs(U[1:]).max() > 0.1          # a genuinely quaternion factor


@pytest.mark.parametrize("kind", ["pds", "eds"])
def test_sec5_family_spectrum(kind):
    m, n, R, p, q = 50, 40, 5, 2.0, 0.25
    A = WL.make_ex51(kind, m, n, R=R, p=p, q=q, seed=1)
    tail = np.arange(1, n - R + 1, dtype=float)
    want = np.concatenate([np.ones(R), (tail + 1.0) ** (-p) if kind == "pds" else 10.0 ** (-q * tail)])
    np.testing.assert_allclose(_qsv(A), np.sort(want)[::-1], rtol=1e-9, atol=1e-13)


def test_sec5_low_rank_plus_noise():
    m, n, R, xi = 50, 40, 5, 0.01
    A = WL.make_ex51("lrn", m, n, R=R, xi=xi, seed=2)
    sv = _qsv(A)
    # R values near 1, the rest at the noise level: (xi / n) * ||E|| with E standard quaternion
    # Gaussian (||E||_2 ~ 2 sqrt(4 n)), far below 1
    assert np.all(np.abs(sv[:R] - 1.0) < 0.05)
    assert sv[R] < 0.05 and sv[R] > 1e-5


def test_c4_batch_generator_on_cpu():
    torch = pytest.importorskip("torch")
    batch = WL.make_c4_batch("cpu", dict(count=3, lo=20, hi=36, rank_cap=12, k_lo=2, k_hi=4))
    for m, n, k, A in batch:
        assert 20 <= m <= 36 and 20 <= n <= 36 and 2 <= k <= 4
        assert A.dtype == torch.float32 and A.shape == (4, m, n) and A.stride(1) % 4 == 0
        sv = _qsv(A.double().numpy())
        R = min(m, n, 12)
        np.testing.assert_allclose(sv[:R], np.exp(-np.arange(1, R + 1) / 8.0), rtol=1e-5)
        assert sv[R:].max(initial=0.0) < 1e-5
