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


def test_c3_generator_range_and_rank_structure():
    """c3: every channel lies in [0, 1] (rescaled to [0, 0.98] plus U(0, 0.02) noise), and
    without the noise each channel is a sum of 64 cosine modes, i.e. rank <= 128."""
    import torch
    A = WL.make_c3("cpu", m=300, n=257)
    assert A.shape == (3, 300, 257)
    assert float(A.min()) >= 0.0 and float(A.max()) <= 1.0
    sv = torch.linalg.svdvals(A[0].double())
    assert float(sv[128] / sv[0]) < 0.05       # the smooth part: 128 real directions


def test_c5_generator_is_divergence_free():
    """c5: every snapshot is a divergence-free velocity field on the periodic grid (spectral
    divergence, up to the 1e-4 noise), and its columns span at most 32 modes."""
    import torch
    g, steps = 16, 12
    A = WL.make_c5("cpu", grid=g, steps=steps, modes=6, seed=3).double().numpy()
    k = np.fft.fftfreq(g) * g
    K = np.meshgrid(k, k, k, indexing="ij")
    for t in range(steps):
        v = A[:, :, t].reshape(3, g, g, g)
        div = sum(np.fft.ifftn(1j * K[d] * np.fft.fftn(v[d])).real for d in range(3))
        # noise 1e-4 per entry, amplified by at most |k| <= 8 per axis
        assert np.abs(div).max() <= 3 * 8 * 4 * 1e-4 + 1e-6 * np.abs(v).max()
    sv = np.linalg.svd(np.concatenate([A[0], A[1], A[2]], 0), compute_uv=False)
    assert sv[6] / sv[0] < 1e-3                    # 6 modes plus the noise floor
