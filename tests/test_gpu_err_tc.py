"""Tensor-core error pass (tensor-core modes of qreconstruct_error) against the exact error of
the same factors, through the C ABI.

For the GPU's own H, X and A the oracle computes ||A - H X||_F / ||A||_F in FP64 (Sec. 5).
The kernel forms H X from BF16 hi/lo pairs (hi*hi + lo*hi + hi*lo, FP32 accumulation): each
real product carries at most 3 * 2^-17 of |h||x| from the splitting plus the FP32
accumulation error, so |(H X)_kernel - H X| <= 2^-15 M elementwise with M = |H| |X| summed
over the Hamilton terms, and the error moves by at most 2^-15 ||M||_F / ||A||_F.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
import workloads as WL

_PLANE = [[0, 1, 2, 3], [1, 0, 3, 2], [2, 3, 0, 1], [3, 2, 1, 0]]


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_14783_gb300 import build as b
    b.build()
    import paper_2404_14783_gb300 as p
    p.load_library()
    return p


def _padded(A):
    """(4, m, n) CUDA FP32 tensor whose rows are 16-byte aligned (pitch a multiple of 4)."""
    m, n = A.shape[1], A.shape[2]
    ldp = (n + 3) // 4 * 4
    buf = torch.zeros(4, m, ldp, dtype=torch.float32, device="cuda")
    buf[:, :, :n] = torch.as_tensor(A, dtype=torch.float32)
    return buf[:, :, :n]


def _bound(H, X, A):
    absH, absX = np.abs(H), np.abs(X)
    M = np.stack([sum(absH[_PLANE[q][b]] @ absX[b] for b in range(4)) for q in range(4)])
    return 2.0 ** -15 * np.linalg.norm(M) / np.linalg.norm(A)


@pytest.mark.parametrize("m,n,s,l,pure", [(256, 128, 21, 43, False), (300, 257, 13, 29, False),
                                          (1000, 700, 101, 203, False), (129, 200, 16, 128, False),
                                          (64, 64, 1, 1, False), (333, 190, 37, 75, True)])
def test_tc_error_matches_exact_error_of_same_factors(pkg, m, n, s, l, pure):
    A = WL.make_decay(m, n, seed=m + s, rank_cap=min(m, n), dtype=np.float32)
    if pure:
        A[0] = 0.0
    Ad = _padded(A)
    planes = [None, Ad[1], Ad[2], Ad[3]] if pure else Ad
    qs = pkg.QSketch(m, n, s, l, prec="bf16x3", seed=3, pure=pure)
    qs.update(planes, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    before = pkg.launch_count()
    err = float(qs.error(planes).item())
    launches = pkg.launch_count() - before
    assert launches == 4          # pack H, pack X^T, tensor-core pass, finalize
    assert qs.device_status() == 0
    H = qs.get("H").cpu().double().numpy()
    X = qs.get("X").cpu().double().numpy()
    A64 = Ad.double().cpu().numpy()
    exact = O.rel_error(A64, H, X)
    bound = _bound(H, X, A64)
    print(f"m={m} n={n} s={s}: tc {err:.9e} exact {exact:.9e} diff {abs(err - exact):.2e} bound {bound:.2e}")
    assert abs(err - exact) <= bound
    assert abs(err - exact) <= 1e-3 * exact


def test_tc_error_of_exact_factors_is_small(pkg):
    """A = H X exactly (rank s quaternion product): the residual is the kernel's own rounding,
    bounded by the same 2^-15 ||M|| / ||A||."""
    m, n, s = 512, 384, 24
    rng = np.random.default_rng(5)
    H = rng.standard_normal((4, m, s)).astype(np.float32)
    X = rng.standard_normal((4, s, n)).astype(np.float32)
    A = O.qmatmul(H.astype(np.float64), X.astype(np.float64)).astype(np.float32)
    Ad = _padded(A)
    qs = pkg.QSketch(m, n, s, 2 * s + 1, prec="bf16x3", seed=1)
    qs.get("H").copy_(torch.as_tensor(H))
    qs.get("X").copy_(torch.as_tensor(X))
    err = float(qs.error(Ad).item())
    bound = _bound(H.astype(np.float64), X.astype(np.float64), Ad.double().cpu().numpy())
    exact = O.rel_error(Ad.double().cpu().numpy(), H.astype(np.float64), X.astype(np.float64))
    print(f"exact-factor case: tc {err:.3e} exact {exact:.3e} bound {bound:.3e}")
    assert err <= exact + bound
