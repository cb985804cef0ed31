"""The two rangefinders over a sweep of kappa(Y) (Sec. 3: pseudo-QR for sketches of moderate
condition, pseudo-SVD for any condition; the paper compares them on Y with kappa from 1e6 up).

Y = U diag(sigma) V* (quaternion, m x s) with sigma log-spaced from 1 down to 1/kappa and U, V
random quaternion-orthonormal is written straight into the handle's Y, and the rangefinder
runs on it.  What the method fixes, checked for each kappa:

  * R(H) = R(Y): the part of Y outside the range of H, ||Y - P_H Y||_F / ||Y||_F.  H is formed
    from Y by one product H = Y D (pseudo-QR) or as an orthonormal Q with Y = QR (pseudo-SVD),
    so rounding leaves u * kappa(D) of Y outside R(H) for pseudo-QR (kappa(D) ~ kappa(Y)):
    FP64 bar 100 u kappa(Y) = 1e-14 kappa.  The FP32 modes form H = Y D in double-float and
    store H in FP32, whose rounding alone leaves ~2.5e-8 of Y outside R(H) at any kappa (the
    oracle's H rounded to FP32): bar 1e-6, as for the bench shape.  Pseudo-SVD's Q comes
    from shifted Cholesky-QR3, whose residual does not grow with kappa: bar 1e-12.
  * pseudo-QR: after three corrections kappa(H) < 10 and equal to the oracle's (same eps
    rule; 1% bar), the correction parameters eps_k equal to the oracle's (1e-3).
  * pseudo-SVD: H*H = I.  H takes one left singular vector per pair of chi_Y's paired
    singular values; rounding resolves the 2-dimensional subspace of a pair only to
    u sigma_1 / gap, so quaternion orthogonality between pairs decays as the pairs crowd
    together at small sigma (the oracle's own H: 3e-14 at kappa 1e2, 4e-12 at 1e6, 1e-8 at
    1e10, 9e-8 at 1e13): bar 1e-10 for kappa <= 1e6, 1e-6 above.  For kappa <= 1e6, where
    the range of Y is well determined (its sensitivity to rounding is u kappa), the projector
    of H equals the oracle's (1e-8) and the count of "bad" pairs equals the oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
import workloads as WL

M, N, S, L = 1000, 200, 40, 81


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_14783_gb300 import build as b
    b.build()
    import paper_2404_14783_gb300 as p
    p.load_library()
    return p


def _make_y(kappa, seed):
    rng = np.random.default_rng(seed)
    U = WL.random_orthonormal(rng, M, S)
    V = WL.random_orthonormal(rng, S, S)
    sig = np.logspace(0.0, -np.log10(kappa), S)
    return O.qmatmul(U * sig[None, None, :], O.qconjT(V))


def _run(pkg, Y, kind, prec, seed):
    qs = pkg.QSketch(M, N, S, L, emb="gaussian", prec=prec, seed=seed)
    dt = torch.float64 if prec == "fp64" else torch.float32
    qs.get("Y").copy_(torch.as_tensor(Y, dtype=dt))
    qs.rangefinder(kind, 3)
    torch.cuda.synchronize()
    H = qs.get("H").cpu().double().numpy()
    sc = qs.get("scalars").cpu().numpy()
    return qs, H, sc


def _outside(H, Y):
    CH, CY = O.chi(H), O.chi(Y)
    Q, _ = np.linalg.qr(CH)
    return np.linalg.norm(CY - Q @ (Q.conj().T @ CY)) / np.linalg.norm(CY)


def _kappa(H):
    sv = np.linalg.svd(O.chi(H), compute_uv=False)
    return sv[0] / sv[-1]


def _proj(H):
    C = O.chi(H)
    return C @ np.linalg.pinv(C)


@pytest.mark.parametrize("kind", ["pseudo_qr", "pseudo_qr_householder"])
@pytest.mark.parametrize("prec,kappa,bar", [("fp64", 1e2, 1e-12), ("fp64", 1e5, 1e-9),
                                            ("fp64", 1e7, 1e-7), ("bf16x3", 1e2, 1e-6),
                                            ("bf16x3", 1e5, 1e-6)])
def test_pseudo_qr_kappa_sweep(pkg, prec, kappa, bar, kind):
    Y = _make_y(kappa, seed=int(np.log10(kappa)))
    if prec != "fp64":
        Y = Y.astype(np.float32).astype(np.float64)     # the values the FP32 handle holds
    qs, H, sc = _run(pkg, Y, kind, prec, seed=1)
    info = {}
    Href = O.pseudo_qr(Y, 3, info=info)
    assert qs.device_status() == 0
    assert np.all(np.isfinite(H))
    assert _outside(H, Y) < bar
    k_gpu, k_ref = _kappa(H), _kappa(Href)
    assert k_gpu < 10
    assert abs(k_gpu - k_ref) <= 1e-2 * k_ref, (k_gpu, k_ref)
    np.testing.assert_allclose(sc[2:5], info["eps"], rtol=1e-3)


@pytest.mark.parametrize("kind,kappa", [("pseudo_svd", 1e2), ("pseudo_svd", 1e6), ("pseudo_svd", 1e10),
                                        ("pseudo_svd", 1e13),
                                        ("pseudo_svd_householder", 1e2),
                                        ("pseudo_svd_householder", 1e6),
                                        ("pseudo_svd_householder", 1e13),
                                        ("pseudo_svd_householder", 1e15),
                                        ("pseudo_svd_householder", 1e16)])
def test_pseudo_svd_kappa_sweep(pkg, kind, kappa):
    """Householder's Q keeps R(H) containing R(Y) to working precision past kappa = 1e15,
    where the Gram of Y (kappa^2 > 1/u) no longer determines it."""
    Y = _make_y(kappa, seed=10 + int(np.log10(kappa)))
    qs, H, sc = _run(pkg, Y, kind, "fp64", seed=2)
    assert np.all(np.isfinite(H))
    orth = 1e-10 if kappa <= 1e6 else 1e-6
    np.testing.assert_allclose(O.qmatmul(O.qconjT(H), H), O.qeye(S), atol=orth)
    assert _outside(H, Y) < 1e-12
    if kappa <= 1e6:
        info = {}
        Href = O.pseudo_svd(Y, f=O.draw_uniform_f(2 * S, 2), info=info)
        assert np.abs(_proj(H) - _proj(Href)).max() < 1e-8
        assert int(sc[5]) == info["t"]
