"""GPU parity of the pseudo-SVD rangefinder (Alg. 2) against the FP64 oracle.

H is unique only up to a unit-quaternion phase per column (and any orthonormal basis of
a repeated singular subspace), so H is compared through its orthogonal projector and
through the basis-invariant product HX (Lemma "HToQ"); its own defining property is
H*H = I.  Tolerances: FP64 1e-10 for projectors and HX (the oracle's pseudo-SVD HX moves by
~3e-15 under 1-ulp input perturbations on c1, and the GPU reaches chi_Y's SVD through a
Cholesky-QR whose Q carries u*kappa(Y) = 3e-10 relative error in the weakest direction of
Y, which HX damps by that direction's share of A); orthonormality 1e-12.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
import workloads as WL


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_14783_gb300 import build as b
    b.build()
    import paper_2404_14783_gb300 as p
    p.load_library()
    return p


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _proj(H):
    C = O.chi(H)
    return C @ np.linalg.pinv(C)


def _emb(n, s, l, m, seed):
    return (O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, seed),
            O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, seed))


def _gpu(pkg, A, s, l, prec="fp64", seed=0):
    m, n = A.shape[1], A.shape[2]
    qs = pkg.QSketch(m, n, s, l, prec=prec, seed=seed)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ad = torch.as_tensor(A, dtype=dt, device="cuda")
    qs.update(Ad, theta=0.0)
    qs.rangefinder("pseudo_svd")
    qs.core()
    err = float(qs.error(Ad).item())
    return qs, err, Ad


def test_pseudo_svd_c1(pkg):
    w = WL.WORKLOADS["c1"]
    A = WL.make_c1()
    qs, err, _ = _gpu(pkg, A, w["s"], w["l"])
    Om, Psi = _emb(w["n"], w["s"], w["l"], w["m"], 0)
    Y, W = O.sketch(A, Om, Psi)
    info = {}
    Href = O.pseudo_svd(Y, f=O.draw_uniform_f(2 * w["s"], 0), info=info)
    H = qs.get("H").cpu().numpy()
    X = qs.get("X").cpu().numpy()
    np.testing.assert_allclose(O.qmatmul(O.qconjT(H), H), O.qeye(w["s"]), atol=1e-12)
    assert np.abs(_proj(H) - _proj(Href)).max() < 1e-10
    Xref = O.qb_core(Href, Psi, W)
    assert rel(O.qmatmul(H, X), O.qmatmul(Href, Xref)) < 1e-10
    assert abs(err - O.rel_error(A, Href, Xref)) < 1e-8 * err
    sc = qs.get("scalars").cpu().numpy()
    assert int(sc[5]) == info["t"]


def test_pseudo_svd_rank_deficient_sketch(pkg):
    """A of rank 5 with s = 7: chi_Y has two numerically zero pairs, which the bad-part
    repair (SVD of chi_{H_b diag f}) must still turn into orthonormal columns; R(H) must
    contain R(Y)."""
    m, n, s, l = 48, 40, 7, 15
    A = WL.make_lowrank(m, n, 5, seed=3)
    qs, err, _ = _gpu(pkg, A, s, l, seed=1)
    Om, Psi = _emb(n, s, l, m, 1)
    Y, _ = O.sketch(A, Om, Psi)
    H = qs.get("H").cpu().numpy()
    sc = qs.get("scalars").cpu().numpy()
    assert int(sc[5]) >= 2
    np.testing.assert_allclose(O.qmatmul(O.qconjT(H), H), O.qeye(s), atol=1e-10)
    CY = O.chi(Y)
    assert np.abs(_proj(H) @ CY - CY).max() < 1e-10 * np.abs(CY).max()
    assert err < 1e-10        # exact recovery: rank(A) <= s (Sec. 5, rank-deficient case)


def test_pseudo_svd_repeated_singular_values(pkg):
    """Y with a repeated quaternion singular value (chi_Y has it four times): the pairs are
    not separated and go through the repair; H must be orthonormal with R(H) = R(Y)."""
    m, n, s, l = 60, 50, 4, 9
    rng = np.random.default_rng(5)
    U = WL.random_orthonormal(rng, m, 4)
    V = WL.random_orthonormal(rng, n, 4)
    A = O.qmatmul(U * np.array([1.0, 1.0, 1.0, 0.5])[None, None, :], O.qconjT(V))
    qs, err, _ = _gpu(pkg, A, s, l, seed=2)
    Om, Psi = _emb(n, s, l, m, 2)
    Y, _ = O.sketch(A, Om, Psi)
    H = qs.get("H").cpu().numpy()
    np.testing.assert_allclose(O.qmatmul(O.qconjT(H), H), O.qeye(s), atol=1e-10)
    assert np.abs(_proj(H) - _proj(Y)).max() < 1e-9
    assert err < 1e-10


def test_pseudo_svd_fp32_pipeline(pkg):
    m, n, s, l = 600, 500, 21, 43
    A = WL.make_decay(m, n, seed=1, rank_cap=500, dtype=np.float32)
    qs, err, Ad = _gpu(pkg, A, s, l, prec="bf16x3", seed=3)
    Om, Psi = _emb(n, s, l, m, 3)
    ref = O.onepass(Ad.double().cpu().numpy(), Om, Psi, "pseudo_svd",
                    f=O.draw_uniform_f(2 * s, 3))
    assert abs(err - ref["err"]) <= 0.01 * ref["err"], (err, ref["err"])
    H = qs.get("H").cpu().double().numpy()
    np.testing.assert_allclose(O.qmatmul(O.qconjT(H), H), O.qeye(s), atol=1e-5)
