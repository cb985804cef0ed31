"""Truncation stage (Alg. 4) on the GPU through the C ABI, against the oracle run on the GPU's
own H and X.

The GPU forms the QSVD of X through the Gram X X* = L L* and a complex Jacobi SVD of chi_L:
singular values carry ~u (sigma_1 / sigma_i)^2 relative error from squaring (u = 1.1e-16 in
FP64, 3.6e-15 in double-float), and the subspace U_r a further 1/gap.  Compared are sigma_r
and the basis-invariant product H_r X_r = H floor(X)_r.
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
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / np.linalg.norm(b))


def _pipeline(pkg, A, s, l, prec, seed):
    m, n = A.shape[1], A.shape[2]
    qs = pkg.QSketch(m, n, s, l, prec=prec, seed=seed)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ad = torch.as_tensor(A, dtype=dt, device="cuda")
    qs.update(Ad, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    return qs, Ad


@pytest.mark.parametrize("case", ["c1_fp64", "decay_bf16x3"])
def test_truncation_matches_oracle(pkg, case):
    if case == "c1_fp64":
        w = WL.WORKLOADS["c1"]
        A, s, l, prec, r, tol_s, tol_p = WL.make_c1(), w["s"], w["l"], "fp64", 10, 1e-8, 1e-8
    else:
        A = WL.make_decay(1000, 700, seed=12, rank_cap=700, dtype=np.float32)
        s, l, prec, r, tol_s, tol_p = 101, 203, "bf16x3", 50, 1e-6, 1e-5
    qs, Ad = _pipeline(pkg, A, s, l, prec, seed=21)
    qs.truncate(r)
    assert qs.device_status() == 0
    H = qs.get("H").cpu().double().numpy()
    X = qs.get("X").cpu().double().numpy()
    Hr_ref, sig_ref, V_ref = O.truncate(H, X, r)
    ref_prod = O.qmatmul(Hr_ref, O.truncated_core(sig_ref, V_ref))
    sig = qs.get("sigma").cpu().numpy()
    Hr = qs.get("Hr").cpu().double().numpy()
    Xr = qs.get("Xr").cpu().double().numpy()
    np.testing.assert_allclose(sig, sig_ref, rtol=tol_s)
    assert rel(O.qmatmul(Hr, Xr), ref_prod) < tol_p
    # the truncated approximation's error, through the allocation-free error entry point
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    # the entry point takes all planes in A's type: the factors rounded to it
    Hr_t, Xr_t = qs.get("Hr").to(Ad.dtype), qs.get("Xr").to(Ad.dtype)
    err_r = float(pkg.reconstruct_error_static(Ad, Hr_t, Xr_t, out).item())
    A64 = Ad.double().cpu().numpy()
    ref_err = O.qnorm(A64 - ref_prod) / O.qnorm(A64)
    assert abs(err_r - ref_err) <= 1e-4 * ref_err + 1e-12, (err_r, ref_err)
    # Thm truncationError on the GPU's own result
    _, SA, _ = O.qsvd_dense(A64) if case == "c1_fp64" else (None, None, None)
    if SA is not None:
        sv = np.linalg.svd(O.chi(H), compute_uv=False)
        lhs = O.qnorm(O.qmatmul(Hr, Xr) - O.qmatmul(H, X))
        rhs = sv[0] / sv[-1] * (O.qnorm(A64 - O.qmatmul(H, X)) + np.sqrt(np.sum(SA[r:] ** 2)))
        assert lhs <= rhs


def test_truncation_rank_validation(pkg):
    qs, _ = _pipeline(pkg, WL.make_gaussian(64, 48, seed=1), 5, 11, "fp64", seed=2)
    with pytest.raises(pkg.QSError):
        qs.truncate(0)
    with pytest.raises(pkg.QSError):
        qs.truncate(6)
