"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (derived from the arithmetic):
  * FP64 steps: 1e-12 relative Frobenius for the sketches (u * sqrt(K) ~ 1e-15 at these K);
    HX and the projector of H carry the intrinsic sensitivity of the range of Y to rounding,
    measured on c1 with the oracle itself (1-ulp input perturbations move the 3-correction
    HX by up to 3.6e-11), so HX is compared at 1e-9; the final error (3e-6 of ||A|| on c1)
    then agrees to 1e-9/3e-6 = 3e-4 relative.
  * FP32 SIMT sketch: 1e-5 relative Frobenius.
  * final relative error: within 1% of the oracle's.
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
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) /
                 max(np.linalg.norm(np.asarray(b, float)), 1e-300))


def _emb(n, s, l, m, kind, seed):
    k = O.EMB_GAUSSIAN if kind == "gaussian" else O.EMB_RADEMACHER
    return (O.draw_embedding(n, s, k, O.STREAM_OMEGA, seed),
            O.draw_embedding(l, m, k, O.STREAM_PSI, seed))


def _proj(H):
    C = O.chi(H)
    return C @ np.linalg.pinv(C)


@pytest.mark.parametrize("kind", ["gaussian", "rademacher"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_draw_matches_published_generator(pkg, kind, prec):
    m, n, s, l = 70, 90, 9, 19
    qs = pkg.QSketch(m, n, s, l, emb=kind, prec=prec, seed=0x1234567890AB)
    Om, Psi = _emb(n, s, l, m, kind, 0x1234567890AB)
    g_om = qs.get("Omega").cpu().numpy().astype(float)
    g_psi = qs.get("Psi").cpu().numpy().astype(float)
    if kind == "rademacher":
        np.testing.assert_array_equal(g_om, Om)
        np.testing.assert_array_equal(g_psi, Psi)
    else:
        tol = 1e-14 if prec == "fp64" else 2e-6
        assert np.abs(g_om - Om).max() <= tol * max(1.0, np.abs(Om).max())
        assert np.abs(g_psi - Psi).max() <= tol * max(1.0, np.abs(Psi).max())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("shape", [(300, 257, 13, 29), (64, 64, 1, 1), (130, 70, 33, 65)])
def test_sketch_parity(pkg, prec, tol, shape):
    m, n, s, l = shape
    A = WL.make_gaussian(m, n, seed=m + n)
    qs = pkg.QSketch(m, n, s, l, emb="gaussian", prec=prec, seed=7)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ad = torch.as_tensor(A, dtype=dt, device="cuda")
    qs.update(Ad, theta=0.0)
    Om, Psi = _emb(n, s, l, m, "gaussian", 7)
    Aref = Ad.double().cpu().numpy()          # the FP32 path's input values, exactly
    Y, W = O.sketch(Aref, Om, Psi)
    assert rel(qs.get("Y").cpu().numpy(), Y) < tol
    assert rel(qs.get("W").cpu().numpy(), W) < tol


def test_sketch_linear_updates_and_theta(pkg):
    """Streaming by linear updates: blocks sum to the whole; theta scales the old sketch."""
    m, n, s, l = 150, 120, 6, 13
    A = WL.make_gaussian(m, n, seed=3)
    Om, Psi = _emb(n, s, l, m, "gaussian", 11)
    qs = pkg.QSketch(m, n, s, l, prec="fp64", seed=11)
    Ad = torch.as_tensor(A, device="cuda")
    for r0, r1 in ((0, 77), (77, 150)):
        for c0, c1 in ((0, 50), (50, 120)):
            qs.update(Ad[:, r0:r1, c0:c1], row0=r0, col0=c0)
    Y, W = O.sketch(A, Om, Psi)
    assert rel(qs.get("Y").cpu().numpy(), Y) < 1e-12
    assert rel(qs.get("W").cpu().numpy(), W) < 1e-12
    # Y <- 0.5 Y + 2 * (block contribution)
    B = A[:, 10:40, 20:90]
    qs.update(Ad[:, 10:40, 20:90], row0=10, col0=20, theta=0.5, eta=2.0)
    Ypad = np.zeros_like(A); Ypad[:, 10:40, 20:90] = B
    Y2, W2 = O.sketch(Ypad, Om, Psi)
    assert rel(qs.get("Y").cpu().numpy(), 0.5 * Y + 2 * Y2) < 1e-12
    assert rel(qs.get("W").cpu().numpy(), 0.5 * W + 2 * W2) < 1e-12


def test_pure_quaternion_skips_real_plane(pkg):
    m, n, s, l = 80, 60, 5, 11
    A = WL.make_gaussian(m, n, seed=9)
    A[0] = 0.0
    qs = pkg.QSketch(m, n, s, l, prec="fp64", seed=2, pure=True)
    Ad = torch.as_tensor(A, device="cuda")
    qs.update([None, Ad[1], Ad[2], Ad[3]], theta=0.0)
    Om, Psi = _emb(n, s, l, m, "gaussian", 2)
    Y, W = O.sketch(A, Om, Psi)
    assert rel(qs.get("Y").cpu().numpy(), Y) < 1e-12
    assert rel(qs.get("W").cpu().numpy(), W) < 1e-12


def _run(pkg, A, s, l, prec, rf="pseudo_qr", ncorr=3, seed=0, emb="gaussian"):
    m, n = A.shape[1], A.shape[2]
    qs = pkg.QSketch(m, n, s, l, emb=emb, prec=prec, seed=seed)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ad = torch.as_tensor(A, dtype=dt, device="cuda")
    qs.update(Ad, theta=0.0)
    qs.rangefinder(rf, ncorr)
    qs.core()
    err = float(qs.error(Ad).item())
    status = qs.device_status()
    return qs, err, status, Ad


def test_pseudo_qr_no_correction_matches_oracle_elementwise(pkg):
    """With a well-conditioned Y the canonical thin QR (R_ii > 0) is unique: H agrees
    entrywise with the oracle's (Alg. 1 steps 1-3)."""
    m, n, s, l = 200, 150, 12, 25
    A = WL.make_gaussian(m, n, seed=21)
    qs, err, status, _ = _run(pkg, A, s, l, "fp64", ncorr=0, seed=4)
    Om, Psi = _emb(n, s, l, m, "gaussian", 4)
    Y, W = O.sketch(A, Om, Psi)
    H0 = O.pseudo_qr(Y, 0)
    assert status == 0
    assert rel(qs.get("H").cpu().numpy(), H0) < 1e-12


def test_c1_fp64_pipeline(pkg):
    w = WL.WORKLOADS["c1"]
    A = WL.make_c1()
    qs, err, status, _ = _run(pkg, A, w["s"], w["l"], "fp64", ncorr=3, seed=0)
    Om, Psi = _emb(w["n"], w["s"], w["l"], w["m"], "gaussian", 0)
    info = {}
    ref = O.onepass(A, Om, Psi, "pseudo_qr", 3)
    O.pseudo_qr(ref["Y"], 3, info=info)
    assert status in (0,), status
    assert rel(qs.get("Y").cpu().numpy(), ref["Y"]) < 1e-12
    assert rel(qs.get("W").cpu().numpy(), ref["W"]) < 1e-12
    H = qs.get("H").cpu().numpy()
    X = qs.get("X").cpu().numpy()
    HX_ref = O.qmatmul(ref["H"], ref["X"])
    assert rel(O.qmatmul(H, X), HX_ref) < 1e-9
    # the error is 3e-6 of ||A||; HX agrees to 1e-9 of ||A||, so err may move by up to
    # 1e-9/3e-6 = 3e-4 relative (a perturbation aligned with the residual)
    assert abs(err - ref["err"]) <= 3e-4 * ref["err"]
    # the rangefinder's own properties: range of Y and kappa(H) < 10 after 3 corrections
    sv = np.linalg.svd(O.chi(H), compute_uv=False)
    assert sv[0] / sv[-1] < 10
    sc = qs.get("scalars").cpu().numpy()
    np.testing.assert_allclose(sc[2:5], info["eps"], rtol=1e-3)


def test_fp32_pipeline_error_within_one_percent(pkg):
    m, n, s, l = 600, 500, 21, 43
    A = WL.make_decay(m, n, seed=1, rank_cap=500, dtype=np.float32)
    qs, err, status, Ad = _run(pkg, A, s, l, "fp32", ncorr=3, seed=3)
    Om, Psi = _emb(n, s, l, m, "gaussian", 3)
    ref = O.onepass(Ad.double().cpu().numpy(), Om, Psi, "pseudo_qr", 3)
    assert abs(err - ref["err"]) <= 0.01 * ref["err"], (err, ref["err"])


_C2_SHAPED = {}


def _c2_shaped_reference():
    """sigma_i = i^-2 spectrum (rank cap 1024), s = 101, l = 203 at 2048 x 2048; the oracle's
    one-pass result on the same FP32 input values."""
    if not _C2_SHAPED:
        m = n = 2048
        s, l = 101, 203
        A = WL.make_decay(m, n, seed=0, rank_cap=1024, dtype=np.float32)
        Om, Psi = _emb(n, s, l, m, "gaussian", 0)
        A64 = A.astype(np.float64)
        ref = {}
        for nc in (0, 3):
            info = {}
            r = O.onepass(A64, Om, Psi, "pseudo_qr", nc)
            O.pseudo_qr(r["Y"], nc, info=info)
            ref[nc] = (r["err"], info.get("eps", []))
        _C2_SHAPED.update(A=A, A64=A64, Psi=Psi, s=s, l=l, ref=ref)
    return _C2_SHAPED


@pytest.mark.parametrize("ncorr", [3, 0])
@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_c2_shaped_pipeline(pkg, prec, ncorr):
    """The bench workload's shape class at 2048 x 2048 in the FP32 modes.

    * R(H) = R(Y) (Alg. 1): the distance of the GPU's own Y from the range of its H is at
      FP32-rounding level (1e-6 bar; an FP32 product H = Y D with the correction factors
      in D measured 2e-4 here).
    * Final error against the oracle's: the sketches carry relative error <= 5e-6, whose
      effect on HX is statistically independent of the residual A - HX and moves the error
      by far less than 1e-4 relative (measured 4e-6); a bar of 1e-3 fails a range tilt
      (1.4%) or an ill-conditioned core formed in FP32 (0.3% at kappa(H) = 7e3).
    * After 3 corrections kappa(H) < 10 and the correction parameters follow the oracle's.
    """
    c = _c2_shaped_reference()
    s, l = c["s"], c["l"]
    qs, err, status, Ad = _run(pkg, c["A"], s, l, prec, ncorr=ncorr, seed=0)
    ref_err, ref_eps = c["ref"][ncorr]
    H = qs.get("H").cpu().double().numpy()
    Y = qs.get("Y").cpu().double().numpy()
    CH, CY = O.chi(H), O.chi(Y)
    Qh, _ = np.linalg.qr(CH)
    assert np.linalg.norm(CY - Qh @ (Qh.conj().T @ CY)) / np.linalg.norm(CY) < 1e-6
    assert status == 0
    assert abs(err - ref_err) <= 1e-3 * ref_err, (err, ref_err)
    if ncorr == 3:
        sv = np.linalg.svd(CH, compute_uv=False)
        assert sv[0] / sv[-1] < 10
        np.testing.assert_allclose(qs.get("scalars").cpu().numpy()[2:5], ref_eps, rtol=1e-3)
