"""The stages after the sketch at the tolerance of the FP64 steps, for every arithmetic of
those stages (qs_config.rf_prec), with the sketch and the rangefinder's input isolated.

Each comparison gives the GPU and the oracle the same input values: Y is written straight
into the handle (pseudo-QR, Alg. 1), and the QB stage (Alg. 3) is checked against the
oracle run on the GPU's own H, W and exported Psi, so that the sensitivity of earlier steps
does not enter.

Tolerances, from the arithmetic (u = 2^-53 for FP64, 2^-48 for double-float, whose values
are an unevaluated sum of two FP32 numbers):
  * pseudo-QR, Y = U diag(sigma) V* with kappa(Y) = 10: H element by element and the three
    correction parameters eps_k, relative, 1e-12 -- for FP64 and for double-float (shown
    equal to FP64 here, on the same Y).  A backward-stable thin QR determines its Q factor
    to ~u kappa(Y), and the corrections are smooth in H, so H carries that error; eps_k is
    a Rayleigh quotient of G_k^{-1}, sensitive as u kappa(G_k) = u kappa(H_k)^2.
  * kappa(Y) = 1e3: the same quantities at the bars that this conditioning allows: H at
    100 u kappa(Y), the eps_k at 100 u kappa(Y)^2 (eps_1 has that sensitivity, and the later
    corrections inherit its error through H_1); the factor 100 stands for the dimension-
    dependent constants (s = 24) of the forward-error bounds of the QR and the solves.
  * QB stage: P = Psi H against the oracle's product, 1e-12; X = P^dagger W against the
    oracle's least-squares solution with the same H, W, Psi, 1e-12 (kappa(P) ~ 6 here).
  * The stop path of the corrections (kappa estimate above 1e8, the range of use the paper
    gives for pseudo-QR): QS_ERR_RANK, all eps_k = 0, H = the uncorrected H_0, whose range
    is Y's to 100 u kappa(Y) (H_0 = Y D with kappa(D) = kappa(Y)).  FP64 storage: kappa(Y)
    = 1e10.  FP32 storage cannot hold such a Y (rounding Y to FP32 alone lifts its smallest
    singular values to ~1e-7 of the largest), so there Y has two equal columns (exactly
    rank deficient).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
import workloads as WL

M, N, S, L = 600, 400, 24, 49
U64, UDF = 2.0 ** -53, 2.0 ** -48
QS_ERR_RANK = 4


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
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def relmax(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.abs(a - b).max() / np.abs(b).max())


def _make_y(kappa, seed, m=M, s=S):
    rng = np.random.default_rng(seed)
    U = WL.random_orthonormal(rng, m, s)
    V = WL.random_orthonormal(rng, s, s)
    sig = np.logspace(0.0, -np.log10(kappa), s)
    return O.qmatmul(U * sig[None, None, :], O.qconjT(V))


def _put(qs, name, M_, f64):
    dt = torch.float64 if f64 else torch.float32
    t = torch.as_tensor(M_, dtype=dt)
    qs.get(name).copy_(t)
    return t.double().numpy()     # the values the GPU holds


# (sketch precision, rf_prec): FP64 storage; FP32 storage with double-float or native FP64
# stages; the split-BF16 tensor-core mode with double-float stages (the bench's setting)
MODES = [("fp64", "df64"), ("fp32", "df64"), ("fp32", "fp64"), ("bf16x3", "df64")]


def _unit(prec, rf):
    return U64 if prec == "fp64" or rf == "fp64" else UDF


@pytest.mark.parametrize("kind", ["pseudo_qr", "pseudo_qr_householder"])
@pytest.mark.parametrize("prec,rf", MODES)
@pytest.mark.parametrize("kappa", [10.0, 1e3])
def test_pseudo_qr_with_corrections_elementwise(pkg, prec, rf, kappa, kind):
    """Both thin-QR routes of Alg. 1 step 2 (Cholesky-QR, Householder reflections) give the
    same canonical Q (R_ii > 0), hence the same H."""
    qs = pkg.QSketch(M, N, S, L, emb="gaussian", prec=prec, rf_prec=rf, seed=3)
    Y = _put(qs, "Y", _make_y(kappa, 11), prec == "fp64")
    qs.rangefinder(kind, 3)
    torch.cuda.synchronize()
    assert qs.device_status() == 0
    H = qs.get("H")
    assert H.dtype == torch.float64          # the FP64-class stages keep H in FP64
    H = H.cpu().numpy()
    eps = qs.get("scalars")[2:5].cpu().numpy()
    info = {}
    Href = O.pseudo_qr(Y, 3, info=info)
    if kappa <= 10:
        bar_h, bar_e = 1e-12, [1e-12] * 3
    else:
        u = _unit(prec, rf)
        bar_h = max(1e-12, 100 * u * kappa)
        bar_e = [max(1e-12, 100 * u * kappa ** 2)] * 3
    assert relmax(H, Href) <= bar_h, (relmax(H, Href), bar_h)
    for k in range(3):
        assert abs(eps[k] - info["eps"][k]) <= bar_e[k] * info["eps"][k], (k, eps[k], info["eps"][k])


@pytest.mark.parametrize("prec,rf", MODES)
def test_qb_stage_on_the_gpus_own_h(pkg, prec, rf):
    """P = Psi H and X = (Psi H)^dagger W (Alg. 3, Alg. QLEQ) against the oracle given the
    GPU's H, W and Psi."""
    A = WL.make_decay(M, N, seed=5, rank_cap=200, dtype=np.float64)
    f64 = prec == "fp64"
    qs = pkg.QSketch(M, N, S, L, emb="gaussian", prec=prec, rf_prec=rf, seed=9)
    Ad = torch.as_tensor(A, dtype=torch.float64 if f64 else torch.float32, device="cuda")
    qs.update(Ad, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    torch.cuda.synchronize()
    assert qs.device_status() == 0
    H = qs.get("H").cpu().numpy()
    W = qs.get("W").cpu().double().numpy()
    Psi = qs.get("Psi").cpu().double().numpy()       # the exported test matrix
    P = qs.get("PsiH").cpu().numpy()
    X = qs.get("X")
    assert X.dtype == torch.float64
    X = X.cpu().numpy()
    Pref = O.qmatmul(Psi, H)
    Xref = O.qb_core(H, Psi, W)
    assert rel(P, Pref) <= 1e-12, rel(P, Pref)
    assert rel(X, Xref) <= 1e-12, rel(X, Xref)
    assert relmax(X, Xref) <= 1e-11, relmax(X, Xref)


@pytest.mark.parametrize("prec,rf", [("fp64", "df64"), ("bf16x3", "df64")])
def test_corrections_stop_beyond_their_range(pkg, prec, rf):
    """The kappa estimate of H_0 exceeds 1e8, so the corrections are skipped (QS_ERR_RANK as
    a warning, all eps_k = 0) and H is the uncorrected H_0, which still spans R(Y)."""
    f64 = prec == "fp64"
    kappa = 1e10
    Y = _make_y(kappa, 21)
    if not f64:
        Y[:, :, S - 1] = Y[:, :, 0]
    qs = pkg.QSketch(M, N, S, L, emb="gaussian", prec=prec, rf_prec=rf, seed=3)
    Y = _put(qs, "Y", Y, f64)
    qs.rangefinder("pseudo_qr", 3)
    torch.cuda.synchronize()
    assert qs.device_status() == QS_ERR_RANK
    sc = qs.get("scalars").cpu().numpy()
    np.testing.assert_array_equal(sc[2:5], 0.0)
    H = qs.get("H").cpu().numpy()
    CH, CY = O.chi(H), O.chi(Y)
    Qh, _ = np.linalg.qr(CH)
    u = _unit(prec, rf)
    resid = np.linalg.norm(CY - Qh @ (Qh.conj().T @ CY)) / np.linalg.norm(CY)
    assert resid <= (100 * u * kappa if f64 else 1e-6), resid
    if not f64:
        return
    # the oracle's Alg. 1 without corrections spans the same space
    H0 = O.pseudo_qr(Y, 0)
    Q0, _ = np.linalg.qr(O.chi(H0))
    dist = np.linalg.norm(Qh @ Qh.conj().T - Q0 @ Q0.conj().T) / np.sqrt(2 * S)
    assert dist <= 100 * u * kappa, dist


def test_double_float_equals_native_fp64_on_the_same_y(pkg):
    """The bench's arithmetic (double-float) against native FP64 on the GPU, same Y, W and
    test matrices, on a decaying spectrum (sigma_i = i^-2, kappa(Y) ~ 1e3): H, P and X agree
    to 30 u_df kappa(Y), the level at which u_df-sized rounding moves a backward-stable QR's
    Q factor (1e-12 when Y is well conditioned, see above)."""
    A = WL.make_decay(M, N, seed=7, rank_cap=200, dtype=np.float32)
    Ad = torch.as_tensor(A, device="cuda")
    out = {}
    Yref = Wref = None
    for rf in ("df64", "fp64"):
        qs = pkg.QSketch(M, N, S, L, emb="gaussian", prec="bf16x3", rf_prec=rf, seed=4)
        qs.update(Ad, theta=0.0)
        if Yref is None:                       # the sketch's reductions are not ordered:
            Yref = qs.get("Y").clone()         # hand both handles the same Y and W
            Wref = qs.get("W").clone()
        else:
            qs.get("Y").copy_(Yref)
            qs.get("W").copy_(Wref)
        qs.rangefinder("pseudo_qr", 3)
        qs.core()
        torch.cuda.synchronize()
        assert qs.device_status() == 0
        out[rf] = {k: qs.get(k).cpu().numpy() for k in ("H", "PsiH", "X")}
    sv = np.linalg.svd(O.chi(Yref.cpu().double().numpy()), compute_uv=False)
    bar = max(1e-12, 30 * UDF * sv[0] / sv[-1])
    for k in ("H", "PsiH", "X"):
        assert rel(out["df64"][k], out["fp64"][k]) <= bar, (k, rel(out["df64"][k], out["fp64"][k]), bar)
