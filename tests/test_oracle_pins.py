"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test is chosen so that a plausible mistake in the oracle (a sign, an index, a
transposed operand, a dropped term) fails it.  The oracle is never compared with itself
through a retyped formula: products are checked against the 2x2 complex route or the
real representation, factorisations against their defining properties, and the method
against closed forms (exact recovery, orthogonal projection, the QB-error identity).
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as WL

GOLD = os.path.join(os.path.dirname(__file__), "golden")
U64 = np.finfo(float).eps / 2


def _facts():
    out = {}
    with open(os.path.join(GOLD, "paper_facts.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def _unit(name):
    v = np.zeros(4)
    v["1ijk".index(name)] = 1.0
    return v


def _q(v):
    return np.asarray(v, float).reshape(4, 1, 1)


def _kappa(H):
    sv = np.linalg.svd(O.chi(H), compute_uv=False)
    return sv[0] / sv[-1]


def _proj(H):
    C = O.chi(H)
    return C @ np.linalg.pinv(C)


# ------------------------------------------------------------------ algebra (Sec. 2)
def test_unit_table_golden():
    with open(os.path.join(GOLD, "quaternion_units.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    assert len(rows) == 16
    for a, b, *prod in rows:
        want = np.array(prod, float)
        got = O.qmatmul(_q(_unit(a)), _q(_unit(b))).ravel()
        np.testing.assert_array_equal(got, want)
        np.testing.assert_allclose(O.qscalar_mul_chi(_unit(a), _unit(b)), want, atol=0)


def test_scalar_product_two_routes_associative_normed():
    rng = np.random.default_rng(1)
    for _ in range(50):
        a, b, c = rng.standard_normal((3, 4))
        ab = O.qmatmul(_q(a), _q(b)).ravel()
        np.testing.assert_allclose(ab, O.qscalar_mul_chi(a, b), rtol=1e-14, atol=1e-14)
        lhs = O.qmatmul(_q(ab), _q(c)).ravel()
        rhs = O.qmatmul(_q(a), O.qmatmul(_q(b), _q(c))).ravel()
        np.testing.assert_allclose(lhs, rhs, rtol=1e-13, atol=1e-13)
        assert abs(np.linalg.norm(ab) - np.linalg.norm(a) * np.linalg.norm(b)) < 1e-13


def test_representations_multiplicative():
    rng = np.random.default_rng(2)
    P, Q = rng.standard_normal((4, 5, 3)), rng.standard_normal((4, 3, 4))
    PQ = O.qmatmul(P, Q)
    np.testing.assert_allclose(O.chi(PQ), O.chi(P) @ O.chi(Q), atol=1e-13)
    np.testing.assert_allclose(O.upsilon(PQ), O.upsilon(P) @ O.upsilon(Q), atol=1e-13)
    np.testing.assert_allclose(O.chi(O.qconjT(P)), O.chi(P).conj().T, atol=0)
    np.testing.assert_allclose(O.upsilon(O.qconjT(P)), O.upsilon(P).T, atol=0)
    # ||Q||_F = ||Q_r||_F = ||Upsilon_Q||_F / 2 (Appendix B.1)
    assert abs(O.qnorm(P) - 0.5 * np.linalg.norm(O.upsilon(P))) < 1e-13
    assert abs(O.qnorm(P) - np.linalg.norm(O.chi(P)) / np.sqrt(2)) < 1e-13
    # (PQ)_r = Upsilon_P Q_r (Appendix B.1): stacked planes of the product
    Qr = Q.reshape(12, 4)
    np.testing.assert_allclose(PQ.reshape(20, 4), O.upsilon(P) @ Qr, atol=1e-13)


def test_symplectic_structure():
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((4, 6, 4))
    m = 6
    J = np.block([[np.zeros((m, m)), -np.eye(m)], [np.eye(m), np.zeros((m, m))]])
    Qc = O.comp(Q)
    np.testing.assert_allclose(O.chi(Q), np.hstack([Qc, J @ np.conj(Qc)]), atol=0)
    n = 4
    Jn = np.block([[np.zeros((n, n)), -np.eye(n)], [np.eye(n), np.zeros((n, n))]])
    np.testing.assert_allclose(J.T @ O.chi(Q) @ Jn, np.conj(O.chi(Q)), atol=1e-14)
    v = Qc[:, 0]
    assert abs(np.vdot(v, J @ np.conj(v))) < 1e-13
    np.testing.assert_array_equal(O.from_comp(Qc), Q)


def test_pinv_penrose_conditions():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((4, 7, 4))
    X = O.qpinv(A)
    AX, XA = O.qmatmul(A, X), O.qmatmul(X, A)
    np.testing.assert_allclose(O.qmatmul(AX, A), A, atol=1e-12)
    np.testing.assert_allclose(O.qmatmul(XA, X), X, atol=1e-12)
    np.testing.assert_allclose(O.qconjT(AX), AX, atol=1e-12)
    np.testing.assert_allclose(O.qconjT(XA), XA, atol=1e-12)


# ------------------------------------------------------------------ sketch (Sec. 4.1)
def test_sketch_bruteforce_scalar_route():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((4, 3, 5))
    Om = rng.standard_normal((4, 5, 2))
    Psi = rng.standard_normal((4, 4, 3))
    Y, W = O.sketch(A, Om, Psi)
    for i in range(3):
        for j in range(2):
            acc = sum(O.qscalar_mul_chi(A[:, i, k], Om[:, k, j]) for k in range(5))
            np.testing.assert_allclose(Y[:, i, j], acc, atol=1e-13)
    for i in range(4):
        for j in range(5):
            acc = sum(O.qscalar_mul_chi(Psi[:, i, k], A[:, k, j]) for k in range(3))
            np.testing.assert_allclose(W[:, i, j], acc, atol=1e-13)
    # order matters: A Omega != (Omega^T-ish) products, i.e. the sketch is not commutative
    Yswap = np.stack([sum(O.qscalar_mul_chi(Om[:, k, 0], A[:, 0, k]) for k in range(5))])
    assert np.abs(Yswap.ravel() - Y[:, 0, 0]).max() > 1e-3


def test_sketch_linear_update():
    """Streaming by linear updates (Sec. 4 and Sec. 5.3): the sum of block sketches equals
    the sketch of the whole matrix."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((4, 9, 11))
    Om, Psi = rng.standard_normal((4, 11, 3)), rng.standard_normal((4, 5, 9))
    Y, W = O.sketch(A, Om, Psi)
    Y2, W2 = np.zeros_like(Y), np.zeros_like(W)
    for r0, r1 in ((0, 4), (4, 9)):
        for c0, c1 in ((0, 6), (6, 11)):
            Ab = A[:, r0:r1, c0:c1]
            Y2[:, r0:r1] += O.qmatmul(Ab, Om[:, c0:c1])
            W2[:, :, c0:c1] += O.qmatmul(Psi[:, :, r0:r1], Ab)
    np.testing.assert_allclose(Y2, Y, atol=1e-12)
    np.testing.assert_allclose(W2, W, atol=1e-12)


# ------------------------------------------------------------------ pseudo-QR (Alg. 1)
def test_pseudo_qr_structure():
    f = _facts()
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((4, 40, 9))
    info = {}
    H0 = O.pseudo_qr(Y, 0, info=info)
    Hc = O.comp(H0)
    np.testing.assert_allclose(Hc.conj().T @ Hc, np.eye(9), atol=1e-13)
    # Y_c = H_c R with R upper triangular, real positive diagonal
    R = info["R"]
    np.testing.assert_allclose(O.comp(Y), Hc @ R, atol=1e-12)
    assert np.allclose(np.tril(R, -1), 0) and np.all(np.diag(R).real > 0)
    assert np.allclose(np.diag(R).imag, 0)
    sv = np.linalg.svd(O.chi(H0), compute_uv=False)
    assert sv[0] <= f["pseudo_qr_sigma_max_bound"] + 1e-12
    lam = np.sort(sv ** 2)
    np.testing.assert_allclose(lam + lam[::-1], 2.0, atol=1e-12)   # 1 +- mu pairs
    np.testing.assert_allclose(_proj(H0), _proj(Y), atol=1e-12)     # R(H) = R(Y)
    H3 = O.pseudo_qr(Y, 3)
    np.testing.assert_allclose(_proj(H3), _proj(Y), atol=1e-11)


def _ill_conditioned_Y(rng, m, s, delta):
    """Y whose compact form is well conditioned but whose quaternion columns are nearly
    dependent: column 2c+1 = (column 2c) j + delta * noise, so that R(Y_c) and R(Y_a)
    nearly meet (Remark "Hc_Ha_T"), which makes kappa(H_0) large."""
    Y = rng.standard_normal((4, m, s))
    jq = np.array([0, 0, 1.0, 0]).reshape(4, 1, 1)
    for c in range(0, s - 1, 2):
        col = Y[:, :, c:c + 1]
        Y[:, :, c + 1:c + 2] = O.qmatmul(col, jq) + delta * rng.standard_normal((4, m, 1))
    return Y


def test_correction_reduces_condition_number():
    f = _facts()
    rng = np.random.default_rng(8)
    for delta in (1e-3, 1e-5, 1e-7):
        Y = _ill_conditioned_Y(rng, 60, 8, delta)
        H = O.pseudo_qr(Y, 0)
        k0 = _kappa(H)
        assert k0 > 1.0 / delta * 1e-2
        assert k0 < f["correction_kappa_in"]
        for _ in range(int(f["correction_steps"])):
            G = O.qmatmul(O.qconjT(H), H)
            eps = O.epsilon_rule(O.chi(G))
            smin = np.linalg.svd(O.chi(H), compute_uv=False)[-1]
            kap = _kappa(H)
            Hn, _ = O.correction_step(H)
            assert eps >= smin * (1 - 1e-9)                       # Rayleigh bound
            if eps <= f["correction_delta_max"] * smin and kap > f["correction_kappa_threshold"]:
                assert _kappa(Hn) < np.sqrt(kap)                  # Prop. CondReductionSpeed
            if kap < 1e4:   # projectors of worse-conditioned H carry u*kappa^2 noise
                np.testing.assert_allclose(_proj(Hn), _proj(H), atol=1e-9)   # range kept
            H = Hn
        assert _kappa(H) < f["correction_kappa_out"]


def test_correction_equals_right_multiplication():
    """(H^dagger)* = H (H*H)^{-1}, so one correction is H ((1-eps) I + eps G^{-1})."""
    rng = np.random.default_rng(9)
    H = O.pseudo_qr(rng.standard_normal((4, 30, 6)), 0)
    Hn, eps = O.correction_step(H)
    G = O.qmatmul(O.qconjT(H), H)
    Ginv = O.from_comp(np.linalg.inv(O.chi(G))[:, :6])
    M = (1 - eps) * O.qeye(6) + eps * Ginv
    np.testing.assert_allclose(Hn, O.qmatmul(H, M), atol=1e-12)


# ------------------------------------------------------------------ pseudo-SVD (Alg. 2)
def test_pseudo_svd_distinct_values():
    rng = np.random.default_rng(10)
    Y = rng.standard_normal((4, 50, 7))
    info = {}
    H = O.pseudo_svd(Y, info=info)
    assert info["t"] == 0
    np.testing.assert_allclose(O.qmatmul(O.qconjT(H), H), O.qeye(7), atol=1e-12)
    # Thm "pseudoSVD": Y = H Sigma V* with V built from V_ul, V_dl in the same way
    V = O.from_comp(np.conj(info["Vh"].T)[:, 0:14:2])
    Sig = info["S"][0:14:2]
    np.testing.assert_allclose(O.qmatmul(H * Sig[None, None, :], O.qconjT(V)), Y, atol=1e-12)
    np.testing.assert_allclose(_proj(H), _proj(Y), atol=1e-12)


def test_pseudo_svd_I2_example():
    """Remark after Thm "pseudoSVD": Y = I_2.  chi_Y = I_4, so no pair is separated and the
    whole basis goes through the bad-part repair; H must still be orthonormal with
    R(H) = R(Y) = Q^2."""
    f = _facts()
    m, s = int(f["i2_example_m"]), int(f["i2_example_s"])
    Y = O.qeye(m)[:, :, :s]
    info = {}
    H = O.pseudo_svd(Y, f=O.draw_uniform_f(2 * s, seed=0), info=info)
    assert info["t"] == s
    np.testing.assert_allclose(O.qmatmul(O.qconjT(H), H), O.qeye(s), atol=1e-12)
    # naive choice of the first s columns of the SVD's U (the counter-example) can fail:
    U = np.linalg.svd(O.chi(Y))[0]
    rng = np.random.default_rng(0)
    Z, _ = np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    Hbad = O.from_comp((U @ Z)[:, :s])
    assert np.abs(O.qmatmul(O.qconjT(Hbad), Hbad) - O.qeye(s)).max() > 1e-3


def test_pseudo_svd_rank_deficient_and_repeated():
    rng = np.random.default_rng(11)
    # rank-deficient Y: 5 independent quaternion columns out of 7
    B = rng.standard_normal((4, 40, 5))
    C = rng.standard_normal((4, 5, 7))
    Y = O.qmatmul(B, C)
    info = {}
    H = O.pseudo_svd(Y, f=O.draw_uniform_f(14, seed=3), info=info)
    assert info["t"] >= 2
    np.testing.assert_allclose(O.qmatmul(O.qconjT(H), H), O.qeye(7), atol=1e-11)
    PH = _proj(H)
    CY = O.chi(Y)
    np.testing.assert_allclose(PH @ CY, CY, atol=1e-10)          # R(H) contains R(Y)
    # repeated singular values: Y = U diag(1,1,1,0.5) V*
    U = WL.random_orthonormal(rng, 30, 4)
    V = WL.random_orthonormal(rng, 4, 4)
    Y = O.qmatmul(U * np.array([1, 1, 1, .5])[None, None, :], O.qconjT(V))
    H = O.pseudo_svd(Y, f=O.draw_uniform_f(8, seed=4), info=info)
    np.testing.assert_allclose(O.qmatmul(O.qconjT(H), H), O.qeye(4), atol=1e-11)
    np.testing.assert_allclose(_proj(H), _proj(Y), atol=1e-10)


# ------------------------------------------------------------------ core (Alg. QLEQ, Alg. 3)
def test_qls_solve_square_and_overdetermined():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((4, 6, 6))
    X = rng.standard_normal((4, 6, 3))
    np.testing.assert_allclose(O.qls_solve(A, O.qmatmul(A, X)), X, atol=1e-11)
    A = rng.standard_normal((4, 15, 6))
    B = rng.standard_normal((4, 15, 4))
    X = O.qls_solve(A, B)
    np.testing.assert_allclose(X, O.qmatmul(O.qpinv(A), B), atol=1e-12)
    Rsd = B - O.qmatmul(A, X)
    np.testing.assert_allclose(O.qmatmul(O.qconjT(A), Rsd), 0, atol=1e-11)   # normal eqs


def _small_problem(seed, m=40, n=35, s=6, l=13, rank=None):
    rng = np.random.default_rng(seed)
    if rank is None:
        A = WL.make_decay(m, n, seed=seed, rank_cap=min(m, n), dtype=np.float64)
    else:
        A = WL.make_lowrank(m, n, rank, seed=seed)
    Om = O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, seed)
    Psi = O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, seed)
    return A, Om, Psi


def test_exact_recovery_rank_le_s():
    A, Om, Psi = _small_problem(13, rank=5, s=7, l=15)
    for rf, nc in (("pseudo_qr", 0), ("pseudo_svd", 0), ("qmgs2", 0)):
        r = O.onepass(A, Om, Psi, rf, n_correction=nc, f=O.draw_uniform_f(14, 13))
        assert r["err"] < 1e-12, (rf, r["err"])


def test_basis_invariance():
    """Lemma "HToQ": H (Psi H)^dagger Psi A does not depend on the basis of R(Y)."""
    A, Om, Psi = _small_problem(14)
    HX = [O.qmatmul(r["H"], r["X"]) for r in
          (O.onepass(A, Om, Psi, rf, f=O.draw_uniform_f(12, 14))
           for rf in ("pseudo_qr", "pseudo_svd", "qmgs2"))]
    scale = O.qnorm(HX[2])
    assert O.qnorm(HX[0] - HX[2]) / scale < 1e-11
    assert O.qnorm(HX[1] - HX[2]) / scale < 1e-11


def test_psi_identity_is_orthogonal_projection():
    """With Psi = I and orthonormal H the method is randomized QSVD's QB step: HX = HH*A."""
    A, Om, _ = _small_problem(15)
    Psi = O.qeye(A.shape[1])
    Y, W = O.sketch(A, Om, Psi)
    H = O.pseudo_svd(Y)
    X = O.qb_core(H, Psi, W)
    np.testing.assert_allclose(O.qmatmul(H, X), O.qmatmul(H, O.qmatmul(O.qconjT(H), A)),
                               atol=1e-12)
    Qo = O.qmgs2(Y)
    np.testing.assert_allclose(O.qmatmul(Qo, O.qconjT(Qo)), O.qmatmul(H, O.qconjT(H)), atol=1e-11)


def test_qb_error_identity():
    """Thm "errorAnalysisOfTwoSketch": ||A-HX||^2 = ||A-QQ*A||^2 + ||Psi2^+ Psi1 (Q_perp* A)||^2."""
    A, Om, Psi = _small_problem(16, m=14, n=12, s=4, l=7)
    r = O.onepass(A, Om, Psi, "pseudo_qr")
    Q = O.qmgs2(r["Y"])
    m = A.shape[1]
    rng = np.random.default_rng(0)
    G = rng.standard_normal((4, m, m - 4))
    G = G - O.qmatmul(Q, O.qmatmul(O.qconjT(Q), G))
    Qp = O.qmgs2(G)
    np.testing.assert_allclose(O.qmatmul(O.qconjT(Qp), Q), 0, atol=1e-12)
    lhs = O.qnorm(A - O.qmatmul(r["H"], r["X"])) ** 2
    t1 = O.qnorm(A - O.qmatmul(Q, O.qmatmul(O.qconjT(Q), A))) ** 2
    P2, P1 = O.qmatmul(Psi, Q), O.qmatmul(Psi, Qp)
    t2 = O.qnorm(O.qmatmul(O.qpinv(P2), O.qmatmul(P1, O.qmatmul(O.qconjT(Qp), A)))) ** 2
    assert abs(lhs - (t1 + t2)) <= 1e-10 * lhs


# ------------------------------------------------------------------ dense QSVD
def test_qsvd_dense_against_real_representation():
    rng = np.random.default_rng(17)
    A = rng.standard_normal((4, 9, 6))
    U, S, V = O.qsvd_dense(A)
    np.testing.assert_allclose(O.qmatmul(U * S[None, None, :], O.qconjT(V)), A, atol=1e-12)
    np.testing.assert_allclose(O.qmatmul(O.qconjT(U), U), O.qeye(6), atol=1e-12)
    # Upsilon_A has each quaternion singular value four times (independent library route)
    sr = np.linalg.svd(O.upsilon(A), compute_uv=False)
    np.testing.assert_allclose(sr[0::4], S, rtol=1e-12)
    # Eckart-Young on a tiny case: the truncated QSVD beats random rank-2 approximations
    k = 2
    Ak = O.qmatmul(U[:, :, :k] * S[None, None, :k], O.qconjT(V[:, :, :k]))
    best = O.qnorm(A - Ak)
    assert abs(best ** 2 - np.sum(S[k:] ** 2)) < 1e-10
    for t in range(20):
        B = rng.standard_normal((4, 9, k))
        Bq = O.qmgs2(B)
        assert O.qnorm(A - O.qmatmul(Bq, O.qmatmul(O.qconjT(Bq), A))) >= best - 1e-12


# ------------------------------------------------------------------ random test matrices
def test_embedding_distributions():
    from scipy import stats
    G = O.draw_embedding(300, 200, O.EMB_GAUSSIAN, O.STREAM_OMEGA, 123)
    for p in range(4):
        assert stats.kstest(G[p].ravel(), "norm").pvalue > 1e-3
    assert abs(np.corrcoef(G[0].ravel(), G[1].ravel())[0, 1]) < 0.02
    Rm = O.draw_embedding(300, 200, O.EMB_RADEMACHER, O.STREAM_OMEGA, 123)
    assert set(np.unique(Rm)) == {-1.0, 1.0}
    assert abs(Rm.mean()) < 0.01
    f = O.draw_uniform_f(10000, 5)
    assert f.min() >= 1.0 and f.max() < 2.0 and stats.kstest(f - 1.0, "uniform").pvalue > 1e-3
    # distinct streams and seeds give different matrices
    assert not np.allclose(G, O.draw_embedding(300, 200, O.EMB_GAUSSIAN, O.STREAM_PSI, 123))


def test_gaussian_pinv_expectation():
    """Lemma "normOfSGT" (Sec. 4.3): for an m x n (m <= n) standard Gaussian quaternion G,
    E ||G^dagger||_F^2 = m / (4(n-m)+2).  Pins the Gaussian law (all four planes N(0,1))."""
    m, n, reps = 4, 9, 400
    vals = [O.qnorm(O.qpinv(O.draw_embedding(m, n, O.EMB_GAUSSIAN, O.STREAM_PSI, 1000 + t))) ** 2
            for t in range(reps)]
    want = m / (4 * (n - m) + 2)
    assert abs(np.mean(vals) - want) < 4 * np.std(vals) / np.sqrt(reps)


def test_gaussian_qb_bound_in_expectation():
    """Thm "prob_qb_error_gaussian": E||HX-A||^2 <= (2l+1)/(2(l-s)+1) (2s+1)/(2(s-r)+1) ||Sigma_2||^2."""
    m, n, r, s, l = 60, 50, 4, 8, 17
    A = WL.make_decay(m, n, seed=3, rank_cap=50, power=1.0, dtype=np.float64)
    _, S, _ = O.qsvd_dense(A)
    tail = np.sum(S[r:] ** 2)
    bound = (2 * l + 1) / (2 * (l - s) + 1) * (2 * s + 1) / (2 * (s - r) + 1) * tail
    errs = []
    for seed in range(30):
        Om = O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, seed)
        Psi = O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, seed)
        res = O.onepass(A, Om, Psi, "pseudo_qr")
        errs.append((res["err"] * O.qnorm(A)) ** 2)
    assert np.mean(errs) <= bound
    assert np.min(errs) >= np.sum(S[s:] ** 2) * (1 - 1e-9)      # never beats the best rank-s


def test_c1_pipeline():
    w = WL.WORKLOADS["c1"]
    A = WL.make_c1()
    Om = O.draw_embedding(w["n"], w["s"], O.EMB_GAUSSIAN, O.STREAM_OMEGA, 0)
    Psi = O.draw_embedding(w["l"], w["m"], O.EMB_GAUSSIAN, O.STREAM_PSI, 0)
    r = O.onepass(A, Om, Psi, "pseudo_qr")
    _, S, _ = O.qsvd_dense(A)
    best = np.sqrt(np.sum(S[w["s"]:] ** 2) / np.sum(S ** 2))
    assert best <= r["err"] < 4 * best
    r2 = O.onepass(A, Om, Psi, "pseudo_svd", f=O.draw_uniform_f(2 * w["s"], 0))
    assert abs(r2["err"] - r["err"]) < 1e-3 * r["err"]


# ----------------------------------------------------------------- truncation stage (Alg. 4)
def _c1_like_factors(seed=3):
    A = WL.make_c1() if seed == 3 else None
    w = WL.WORKLOADS["c1"]
    Om = O.draw_embedding(w["n"], w["s"], O.EMB_GAUSSIAN, O.STREAM_OMEGA, seed)
    Psi = O.draw_embedding(w["l"], w["m"], O.EMB_GAUSSIAN, O.STREAM_PSI, seed)
    res = O.onepass(A, Om, Psi, "pseudo_qr", 3)
    return A, res["H"], res["X"]


def test_truncation_eckart_young_and_full_rank():
    """floor(X)_r = U_r Sigma_r V_r* leaves exactly the tail energy of X (Eckart-Young, a
    closed form from the QSVD), and r = s reproduces H X."""
    A, H, X = _c1_like_factors()
    s = X.shape[1]
    _, S, _ = O.qsvd_dense(X)
    for r in (1, 5, 10, s):
        Hr, sig, V = O.truncate(H, X, r)
        U, _, _ = O.qsvd_dense(X)
        Xr = O.qmatmul(U[:, :, :r], O.truncated_core(sig, V))
        tail = np.sqrt(np.sum(S[r:] ** 2))
        assert abs(O.qnorm(X - Xr) - tail) <= 1e-10 * O.qnorm(X)
        np.testing.assert_allclose(O.qmatmul(Hr, O.truncated_core(sig, V)), O.qmatmul(H, Xr),
                                   atol=1e-12 * O.qnorm(H) * O.qnorm(X))
    Hs, sig, V = O.truncate(H, X, s)
    assert O.qnorm(O.qmatmul(Hs, O.truncated_core(sig, V)) - O.qmatmul(H, X)) <= 1e-11 * O.qnorm(O.qmatmul(H, X))


def test_truncation_error_theorem():
    """Thm truncationError: ||H floor(X)_r - H X|| <= kappa(H) (||A - HX|| + ||Sigma_2||_F)."""
    A, H, X = _c1_like_factors()
    _, SA, _ = O.qsvd_dense(A)
    sv = np.linalg.svd(O.chi(H), compute_uv=False)
    kap = sv[0] / sv[-1]
    HX = O.qmatmul(H, X)
    for r in (3, 8, 10, 15):
        Hr, sig, V = O.truncate(H, X, r)
        lhs = O.qnorm(O.qmatmul(Hr, O.truncated_core(sig, V)) - HX)
        rhs = kap * (O.qnorm(A - HX) + np.sqrt(np.sum(SA[r:] ** 2)))
        assert lhs <= rhs, (r, lhs, rhs)


def test_truncation_planted_mistake_fails():
    """Taking the trailing instead of the leading singular triples breaks Eckart-Young."""
    A, H, X = _c1_like_factors()
    U, S, V = O.qsvd_dense(X)
    r = 5
    Xbad = O.qmatmul(U[:, :, -r:], O.truncated_core(S[-r:], V[:, :, -r:]))
    assert abs(O.qnorm(X - Xbad) - np.sqrt(np.sum(S[r:] ** 2))) > 1e-3 * O.qnorm(X)


def test_epsilon_rule_closed_form():
    """Reading of Sec. 3.1's "two or three power iterates": three iterates v <- A^{-1} v / |.|
    on A = chi_G from the normalised all-ones vector v0, eps = 1/sqrt(rho) of the last
    Rayleigh quotient.  In the eigenbasis A = V diag(lam) V*, with c = V* v0, that quotient is
    rho = sum |c_i|^2 lam_i^-5 / sum |c_i|^2 lam_i^-4 (a textbook identity, computed here by
    a Hermitian eigendecomposition instead of linear solves).  Two iterates (rho with
    exponents -3 / -2) must not match."""
    rng = np.random.default_rng(17)
    for s in (3, 6):
        H = rng.standard_normal((4, 3 * s, s))   # no isolated small eigenvalue: the
        A = O.chi(O.qmatmul(O.qconjT(H), H))      # iterate counts give different eps
        lam, V = np.linalg.eigh(A)
        v0 = np.ones(2 * s) / np.sqrt(2 * s)
        c2 = np.abs(V.conj().T @ v0) ** 2
        want = 1.0 / np.sqrt(np.sum(c2 * lam ** -5.0) / np.sum(c2 * lam ** -4.0))
        assert abs(O.epsilon_rule(A) - want) <= 1e-10 * want
        two = 1.0 / np.sqrt(np.sum(c2 * lam ** -3.0) / np.sum(c2 * lam ** -2.0))
        assert abs(two - want) > 1e-3 * want


def test_pair_classification_reading():
    """Reading of Sec. 3.2's "good" pairs (singular values of chi_Y that still appear exactly
    twice; the paper gives no tolerance): pair i = (S[2i], S[2i+1]) is good when its two
    values agree within tau S[0] and it is separated by more than tau S[0] from both
    neighbours; the bad part starts at the first failing pair.  Hand-built sequences with
    tau = 1e-6 and their known counts of leading good pairs."""
    tau = 1e-6
    cases = [
        ([5, 5, 3, 3, 1, 1], 3),                      # all pairs clean
        ([5, 5, 3, 2.9, 1, 1], 1),                    # pair 1 split by 0.1 > tau * 5
        ([5, 5, 3, 3 - 1e-7, 1, 1], 3),               # split below tau * 5: still a pair
        ([5, 5, 5, 5, 1, 1], 0),                      # a repeated quaternion value: four equal
        ([5, 5, 2, 2, 2, 2], 1),                      # repetition at the end
        ([5, 5, 2, 2, 0, 0, 0, 0], 2),                # two zero quaternion values (rank loss)
        ([5, 5, 2, 2, 0, 0], 3),                      # one zero value: an exact pair
        ([5, 5, 1 + 4e-6, 1 + 4e-6, 1, 1], 1),        # neighbours 4e-6 apart < tau * 5
    ]
    for S, g in cases:
        S = np.asarray(S, dtype=float)
        assert O.classify_pairs(S, len(S) // 2, tau=tau) == g, (S, g)
    # the default tau = 2 s 1e3 u: pairs closer than that relative to S[0] are not separated
    s = 4
    t0 = 2 * s * 1e3 * U64
    S = np.array([1, 1, 0.5, 0.5, 0.5 - 0.5 * t0, 0.5 - 0.5 * t0, 0.1, 0.1])
    assert O.classify_pairs(S, s) == 1


def test_philox_known_answers():
    """The counter-based generator both sides implement, against the known-answer vectors
    published with its definition (tests/golden/philox4x32_10_kat.txt)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = O.philox4x32_10(*(np.array([v], dtype=np.uint64) for v in w[:4]), w[4], w[5])
        assert [int(np.asarray(x).ravel()[0]) for x in out] == w[6:10]


# ---------------------------------------------------------------- the Lorenz-type system
def test_lorenz_rhs_at_a_hand_computed_point():
    """The right-hand side of the paper's 4D system at (1, 2, 3, 4), a = 15, b = 2, c = 28:
    (15 (2 - 1), 28 - 2 - 3 + 4, -6 + 2, 27 * 2 + 4 - 1/2) = (15, 27, -4, 57.5)."""
    v = O.lorenz4d_rhs(np.array([1.0, 2.0, 3.0, 4.0]))
    np.testing.assert_array_equal(v, [15.0, 27.0, -4.0, 57.5])


def test_rk4_order_and_exact_linear_step():
    """The RK4 step is exact to fifth order on u' = lam u (the truncated exponential series),
    and on the Lorenz system halving the step divides the error at a fixed time by ~16."""
    h, lam = 0.1, -1.3
    z = lam * h
    step = O.rk4_step(lambda u: lam * u, np.array([1.0]), h)[0]
    assert abs(step - (1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24)) < 1e-15
    u0 = WL.lorenz_initial_states(3, seed=1)
    T = 0.05
    ref = O.lorenz4d_snapshots(u0, 1600, T / 1600)[:, -1]
    e = [np.abs(O.lorenz4d_snapshots(u0, n, T / n)[:, -1] - ref).max() for n in (50, 100)]
    assert 12.0 < e[0] / e[1] < 20.0, e
