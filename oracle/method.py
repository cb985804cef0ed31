"""The one-pass method, step by step, in FP64 (oracle).

Sketch (Sec. 4.1, eq. Y = A Omega, W = Psi A), the two rangefinders pseudo-QR (Alg. 1,
Sec. 3.1) and pseudo-SVD (Alg. 2 "pseudo-SVD", Sec. 3.2), the quaternion linear-equation
solver through the complex representation (Alg. "QLEQ", Sec. 3.1), the QB stage (Alg. 3)
and the relative error of Sec. 5.  Readings of points where the paper is silent are
stated at each function.  Test infrastructure only (see the package docstring).
"""
import numpy as np

from .quaternion import qmatmul, qconjT, chi, comp, from_comp, qnorm

U64 = np.finfo(np.float64).eps / 2.0     # unit roundoff of FP64


# ---------------------------------------------------------------- sketch (Sec. 4.1)
def sketch(A, Omega, Psi):
    """Y = A Omega (m x s) and W = Psi A (l x n), quaternion products (Sec. 4.1)."""
    return qmatmul(A, Omega), qmatmul(Psi, A)


# ---------------------------------------------------------------- pseudo-QR (Alg. 1)
def thin_qr_complex(M):
    """Thin complex QR M = U R with R_ii real and positive (Alg. 1 step 2; the paper calls
    MATLAB ``qr(Y_c, 0)`` whose phase convention is unstated, so the phases are fixed by
    R_ii > 0, which makes the factorisation unique for full column rank)."""
    U, R = np.linalg.qr(M, mode="reduced")
    d = np.diag(R).copy()
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return U * ph[None, :], np.conj(ph)[:, None] * R


def epsilon_rule(chiG, iters=3):
    """Correction parameter eps ~ sigma_s(H) from power iterates on chi_G^{-1}, G = H*H
    (Sec. 3.1 after Prop. "CondReductionSpeed": two or three power iterates approximating
    sigma_1(H^dagger)).  Reading: start from the normalised all-ones 2s-vector, take
    ``iters`` iterates w = chi_G^{-1} v, rho = Re(v* w), v = w / |w|, and return
    eps = 1 / sqrt(rho) of the last iterate; rho <= lambda_max(G^{-1}) so eps >= sigma_s."""
    n = chiG.shape[0]
    v = np.ones(n, dtype=complex) / np.sqrt(n)
    rho = 1.0
    for _ in range(iters):
        w = np.linalg.solve(chiG, v)
        rho = float(np.real(np.vdot(v, w)))
        v = w / np.linalg.norm(w)
    return 1.0 / np.sqrt(rho)


def correction_step(H, power_iters=3):
    """One correction H_new = (1 - eps) H + eps (H^dagger)* (eq. "CondNumReductionIter").
    H^dagger comes from solving chi_{H*H} Z = (H*)_c with Alg. QLEQ, as Alg. 1 step 4 says."""
    G = qmatmul(qconjT(H), H)
    chiG = chi(G)
    eps = epsilon_rule(chiG, power_iters)
    Z = np.linalg.solve(chiG, comp(qconjT(H)))
    Hdag = from_comp(Z)
    return (1.0 - eps) * H + eps * qconjT(Hdag), eps


def pseudo_qr(Y, n_correction=3, power_iters=3, info=None):
    """Pseudo-QR rangefinder (Alg. 1): (1) Y_c; (2) thin complex QR of Y_c; (3) H_0 = U(1:m,:),
    H_1 = -conj(U(m+1:2m,:)); (4) ``n_correction`` correction steps (default 3, the paper's
    "often 3")."""
    U, R = thin_qr_complex(comp(Y))
    H = from_comp(U)
    eps_list = []
    for _ in range(n_correction):
        H, eps = correction_step(H, power_iters)
        eps_list.append(eps)
    if info is not None:
        info["R"] = R
        info["eps"] = eps_list
    return H


# ---------------------------------------------------------------- pseudo-SVD (Alg. 2)
def classify_pairs(S, s, tau=None):
    """Number of leading "good" pairs of the descending singular values S (length 2s) of
    chi_Y (Sec. 3.2: good values still appear exactly twice; the paper gives no tolerance).
    Reading: pair i = (S[2i], S[2i+1]) is good when |S[2i]-S[2i+1]| <= tau S[0] and it is
    separated by more than tau S[0] from both neighbours, with tau = 2s * 1e3 * u; the bad
    part is everything from the first failing pair on (it holds the small values)."""
    if tau is None:
        tau = 2 * s * 1e3 * U64
    thr = tau * S[0]
    for i in range(s):
        a, b = S[2 * i], S[2 * i + 1]
        ok = abs(a - b) <= thr
        if i > 0:
            ok = ok and (S[2 * i - 1] - a) > thr
        if i < s - 1:
            ok = ok and (b - S[2 * i + 2]) > thr
        if not ok:
            return i
    return s


def pseudo_svd(Y, f=None, tau=None, info=None):
    """Pseudo-SVD rangefinder (Alg. 2).  (1) complex SVD of chi_Y, split U = [U_g, U_b];
    (2) H_g from U_g, one left vector per duplicated pair (columns 1, 3, 5, ... of the
    descending SVD: taking the first s columns would put u and J conj(u) together);
    (3) bad part through the SVD route of eq. (H_b diag(f)) for every t > 0 (the branch
    condition "t <~ s" is garbled; the paper calls this route the more accurate one);
    (4) H = [H_g, H_b~].  ``f`` (length >= 2t, values in [1, 2)) is the random scaling."""
    s = Y.shape[2]
    U, S, Vh = np.linalg.svd(chi(Y), full_matrices=False)
    g = classify_pairs(S, s, tau)
    t = s - g
    Hg = from_comp(U[:, 0:2 * g:2])
    if info is not None:
        info.update(S=S, t=t, U=U, Vh=Vh)
    if t == 0:
        return Hg
    Ub = U[:, 2 * g:2 * s]                       # 2m x 2t
    Hb = from_comp(Ub)                           # m x 2t quaternion, (H_b)_c = U_b
    if f is None:
        raise ValueError("pseudo_svd needs the scaling vector f when a bad part exists")
    Hb = Hb * np.asarray(f[:2 * t], dtype=float)[None, None, :]   # H_b diag(f)
    Uh, Sh, _ = np.linalg.svd(chi(Hb), full_matrices=False)      # 2m x 4t
    Hbt = from_comp(Uh[:, 0:2 * t:2])            # one column per pair of the t leading pairs
    if info is not None:
        info["Sh"] = Sh
    return np.concatenate([Hg, Hbt], axis=2)


# ---------------------------------------------------------------- core (Alg. QLEQ, Alg. 3)
def qls_solve(A, B):
    """Quaternion linear equations A X = B through the complex representation (Alg. QLEQ):
    build chi_A and B_c, solve chi_A Z = B_c (least squares for overdetermined systems, as
    MATLAB's backslash does), X = Z(1:n2,:) - conj(Z(n2+1:2n2,:)) j."""
    Z = np.linalg.lstsq(chi(A), comp(B), rcond=None)[0]
    return from_comp(Z)


def qb_core(H, Psi, W):
    """QB stage (Alg. 3 step 2): X = (Psi H) \\ W."""
    return qls_solve(qmatmul(Psi, H), W)


def rel_error(A, H, X):
    """Relative error ||A - H X||_F / ||A||_F (Sec. 5)."""
    return qnorm(A - qmatmul(H, X)) / qnorm(A)


def onepass(A, Omega, Psi, rangefinder="pseudo_qr", n_correction=3, f=None):
    """Sketch, rangefinder and QB stage (Sec. 4.1, Alg. 3).  Returns dict(Y, W, H, X, err)."""
    Y, W = sketch(A, Omega, Psi)
    if rangefinder == "pseudo_qr":
        H = pseudo_qr(Y, n_correction)
    elif rangefinder == "pseudo_svd":
        H = pseudo_svd(Y, f=f)
    elif rangefinder == "qmgs2":
        H = qmgs2(Y)
    else:
        raise ValueError(rangefinder)
    X = qb_core(H, Psi, W)
    return dict(Y=Y, W=W, H=H, X=X, err=rel_error(A, H, X))


# ---------------------------------------------------------------- independent references
def truncate(H, X, r):
    """Truncation stage (Alg. 4): the QSVD X = U Sigma V* (qsvd_dense), its r leading
    triples, and H_r = H U_r.  Returns (H_r, sigma_r, V_r), so that the rank-r approximation
    is H_r diag(sigma_r) V_r* = H floor(X)_r."""
    U, S, V = qsvd_dense(X)
    return qmatmul(H, U[:, :, :r]), S[:r], V[:, :, :r]


def truncated_core(sigma, V):
    """diag(sigma) V* (r x n): the factor that multiplies H_r in the truncated approximation."""
    Vs = qconjT(V)
    return Vs * np.asarray(sigma)[None, :, None]


def _qip(u, v):
    """Quaternion inner product <u, v> = u* v of two (4, m, 1) vectors (Sec. 2.1)."""
    return qmatmul(qconjT(u), v)


def qmgs2(Y):
    """Quaternion modified Gram-Schmidt, applied twice per column (the textbook orthonormaliser
    in the right quaternion vector space of Sec. 2.1): an orthonormal Q with R(Q) = R(Y),
    independent of the complex-representation rangefinders."""
    Q = np.array(Y, dtype=float, copy=True)
    s = Q.shape[2]
    for j in range(s):
        v = Q[:, :, j:j + 1]
        for _ in range(2):
            for i in range(j):
                qi = Q[:, :, i:i + 1]
                v = v - qmatmul(qi, _qip(qi, v))      # right scalar multiple
        Q[:, :, j:j + 1] = v / qnorm(v)
    return Q


def qsvd_dense(A):
    """Compact QSVD A = U Sigma V* through the SVD of chi_A (Thm "QSVD" and the proposition
    relating it to the SVD of chi_A, Sec. 2.2): chi_A has every singular value twice; one
    triple per pair (columns 1, 3, 5, ...) gives U, Sigma, V.  Valid for distinct values."""
    Uc, S, Vh = np.linalg.svd(chi(A), full_matrices=False)
    k = min(A.shape[1], A.shape[2])
    U = from_comp(Uc[:, 0:2 * k:2])
    V = from_comp(np.conj(Vh.T)[:, 0:2 * k:2])
    return U, S[0:2 * k:2], V
