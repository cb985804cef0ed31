"""Quaternion algebra and the matrix representations of Sec. 2 and Appendix B.1 (oracle).

Test infrastructure only (see the package docstring).  FP64 throughout.
"""
import numpy as np


def qzeros(r, c):
    return np.zeros((4, r, c))


def qeye(n):
    e = np.zeros((4, n, n))
    e[0] = np.eye(n)
    return e


def qmatmul(P, Q):
    """Quaternion matrix product PQ (Sec. 2: i^2 = j^2 = k^2 = ijk = -1, associative and
    distributive, non-commutative).  Expanding (p_w + p_x i + p_y j + p_z k)(q_w + ...)
    with ij = k, jk = i, ki = j, ji = -k, kj = -i, ik = -j gives the four planes below.
    Pinned by the unit table (tests/golden/quaternion_units.txt), associativity, and by
    chi(PQ) = chi(P) chi(Q) with the independently built complex representation."""
    Pw, Px, Py, Pz = P
    Qw, Qx, Qy, Qz = Q
    w = Pw @ Qw - Px @ Qx - Py @ Qy - Pz @ Qz
    x = Pw @ Qx + Px @ Qw + Py @ Qz - Pz @ Qy
    y = Pw @ Qy - Px @ Qz + Py @ Qw + Pz @ Qx
    z = Pw @ Qz + Px @ Qy - Py @ Qx + Pz @ Qw
    return np.stack([w, x, y, z])


def qconjT(Q):
    """Conjugate transpose Q* = Q_w^T - Q_x^T i - Q_y^T j - Q_z^T k (Sec. 2)."""
    return np.stack([Q[0].T, -Q[1].T, -Q[2].T, -Q[3].T])


def qnorm(Q):
    """Frobenius norm: root-sum-square of the four planes (Sec. 2)."""
    return float(np.sqrt(np.sum(Q * Q)))


def _split(Q):
    """Q = Q_0 + Q_1 j with Q_0 = Q_w + Q_x i, Q_1 = Q_y + Q_z i (Sec. 2.2)."""
    return Q[0] + 1j * Q[1], Q[2] + 1j * Q[3]


def chi(Q):
    """Full complex representation chi_Q = [[Q_0, Q_1], [-conj(Q_1), conj(Q_0)]] (Sec. 2.2)."""
    Q0, Q1 = _split(Q)
    return np.block([[Q0, Q1], [-np.conj(Q1), np.conj(Q0)]])


def comp(Q):
    """Compact complex representation Q_c = [Q_0; -conj(Q_1)] in C^{2m x n} (Sec. 2.2)."""
    Q0, Q1 = _split(Q)
    return np.vstack([Q0, -np.conj(Q1)])


def from_comp(Z):
    """Inverse of ``comp``: the quaternion X with X_c = Z, i.e. X = Z_top - conj(Z_bot) j
    (Alg. 2 step 3; the same map builds H from U in Alg. 1 step 3)."""
    n = Z.shape[0] // 2
    X0 = Z[:n]
    X1 = -np.conj(Z[n:])
    return np.stack([X0.real, X0.imag, X1.real, X1.imag])


def upsilon(Q):
    """Real representation (Appendix B.1): the 4m x 4n block matrix
    [[w,-x,-y,-z],[x,w,-z,y],[y,z,w,-x],[z,-y,x,w]] acting on the stacked planes."""
    w, x, y, z = Q
    return np.block([[w, -x, -y, -z], [x, w, -z, y], [y, z, w, -x], [z, -y, x, w]])


def qpinv(A):
    """Moore-Penrose inverse through chi_{A^dagger} = (chi_A)^dagger (Sec. 2.2 lemma):
    the compact columns of pinv(chi_A) restricted to the first block column."""
    P = np.linalg.pinv(chi(A))          # 2n x 2m
    m = A.shape[1]
    # chi_{A^+} = [[X0, X1], [-conj X1, conj X0]]: its first m columns are (A^+)_c
    return from_comp(P[:, :m])


def qscalar_mul_chi(p, q):
    """Product of two quaternion scalars (length-4 arrays) through their 2x2 complex
    representation, an independent route used to check ``qmatmul``."""
    P = chi(np.asarray(p, dtype=float).reshape(4, 1, 1))
    Q = chi(np.asarray(q, dtype=float).reshape(4, 1, 1))
    R = P @ Q
    return np.array([R[0, 0].real, R[0, 0].imag, R[0, 1].real, R[0, 1].imag])
