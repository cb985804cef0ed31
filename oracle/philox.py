"""Counter-based random test matrices (oracle side).

The test matrices Omega (n x s) and Psi (l x m) are quaternion Gaussian (Definition of a
standard Gaussian quaternion matrix, Sec. 4.3: all entries of the four real planes i.i.d.
N(0,1)) or quaternion sub-Gaussian (Sec. 4.4; here Rademacher +-1 on each plane).  They
are drawn from Philox4x32-10, the counter-based generator published by Salmon, Moraes,
Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC'11), implemented here
from that definition.  The CUDA path implements the same published generator on its own;
the two share no code.

Element mapping (both sides): key = (seed mod 2^32, seed div 2^32); the quaternion entry at
row-major index e of the matrix drawn on stream ``t`` uses counter (e mod 2^32, e div 2^32,
t, 0).  Its four output words x0..x3 give the planes w, x, y, z:
  Gaussian   : Box-Muller on (x0, x1) -> (w, x) and on (x2, x3) -> (y, z), with
               u = (x + 1/2) 2^-32, r = sqrt(-2 ln u_a), (r cos 2 pi u_b, r sin 2 pi u_b);
  Rademacher : plane p is +1 if bit 31 of x_p is clear, else -1.
Test infrastructure only (see the package docstring).
"""
import numpy as np

EMB_GAUSSIAN = 0
EMB_RADEMACHER = 1
STREAM_OMEGA = 1
STREAM_PSI = 2
STREAM_PSVD_F = 3

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit counters; returns four uint32 arrays.

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key is bumped by
    the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3)]
    c = list(np.broadcast_arrays(*c))
    c = [v.copy() for v in c]
    ka, kb = int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF
    for r in range(10):
        if r:
            ka = (ka + _W0) & 0xFFFFFFFF
            kb = (kb + _W1) & 0xFFFFFFFF
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ np.uint64(ka), lo1, hi0 ^ c[3] ^ np.uint64(kb), lo0]
    return [v.astype(np.uint32) for v in c]


def _words(rows, cols, stream, seed, extra=0):
    e = np.arange(rows * cols, dtype=np.uint64)
    return philox4x32_10(e & _MASK, e >> np.uint64(32), np.uint64(stream), np.uint64(extra),
                         seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def _unit(x):
    return (x.astype(np.float64) + 0.5) * 2.0 ** -32


def draw_embedding(rows, cols, kind, stream, seed):
    """Quaternion test matrix of shape (4, rows, cols), FP64 values (see module docstring)."""
    x = _words(rows, cols, stream, seed)
    if kind == EMB_RADEMACHER:
        planes = [1.0 - 2.0 * (w >> np.uint32(31)).astype(np.float64) for w in x]
    elif kind == EMB_GAUSSIAN:
        planes = []
        for a, b in ((x[0], x[1]), (x[2], x[3])):
            r = np.sqrt(-2.0 * np.log(_unit(a)))
            t = 2.0 * np.pi * _unit(b)
            planes += [r * np.cos(t), r * np.sin(t)]
    else:
        raise ValueError("unknown embedding kind")
    return np.stack([p.reshape(rows, cols) for p in planes])


def draw_uniform_f(count, seed, call_index=0):
    """Scaling vector f_j ~ Uniform(0,1) + 1 of the pseudo-SVD bad-part repair (Sec. 3.2,
    eq. for H_b diag(f)); counter (j, 0, STREAM_PSVD_F, call_index), word x0."""
    j = np.arange(count, dtype=np.uint64)
    x = philox4x32_10(j & _MASK, j >> np.uint64(32), np.uint64(STREAM_PSVD_F),
                      np.uint64(call_index), seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return 1.0 + _unit(x[0])
