"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the CUDA-path binding's callers and the oracle's
callers.  It holds none of the method's arithmetic: it only builds input matrices A
(four real component planes) and names the sketch sizes of each workload.  The random
test matrices Omega and Psi are NOT drawn here: each side draws them from the published
Philox4x32-10 definition.

Quaternion matrices are numpy arrays of shape (4, rows, cols) (planes w, x, y, z).

Workloads (sizes from the paper's experiments, Sec. 5; synthetic stand-ins for data sets
that are not available):
  c1  512 x 384, FP64: A = U diag(0.5^i, i<=10) V* + 1e-6 E with quaternion Gaussian
      factors U (512x10), V (384x10) whose planes are N(0, 1/4) and noise E of the same
      law; k=10, s=21, l=43; Gaussian embeddings.
  c2  8192 x 8192, FP32: A = U diag(i^-2) V* with random quaternion-orthonormal U, V;
      the spectrum is truncated at R = 1024 (sigma_R = 9.5e-7; the dropped tail is
      1.7e-5 of ||A||_F); k=50, s=101, l=203; Gaussian embeddings.
  c4  a batch of 256 matrices, m, n ~ U[256, 4096] independently, k ~ U{8..64},
      s = 2k + 1, l = 2s + 1, sigma_j = exp(-j/8) on R = min(m, n, 320) columns (sigma_320 is
      4e-18, below FP32 resolution), FP32 data, Rademacher embeddings (make_c4_batch, built
      on the device: it is a throughput workload, its parity cases are smaller).
  ex51-{lrn,pds,eds}  the synthetic family of Sec. 5 (Example "syntheticData"): A = U Sigma V*,
      2000 x 1600, with Sigma = diag(1 (R times), 0, ...) + (xi / n) E (low rank plus noise,
      E a standard quaternion Gaussian), diag(1 (R times), 2^-p, 3^-p, ...) (polynomial
      decay) or diag(1 (R times), 10^-q, 10^-2q, ...) (exponential decay); the paper plots
      xi = 0.01, p = 2, q = 0.25 and does not state R (R = 10 here, the count of leading
      ones in the practical-sketching test matrices the example follows).
  c3  31365 x 27125 pure quaternion (real part 0), FP32, image-like: per channel (i, j, k)
      f(p, q) = sum_{t<64} a_t cos(2 pi (u_t p / m + v_t q / n) + phi_t) with integer
      frequencies u_t, v_t ~ U{0..8}, a_t ~ N(0, 1), phi_t ~ U[0, 2 pi), min-max rescaled to
      [0, 0.98], plus U(0, 0.02) noise; k=100, s=201, l=403; Rademacher embeddings
      (make_c3, built on the device).
  c5  2,097,152 x 256 pure quaternion (a 128^3 grid times 256 time steps; the velocity
      components are the i, j, k parts), FP32: 32 divergence-free Taylor-Green-type modes
      (A_x cos(a x) sin(b y) sin(c z), A_y sin(a x) cos(b y) sin(c z), 0) with integer
      wavenumbers a, b, c in 1..4 and A_x a + A_y b = 0, each turned by a random signed
      permutation of the axes (an orthogonal map of the periodic grid onto itself, which
      keeps the field divergence free), times a time-periodic amplitude
      alpha_t sin(2 pi tau / T_t + phi_t), plus 1e-4 Gaussian noise; k=20, s=41, l=83;
      Gaussian embeddings (make_c5, built on the device).
  lorenz  20000 x 10000 full quaternion, FP32: the states x + y i + z j + w k of the paper's
      4D Lorenz-type system (Sec. 5; a = 15, b = 2, c = 28) along 10000 trajectories from
      initial states on the sphere of radius 20, after each of 20000 fourth-order
      Runge-Kutta steps of dt = 1e-3 (t in (0, 20]; the paper's solver steps are not stated),
      integrated on the GPU (qs_lorenz4d) in FP64; k=100, s=201, l=403; Gaussian embeddings.
Random quaternion-orthonormal factors are built as U = D Q W: Q real orthonormal (QR of a
real Gaussian), W the unitary polar factor of an R x R quaternion Gaussian (from the
eigendecomposition of its Hermitian complex form), D a diagonal of random unit
quaternions.  Each factor is unitary, hence so is the product.  For the large square
factors of the Sec. 5 family the polar factor is replaced by a second real orthogonal
factor and unit-quaternion diagonal, U = D1 Q1 D2 Q2 (also unitary; the eigendecomposition
of a 3200 x 3200 complex matrix would take most of a minute).
"""
import numpy as np

WORKLOADS = {
    "c1": dict(m=512, n=384, k=10, s=21, l=43, precision="fp64", emb="gaussian", seed=0),
    "c2": dict(m=8192, n=8192, k=50, s=101, l=203, precision="bf16x3", emb="gaussian",
               seed=0, rank_cap=1024),
    # batch: m, n ~ U[256, 4096], k ~ U{8..64}, s = 2k + 1, l = 2s + 1, sigma_j = exp(-j/8)
    # on R = min(m, n, 320) columns, Rademacher embeddings, split-BF16 sketch
    "c4": dict(count=256, lo=256, hi=4096, k_lo=8, k_hi=64, rank_cap=320, precision="bf16x3",
               emb="rademacher", seed=0),
    # image-like pure quaternion (the colour-image experiment's shape), Rademacher embeddings
    "c3": dict(m=31365, n=27125, k=100, s=201, l=403, precision="bf16x3", emb="rademacher",
               seed=0, pure=True, modes=64),
    # hyperchaotic-system snapshots: 20000 time instances x 10000 initial states (RK4, dt 1e-3)
    "lorenz": dict(m=20000, n=10000, k=100, s=201, l=403, precision="bf16x3", emb="gaussian",
                   seed=0, dt=1e-3, a=15.0, b=2.0, c=28.0, radius=20.0),
    # tall flow-snapshot pure quaternion (128^3 grid x 256 time steps), Gaussian embeddings
    "c5": dict(m=128 ** 3, n=256, k=20, s=41, l=83, precision="bf16x3", emb="gaussian", seed=0,
               pure=True, grid=128, modes=32),
}


def _qmul_planes(P, Q):
    # entrywise product of quaternion arrays (broadcasting), used only to apply the
    # unit-quaternion diagonal when building inputs
    pw, px, py, pz = P
    qw, qx, qy, qz = Q
    return np.stack([pw * qw - px * qx - py * qy - pz * qz,
                     pw * qx + px * qw + py * qz - pz * qy,
                     pw * qy - px * qz + py * qw + pz * qx,
                     pw * qz + px * qy - py * qx + pz * qw])


def _unitary_quaternion(rng, R):
    """Polar factor of an R x R quaternion Gaussian G: W = G (G*G)^{-1/2}, computed on the
    2R x 2R complex form [[G0, G1], [-conj G1, conj G0]]; W is read back from its first
    block column."""
    G = rng.standard_normal((4, R, R))
    G0, G1 = G[0] + 1j * G[1], G[2] + 1j * G[3]
    C = np.block([[G0, G1], [-np.conj(G1), np.conj(G0)]])
    lam, V = np.linalg.eigh(C.conj().T @ C)
    P = C @ (V * (1.0 / np.sqrt(lam))[None, :]) @ V.conj().T
    W0, W1 = P[:R, :R], P[:R, R:]
    return np.stack([W0.real, W0.imag, W1.real, W1.imag])


def random_orthonormal(rng, m, R):
    """Random m x R quaternion matrix with orthonormal columns, U = D Q W."""
    Q, _ = np.linalg.qr(rng.standard_normal((m, R)))
    W = _unitary_quaternion(rng, R)
    QW = np.stack([Q @ W[p] for p in range(4)])
    d = rng.standard_normal((4, m, 1))
    d /= np.sqrt(np.sum(d * d, axis=0, keepdims=True))
    return _qmul_planes(d, QW)


def _unit_diag(rng, m):
    d = rng.standard_normal((4, m, 1))
    return d / np.sqrt(np.sum(d * d, axis=0, keepdims=True))


def random_orthonormal_fast(rng, m, R):
    """Random m x R quaternion matrix with orthonormal columns, U = D1 Q1 D2 Q2 (Q1 m x R
    real orthonormal, Q2 R x R real orthogonal, D1, D2 diagonals of unit quaternions)."""
    Q1, _ = np.linalg.qr(rng.standard_normal((m, R)))
    Q2, _ = np.linalg.qr(rng.standard_normal((R, R)))
    D1Q1 = _qmul_planes(_unit_diag(rng, m), np.broadcast_to(Q1, (4, m, R)) * np.array([1.0, 0, 0, 0])[:, None, None])
    T = _qmul_planes(D1Q1, _unit_diag(rng, R).transpose(0, 2, 1))     # D1 Q1 D2 (column scaling)
    return np.stack([T[p] @ Q2 for p in range(4)])


def _qprod(P, Q):
    """Quaternion matrix product P Q (plane form), for building inputs."""
    return np.stack([P[0] @ Q[0] - P[1] @ Q[1] - P[2] @ Q[2] - P[3] @ Q[3],
                     P[0] @ Q[1] + P[1] @ Q[0] + P[2] @ Q[3] - P[3] @ Q[2],
                     P[0] @ Q[2] - P[1] @ Q[3] + P[2] @ Q[0] + P[3] @ Q[1],
                     P[0] @ Q[3] + P[1] @ Q[2] - P[2] @ Q[1] + P[3] @ Q[0]])


def make_ex51(kind, m=2000, n=1600, R=10, xi=0.01, p=2.0, q=0.25, seed=0, dtype=np.float64):
    """The Sec. 5 synthetic family (m >= n): kind "lrn" (low rank plus noise), "pds"
    (polynomial decay) or "eds" (exponential decay); A = U Sigma V* with U (m x n), V (n x n)
    random quaternion-orthonormal."""
    rng = np.random.default_rng(seed)
    U = random_orthonormal_fast(rng, m, n)
    V = random_orthonormal_fast(rng, n, n)
    tail = np.arange(1, n - R + 1, dtype=np.float64)
    if kind == "lrn":
        Sig = (xi / n) * rng.standard_normal((4, n, n))
        Sig[0, np.arange(R), np.arange(R)] += 1.0
        Vt = np.stack([V[0].T, -V[1].T, -V[2].T, -V[3].T])
        return _qprod(_qprod(U, Sig), Vt).astype(dtype)
    if kind == "pds":
        sigma = np.concatenate([np.ones(R), (tail + 1.0) ** (-p)])
    elif kind == "eds":
        sigma = np.concatenate([np.ones(R), 10.0 ** (-q * tail)])
    else:
        raise ValueError(kind)
    return _assemble(U, sigma, V, dtype=dtype)


def _assemble(U, sigma, V, device=None, dtype=np.float64):
    """A = U diag(sigma) V* (quaternion).  With a torch ``device`` the product runs there in
    FP64 (untimed input construction); otherwise in numpy."""
    Us = U * sigma[None, None, :]
    Vt = np.stack([V[0].T, -V[1].T, -V[2].T, -V[3].T])
    if device is not None:
        import torch
        a = torch.as_tensor(Us, device=device)
        b = torch.as_tensor(Vt, device=device)
        w = a[0] @ b[0] - a[1] @ b[1] - a[2] @ b[2] - a[3] @ b[3]
        x = a[0] @ b[1] + a[1] @ b[0] + a[2] @ b[3] - a[3] @ b[2]
        y = a[0] @ b[2] - a[1] @ b[3] + a[2] @ b[0] + a[3] @ b[1]
        z = a[0] @ b[3] + a[1] @ b[2] - a[2] @ b[1] + a[3] @ b[0]
        tdt = torch.float64 if dtype == np.float64 else torch.float32
        return torch.stack([w, x, y, z]).to(tdt).contiguous()
    Aw = Us[0] @ Vt[0] - Us[1] @ Vt[1] - Us[2] @ Vt[2] - Us[3] @ Vt[3]
    Ax = Us[0] @ Vt[1] + Us[1] @ Vt[0] + Us[2] @ Vt[3] - Us[3] @ Vt[2]
    Ay = Us[0] @ Vt[2] - Us[1] @ Vt[3] + Us[2] @ Vt[0] + Us[3] @ Vt[1]
    Az = Us[0] @ Vt[3] + Us[1] @ Vt[2] - Us[2] @ Vt[1] + Us[3] @ Vt[0]
    return np.stack([Aw, Ax, Ay, Az]).astype(dtype)


def make_c1(seed=0, m=512, n=384, rank=10, noise=1e-6):
    """c1: quaternion-Gaussian factors with N(0,1/4) planes, sigma_i = 0.5^i (i <= rank),
    plus ``noise`` times a quaternion Gaussian with N(0,1/4) planes.  FP64."""
    rng = np.random.default_rng(seed)
    U = 0.5 * rng.standard_normal((4, m, rank))
    V = 0.5 * rng.standard_normal((4, n, rank))
    sigma = 0.5 ** np.arange(1, rank + 1)
    A = _assemble(U, sigma, V)
    return A + noise * 0.5 * rng.standard_normal((4, m, n))


def make_decay(m, n, seed=0, rank_cap=1024, power=2.0, device=None, dtype=np.float32):
    """c2-type: A = U diag(i^-power) V* with random quaternion-orthonormal U, V and the
    spectrum truncated at R = min(m, n, rank_cap)."""
    rng = np.random.default_rng(seed)
    R = min(m, n, rank_cap)
    U = random_orthonormal(rng, m, R)
    V = random_orthonormal(rng, n, R)
    sigma = np.arange(1, R + 1, dtype=np.float64) ** (-power)
    return _assemble(U, sigma, V, device=device, dtype=dtype)


def make_lowrank(m, n, rank, seed=0, dtype=np.float64):
    """Exactly rank-``rank`` quaternion matrix (product of two quaternion Gaussians)."""
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((4, m, rank))
    V = rng.standard_normal((4, n, rank))
    return _assemble(U, np.ones(rank), V, dtype=dtype)


def make_gaussian(m, n, seed=0, dtype=np.float64):
    """Quaternion Gaussian with N(0,1) planes."""
    return np.random.default_rng(seed).standard_normal((4, m, n)).astype(dtype)


def make_c4_batch(device, spec=None):
    """The c4 batch on a torch device: list of (m, n, k, A) with A a (4, m, n) FP32 tensor
    (leading dimension padded to a multiple of 4), A = U diag(exp(-j/8)) V* with
    U = D1 Q1 D2 Q2-type quaternion-orthonormal factors drawn with torch on the device."""
    import torch
    spec = dict(WORKLOADS["c4"], **(spec or {}))
    rng = np.random.default_rng(spec["seed"])
    gen = torch.Generator(device=device)
    gen.manual_seed(int(spec["seed"]))
    dt = torch.float64

    def unit(shape):
        d = torch.randn((4,) + shape, generator=gen, device=device, dtype=dt)
        return d / torch.sqrt((d * d).sum(0, keepdim=True))

    def qm(a, b):   # entrywise Hamilton product with broadcasting (diagonal scalings)
        return torch.stack([a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
                            a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                            a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1],
                            a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0]])

    def orth(rows, R):
        Q1 = torch.linalg.qr(torch.randn((rows, R), generator=gen, device=device, dtype=dt)).Q
        Q2 = torch.linalg.qr(torch.randn((R, R), generator=gen, device=device, dtype=dt)).Q
        real = torch.stack([Q1, torch.zeros_like(Q1), torch.zeros_like(Q1), torch.zeros_like(Q1)])
        T = qm(qm(unit((rows, 1)), real), unit((1, R)))       # D1 Q1 D2
        return torch.stack([T[p] @ Q2 for p in range(4)])

    out = []
    for _ in range(spec["count"]):
        m, n = (int(v) for v in rng.integers(spec["lo"], spec["hi"] + 1, size=2))
        k = int(rng.integers(spec["k_lo"], spec["k_hi"] + 1))
        R = min(m, n, spec["rank_cap"])
        # factors in FP64, the product in FP32 (the data's precision; FP64 matrix products
        # would dominate the set-up on a GPU whose FP64 rate is low)
        U = (orth(m, R) * torch.exp(-torch.arange(1, R + 1, device=device, dtype=dt) / 8.0)).float()
        V = orth(n, R).float()
        Vt = torch.stack([V[0].T, -V[1].T, -V[2].T, -V[3].T])
        w = U[0] @ Vt[0] - U[1] @ Vt[1] - U[2] @ Vt[2] - U[3] @ Vt[3]
        x = U[0] @ Vt[1] + U[1] @ Vt[0] + U[2] @ Vt[3] - U[3] @ Vt[2]
        y = U[0] @ Vt[2] - U[1] @ Vt[3] + U[2] @ Vt[0] + U[3] @ Vt[1]
        z = U[0] @ Vt[3] + U[1] @ Vt[2] - U[2] @ Vt[1] + U[3] @ Vt[0]
        buf = torch.zeros((4, m, (n + 3) // 4 * 4), dtype=torch.float32, device=device)
        buf[:, :, :n] = torch.stack([w, x, y, z])
        out.append((m, n, k, buf[:, :, :n]))
    return out


def _pad4(n):
    return (n + 3) // 4 * 4


def make_c3(device, m=None, n=None, seed=None, modes=None, rows=None):
    """c3 (image-like pure quaternion) on a torch device: a (3, m, ldd) FP32 tensor holding the
    i, j, k planes (ldd = n rounded up to a multiple of 4), viewed as (3, m, n); the real
    plane is zero and not stored.  Smaller m, n give shape classes with the same structure;
    ``rows`` keeps only the first rows of the m-row image (rescaled on those rows)."""
    import torch
    spec = WORKLOADS["c3"]
    m = spec["m"] if m is None else m
    n = spec["n"] if n is None else n
    seed = spec["seed"] if seed is None else seed
    modes = spec["modes"] if modes is None else modes
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) + 1)
    mr = m if rows is None else min(rows, m)
    buf = torch.empty((3, mr, _pad4(n)), dtype=torch.float32, device=device)
    p = torch.arange(mr, device=device, dtype=torch.float64) / m
    q = torch.arange(n, device=device, dtype=torch.float64) / n
    for ch in range(3):
        u = torch.as_tensor(rng.integers(0, 9, modes), device=device, dtype=torch.float64)
        v = torch.as_tensor(rng.integers(0, 9, modes), device=device, dtype=torch.float64)
        a = torch.as_tensor(rng.standard_normal(modes), device=device)
        phi = torch.as_tensor(rng.uniform(0.0, 2.0 * np.pi, modes), device=device)
        alpha = 2.0 * np.pi * p[:, None] * u[None, :] + phi[None, :]       # m x modes
        beta = 2.0 * np.pi * q[:, None] * v[None, :]                       # n x modes
        # cos(alpha + beta) = cos alpha cos beta - sin alpha sin beta: a rank-2 modes product
        L = torch.cat([a * torch.cos(alpha), -a * torch.sin(alpha)], 1).float()
        Rt = torch.cat([torch.cos(beta), torch.sin(beta)], 1).float()
        f = buf[ch, :, :n]
        torch.matmul(L, Rt.T, out=f) if f.is_contiguous() else f.copy_(L @ Rt.T)
        lo, hi = f.min(), f.max()
        f.sub_(lo).mul_(0.98 / (hi - lo))
        f.add_(torch.rand((mr, n), generator=gen, device=device, dtype=torch.float32).mul_(0.02))
    return buf[:, :, :n]


def make_c5(device, grid=None, steps=None, seed=None, modes=None):
    """c5 (tall flow snapshots, pure quaternion) on a torch device: a (3, grid^3, steps) FP32
    tensor with the i, j, k planes (velocity components); rows are grid points (x slowest),
    columns are time steps.  The real plane is zero and not stored."""
    import torch
    spec = WORKLOADS["c5"]
    grid = spec["grid"] if grid is None else grid
    steps = spec["n"] if steps is None else steps
    seed = spec["seed"] if seed is None else seed
    modes = spec["modes"] if modes is None else modes
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) + 1)
    x = 2.0 * np.pi * torch.arange(grid, device=device, dtype=torch.float64) / grid
    m = grid ** 3
    U = torch.empty((3, m, modes), dtype=torch.float32, device=device)
    for t in range(modes):
        a, b, c = (int(v) for v in rng.integers(1, 5, 3))
        nrm = np.hypot(a, b)
        ax, ay = b / nrm, -a / nrm                       # ax a + ay b = 0: divergence free
        fx = [torch.cos(a * x), torch.sin(b * x), torch.sin(c * x)]
        fy = [torch.sin(a * x), torch.cos(b * x), torch.sin(c * x)]
        comp = [ax * fx[0][:, None, None] * fx[1][None, :, None] * fx[2][None, None, :],
                ay * fy[0][:, None, None] * fy[1][None, :, None] * fy[2][None, None, :],
                torch.zeros((grid, grid, grid), device=device, dtype=torch.float64)]
        # random signed permutation P of the axes: v(x) = P u(P^T x)
        perm = rng.permutation(3)
        sign = rng.choice([-1.0, 1.0], 3)
        field = torch.stack(comp)                         # (3, gx, gy, gz), u(x)
        for d in range(3):                                # u(P^T x): reflect, then permute axes
            if sign[d] < 0:
                field = torch.roll(torch.flip(field, dims=[1 + d]), shifts=1, dims=1 + d)
        field = field.permute(0, *(1 + int(np.argsort(perm)[e]) for e in range(3)))
        newf = torch.empty_like(field)
        for d in range(3):                                # components: (P u)_perm[d] = sign[d] u_d
            newf[int(perm[d])] = sign[d] * field[d]
        U[:, :, t] = newf.reshape(3, m).float()
    tau = torch.arange(steps, device=device, dtype=torch.float64)
    amp = torch.empty((modes, steps), device=device, dtype=torch.float64)
    for t in range(modes):
        alpha = (0.5 + rng.uniform()) * 0.85 ** t
        period = rng.uniform(16.0, 256.0)
        amp[t] = alpha * torch.sin(2.0 * np.pi * tau / period + rng.uniform(0.0, 2.0 * np.pi))
    A = torch.empty((3, m, steps), dtype=torch.float32, device=device)
    ampf = amp.float()
    for ch in range(3):
        torch.matmul(U[ch], ampf, out=A[ch])
        A[ch].add_(torch.randn((m, steps), generator=gen, device=device, dtype=torch.float32).mul_(1e-4))
    return A


def lorenz_initial_states(cols, seed=0, radius=20.0):
    """(4, cols) FP64 initial states (x, y, z, w) drawn uniformly on the sphere of the given
    radius (normalised Gaussian vectors), as in the paper's hyperchaotic-system example."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((4, cols))
    return radius * u / np.linalg.norm(u, axis=0, keepdims=True)
