"""Parity at the full sizes the bench times, in the bench's launch configuration.

c2 (8192 x 8192 quaternion A, FP32 planes, sigma_i = i^-2, s = 101, l = 203, Gaussian test
matrices, split-BF16 sketch, pseudo-QR with three corrections): the whole path against the
FP64 oracle on the same input values and test matrices -- the sketches element by element
(1e-5 relative Frobenius, the split-BF16 tolerance), R(H) = R(Y) for the GPU's own Y (1e-6:
H is stored in FP32), kappa(H) < 10 after the corrections, and the final relative error
within 1e-3 of the oracle's (the bar of the 2048 x 2048 shape class; the sketch error moves
it by ~4e-6).

c3 (31365 x 27125 pure quaternion image, Rademacher, s = 201, l = 403) and c5 (2,097,152 x
256 pure quaternion flow snapshots, Gaussian, s = 41, l = 83), split-BF16 sketch, pseudo-QR
with three corrections, double-float stages: the oracle cannot afford the dense products at
these sizes, so it checks what it can compute exactly -- 256 sampled rows of Y and sampled
columns of W (rows of Y and columns of W are independent: 1e-5), the rangefinder on the
GPU's own Y (H element by element at 100 u_df kappa(Y)^2, the sensitivity of the correction
parameters; H X on sampled rows, which depends only on the range of H, at 100 u_df kappa(Y)),
X = (Psi H)^dagger W on the GPU's own H, W and exported Psi (10 sqrt(m) u_df kappa(Psi H):
Psi H sums m terms), and the error pass against the oracle's error of the same
factors (c5: all rows; c3: a 2048-row block through the allocation-free entry point, and the
whole matrix against an FP64 torch evaluation, within the split-BF16 bound of the error pass).

c4 (256 matrices, m, n ~ U[256, 4096], the batched call: persistent launches of 32 matrices):
every matrix's sketches equal its own single-matrix update (1e-6: only the order of the L2
reductions differs), and a sample of matrices (the largest, the smallest, one in between)
equals the oracle's sketch (1e-5).
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


def test_c2_full_size_whole_path(pkg):
    w = WL.WORKLOADS["c2"]
    m, n, s, l, seed = w["m"], w["n"], w["s"], w["l"], w["seed"]
    Ad = WL.make_decay(m, n, seed=seed, rank_cap=w["rank_cap"], device="cuda",
                       dtype=np.float32).contiguous()
    qs = pkg.QSketch(m, n, s, l, emb="gaussian", prec="bf16x3", seed=seed)
    qs.reset(seed=seed)
    qs.update(Ad, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    err = float(qs.error(Ad).item())
    assert qs.device_status() == 0
    Y = qs.get("Y").cpu().double().numpy()
    W = qs.get("W").cpu().double().numpy()
    H = qs.get("H").cpu().double().numpy()
    A = Ad.double().cpu().numpy()
    del Ad
    Om = O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, seed)
    Psi = O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, seed)
    ref = O.onepass(A, Om, Psi, "pseudo_qr", 3)
    assert rel(Y, ref["Y"]) < 1e-5
    assert rel(W, ref["W"]) < 1e-5
    CH, CY = O.chi(H), O.chi(Y)
    Qh, _ = np.linalg.qr(CH)
    assert np.linalg.norm(CY - Qh @ (Qh.conj().T @ CY)) / np.linalg.norm(CY) < 1e-6
    sv = np.linalg.svd(CH, compute_uv=False)
    assert sv[0] / sv[-1] < 10
    assert abs(err - ref["err"]) <= 1e-3 * ref["err"], (err, ref["err"])


def test_c4_full_batch(pkg):
    spec = WL.WORKLOADS["c4"]
    batch = WL.make_c4_batch("cuda")
    sk, sk1, mats, shapes = [], [], [], []
    for i, (m, n, k, A) in enumerate(batch):
        s = 2 * k + 1
        l = min(2 * s + 1, m, n)
        kw = dict(emb=spec["emb"], prec="bf16x3", seed=spec["seed"] + i)
        sk.append(pkg.QSketch(m, n, s, l, **kw))
        sk1.append(pkg.QSketch(m, n, s, l, **kw))
        mats.append(A)
        shapes.append((m, n, s, l))
    pkg.update_batched(sk, mats)
    for q, A in zip(sk1, mats):
        q.update(A, theta=0.0)
    torch.cuda.synchronize()
    for i in range(len(sk)):
        assert sk[i].device_status() == 0
        assert rel(sk[i].get("Y").cpu().numpy(), sk1[i].get("Y").cpu().numpy()) < 1e-6, i
        assert rel(sk[i].get("W").cpu().numpy(), sk1[i].get("W").cpu().numpy()) < 1e-6, i
    sizes = [m * n for m, n, _, _ in shapes]
    sample = {int(np.argmax(sizes)), int(np.argmin(sizes)), len(sk) // 2}
    for i in sorted(sample):
        m, n, s, l = shapes[i]
        A = mats[i].double().cpu().numpy()
        Om = O.draw_embedding(n, s, O.EMB_RADEMACHER, O.STREAM_OMEGA, spec["seed"] + i)
        Psi = O.draw_embedding(l, m, O.EMB_RADEMACHER, O.STREAM_PSI, spec["seed"] + i)
        Yr, Wr = O.sketch(A, Om, Psi)
        assert rel(sk[i].get("Y").cpu().numpy(), Yr) < 1e-5, i
        assert rel(sk[i].get("W").cpu().numpy(), Wr) < 1e-5, i


UDF = 2.0 ** -48
_PLANE = [[0, 1, 2, 3], [1, 0, 3, 2], [2, 3, 0, 1], [3, 2, 1, 0]]


def _np4(planes):
    """FP64 numpy (4, r, c) of a plane list (None = zero plane)."""
    ref = next(p for p in planes if p is not None)
    return np.stack([np.zeros(tuple(ref.shape)) if p is None else p.double().cpu().numpy()
                     for p in planes])


def _kappa(Y):
    """kappa(Y) from the eigenvalues of chi(Y* Y) (the Gram, 2s x 2s)."""
    ev = np.linalg.eigvalsh(O.chi(O.qmatmul(O.qconjT(Y), Y)))
    return float(np.sqrt(ev[-1] / max(ev[0], 1e-300)))


def _tall_whole_path_checks(pkg, name, planes, chunk):
    w = WL.WORKLOADS[name]
    m, n, s, l, seed = w["m"], w["n"], w["s"], w["l"], w["seed"]
    qs = pkg.QSketch(m, n, s, l, emb=w["emb"], prec="bf16x3", seed=seed, pure=True)
    qs.update(planes, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    err = float(qs.error(planes).item())
    torch.cuda.synchronize()
    assert qs.device_status() == 0
    Om = qs.get("Omega").cpu().double().numpy()
    rng = np.random.default_rng(1)
    # sketches on sampled rows of Y and columns of W
    rows = np.sort(rng.choice(m, 256, replace=False))
    ncol = min(256, n) if name == "c3" else 32
    cols = np.sort(rng.choice(n, ncol, replace=False))
    rows_t = torch.as_tensor(rows, device="cuda")
    cols_t = torch.as_tensor(cols, device="cuda")
    Ar = _np4([None if p is None else p.index_select(0, rows_t) for p in planes])
    Yg = qs.get("Y")
    assert rel(Yg[:, rows_t, :].cpu().double().numpy(), O.qmatmul(Ar, Om)) < 1e-5
    Wref = np.zeros((4, l, ncol))
    Psi_d = qs.get("Psi")
    for r0 in range(0, m, chunk):   # W[:, cols] = sum over row chunks of Psi[:, chunk] A[chunk, cols]
        r1 = min(m, r0 + chunk)
        Ac = _np4([None if p is None else p[r0:r1].index_select(1, cols_t) for p in planes])
        Wref += O.qmatmul(Psi_d[:, :, r0:r1].cpu().double().numpy(), Ac)
    assert rel(qs.get("W")[:, :, cols_t].cpu().double().numpy(), Wref) < 1e-5
    # rangefinder on the GPU's own Y; QB stage on the GPU's own H, W and Psi
    Y = Yg.cpu().double().numpy()
    H = qs.get("H").cpu().numpy()
    Href = O.pseudo_qr(Y, 3)
    kap = _kappa(Y)
    # H itself carries the sensitivity of eps_1 (u kappa(G_0) = u kappa(Y)^2, see the precision
    # tests); its range does not, and H X is basis invariant (Lemma HToQ): H X on sampled rows
    # against the oracle's H_ref X_ref at 100 u kappa(Y)
    dh = float(np.abs(H - Href).max() / np.abs(Href).max())
    assert dh <= max(1e-12, 100 * UDF * kap ** 2), (dh, kap)
    assert _kappa(H) < 10
    del Y
    W = qs.get("W").cpu().double().numpy()
    P = np.zeros((4, l, s))
    Pref = np.zeros((4, l, s))
    for r0 in range(0, m, chunk):
        r1 = min(m, r0 + chunk)
        Pc = Psi_d[:, :, r0:r1].cpu().double().numpy()
        P += O.qmatmul(Pc, H[:, r0:r1])
        Pref += O.qmatmul(Pc, Href[:, r0:r1])
    X = qs.get("X").cpu().numpy()
    Xref = O.qls_solve(P, W)
    # P = Psi H sums m terms per entry: rounding ~ sqrt(m) u_df relative, which X carries
    # times kappa(P)
    bar_x = max(1e-12, 10 * np.sqrt(m) * UDF * _kappa(P))
    assert rel(X, Xref) <= bar_x, (rel(X, Xref), bar_x)
    HXr = O.qmatmul(H[:, rows], X)
    HXr_ref = O.qmatmul(Href[:, rows], O.qls_solve(Pref, W))
    assert rel(HXr, HXr_ref) <= max(1e-12, 100 * UDF * kap), (rel(HXr, HXr_ref), kap)
    del Href
    return qs, err, H, X


def test_c5_full_size_whole_path(pkg):
    P3 = WL.make_c5("cuda")
    planes = [None, P3[0], P3[1], P3[2]]
    qs, err, H, X = _tall_whole_path_checks(pkg, "c5", planes, chunk=1 << 18)
    m = WL.WORKLOADS["c5"]["m"]
    num = den = 0.0                    # the oracle's error of the GPU's own factors, all rows
    bound = 0.0
    for r0 in range(0, m, 1 << 18):
        r1 = min(m, r0 + (1 << 18))
        Ac = _np4([None if p is None else p[r0:r1] for p in planes])
        Hc = H[:, r0:r1]
        num += O.qnorm(Ac - O.qmatmul(Hc, X)) ** 2
        den += O.qnorm(Ac) ** 2
        M = np.stack([sum(np.abs(Hc[_PLANE[q][b]]) @ np.abs(X[b]) for b in range(4)) for q in range(4)])
        bound += np.linalg.norm(M) ** 2
    exact = np.sqrt(num / den)
    tol = 2.0 ** -15 * np.sqrt(bound / den) + 1e-12   # split-BF16 H X in the error pass
    assert abs(err - exact) <= tol, (err, exact, tol)


def test_c3_full_size_whole_path(pkg):
    P3 = WL.make_c3("cuda")
    planes = [None, P3[0], P3[1], P3[2]]
    qs, err, H, X = _tall_whole_path_checks(pkg, "c3", planes, chunk=1 << 14)
    # error pass: a 2048-row block through the allocation-free SIMT entry point against the
    # oracle, then the whole matrix against that entry point
    Hg32 = qs.get("H").float()
    Xg32 = qs.get("X").float()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    blk = [None] + [p[:2048] for p in planes[1:]]
    r_blk = float(pkg.reconstruct_error_static(blk, Hg32[:, :2048], Xg32, out).item())
    Ab = _np4(blk)
    Hb = Hg32[:, :2048].double().cpu().numpy()
    X32 = Xg32.double().cpu().numpy()
    exact_blk = O.rel_error(Ab, Hb, X32)
    s = WL.WORKLOADS["c3"]["s"]
    M = np.stack([sum(np.abs(Hb[_PLANE[q][b]]) @ np.abs(X32[b]) for b in range(4)) for q in range(4)])
    tol_blk = 2 * s * 2.0 ** -24 * np.linalg.norm(M) / O.qnorm(Ab)
    assert abs(r_blk - exact_blk) <= tol_blk, (r_blk, exact_blk, tol_blk)
    # the whole matrix: ||A - H X||_F in FP64 with torch (row blocks), against the tensor-core
    # pass, whose H X from BF16 hi/lo pairs is within 2^-15 |H||X| per Hamilton term; bounded
    # here through ||(|H||X|)_q||_F <= sum_b ||H_{q,b}||_F ||X_b||_F
    Hd, Xd = qs.get("H"), qs.get("X")
    num = den = 0.0
    for r0 in range(0, Hd.shape[1], 4096):
        r1 = min(Hd.shape[1], r0 + 4096)
        hb = Hd[:, r0:r1]
        prod = [hb[0] @ Xd[0] - hb[1] @ Xd[1] - hb[2] @ Xd[2] - hb[3] @ Xd[3],
                hb[0] @ Xd[1] + hb[1] @ Xd[0] + hb[2] @ Xd[3] - hb[3] @ Xd[2],
                hb[0] @ Xd[2] - hb[1] @ Xd[3] + hb[2] @ Xd[0] + hb[3] @ Xd[1],
                hb[0] @ Xd[3] + hb[1] @ Xd[2] - hb[2] @ Xd[1] + hb[3] @ Xd[0]]
        for q in range(4):
            a = planes[q][r0:r1].double() if planes[q] is not None else torch.zeros_like(prod[q])
            num += float(((a - prod[q]) ** 2).sum())
            den += float((a * a).sum())
    exact = np.sqrt(num / den)
    hn = [float(torch.linalg.norm(Hd[p])) for p in range(4)]
    xn = [float(torch.linalg.norm(Xd[p])) for p in range(4)]
    bnd = np.sqrt(sum(sum(hn[_PLANE[q][b]] * xn[b] for b in range(4)) ** 2 for q in range(4)))
    tol = 2.0 ** -15 * bnd / np.sqrt(den) + 1e-12
    assert abs(err - exact) <= tol, (err, exact, tol)
