"""Parity at the full sizes the bench times, in the bench's launch configuration.

c2 (8192 x 8192 quaternion A, FP32 planes, sigma_i = i^-2, s = 101, l = 203, Gaussian test
matrices, split-BF16 sketch, pseudo-QR with three corrections): the whole path against the
FP64 oracle on the same input values and test matrices -- the sketches element by element
(1e-5 relative Frobenius, the split-BF16 tolerance), R(H) = R(Y) for the GPU's own Y (1e-6:
H is stored in FP32), kappa(H) < 10 after the corrections, and the final relative error
within 1e-3 of the oracle's (the bar of the 2048 x 2048 shape class; the sketch error moves
it by ~4e-6).

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
