"""GPU parity of the fused tcgen05 sketch (BF16 and split-BF16) against the FP64 oracle.

Tolerances (relative Frobenius): split-BF16 (3 products, FP32 accumulation) 1e-5; plain
BF16 8e-3 (A and the test matrices rounded to 8 significant bits).  The oracle draws the
test matrices from its own Philox4x32-10; the GPU draws in FP32 arithmetic, within 2e-6
of the oracle's values, far inside both tolerances.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
import workloads as WL

TOL = {"bf16x3": 1e-5, "bf16": 8e-3}


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


def _dev(A):
    """Device copy of A whose row pitch is padded to a multiple of 4 elements (the TMA
    path needs 16-byte row pitches); returns the (4, m, n) view."""
    m, n = A.shape[1], A.shape[2]
    buf = torch.zeros((4, m, (n + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    buf[:, :, :n] = torch.as_tensor(A, device="cuda")
    return buf[:, :, :n]


def _emb(n, s, l, m, seed, kind=O.EMB_GAUSSIAN):
    return (O.draw_embedding(n, s, kind, O.STREAM_OMEGA, seed),
            O.draw_embedding(l, m, kind, O.STREAM_PSI, seed))


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("shape", [(256, 128, 21, 43), (300, 257, 13, 29), (128, 64, 1, 1),
                                   (1000, 700, 101, 203), (129, 200, 16, 128),
                                   # s > 128: single-plane Y waves with Omega in two row halves;
                                   # l > 256: three and four 128-row slices of Psi
                                   (600, 500, 201, 403), (320, 300, 140, 290), (300, 260, 256, 256)])
def test_tc_sketch_parity(pkg, prec, shape):
    m, n, s, l = shape
    A = WL.make_gaussian(m, n, seed=m * 7 + n).astype(np.float32)
    qs = pkg.QSketch(m, n, s, l, emb="gaussian", prec=prec, seed=5)
    Ad = _dev(A)
    qs.update(Ad, theta=0.0)
    torch.cuda.synchronize()
    assert qs.device_status() == 0
    Om, Psi = _emb(n, s, l, m, 5)
    Y, W = O.sketch(A.astype(np.float64), Om, Psi)
    assert rel(qs.get("Y").cpu().numpy(), Y) < TOL[prec]
    assert rel(qs.get("W").cpu().numpy(), W) < TOL[prec]


def test_tc_rademacher_and_repeat(pkg):
    """Rademacher test matrices are exact in BF16; a second update with theta = 0 overwrites."""
    m, n, s, l = 384, 320, 17, 35
    A = WL.make_gaussian(m, n, seed=2).astype(np.float32)
    qs = pkg.QSketch(m, n, s, l, emb="rademacher", prec="bf16x3", seed=9)
    Ad = torch.as_tensor(A, device="cuda")
    qs.update(Ad, theta=0.0)
    qs.update(Ad, theta=0.0)
    Om, Psi = _emb(n, s, l, m, 9, O.EMB_RADEMACHER)
    Y, W = O.sketch(A.astype(np.float64), Om, Psi)
    assert rel(qs.get("Y").cpu().numpy(), Y) < 1e-5
    assert rel(qs.get("W").cpu().numpy(), W) < 1e-5


def test_tc_block_updates_pure_and_eta(pkg):
    m, n, s, l = 320, 256, 9, 19
    A = WL.make_gaussian(m, n, seed=4).astype(np.float32)
    A[0] = 0.0
    qs = pkg.QSketch(m, n, s, l, prec="bf16x3", seed=3, pure=True)
    Ad = torch.as_tensor(A, device="cuda")
    for r0, r1 in ((0, 200), (200, 320)):
        for c0, c1 in ((0, 128), (128, 256)):
            blk = Ad[:, r0:r1, c0:c1]
            qs.update([None, blk[1], blk[2], blk[3]], row0=r0, col0=c0, eta=0.5)
    Om, Psi = _emb(n, s, l, m, 3)
    Y, W = O.sketch(A.astype(np.float64), Om, Psi)
    assert rel(qs.get("Y").cpu().numpy(), 0.5 * Y) < 1e-5
    assert rel(qs.get("W").cpu().numpy(), 0.5 * W) < 1e-5


def test_tc_pipeline_error_within_one_percent(pkg):
    m, n, s, l = 1024, 896, 41, 83
    A = WL.make_decay(m, n, seed=6, rank_cap=600, dtype=np.float32)
    qs = pkg.QSketch(m, n, s, l, prec="bf16x3", seed=8)
    Ad = torch.as_tensor(A, device="cuda")
    qs.update(Ad, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    err = float(qs.error(Ad).item())
    Om, Psi = _emb(n, s, l, m, 8)
    ref = O.onepass(A.astype(np.float64), Om, Psi, "pseudo_qr", 3)
    assert abs(err - ref["err"]) <= 0.01 * ref["err"], (err, ref["err"])


def test_tc_c3_shaped_pipeline(pkg):
    """The c3 shape class (pure quaternion A, Rademacher test matrices, s = 201, l = 403) at
    2048 x 1536: sketch parity, and the final error within 1e-3 of the oracle's (the sketch
    error, <= 1e-5 relative, moves it far less; see test_gpu_pipeline)."""
    m, n, s, l = 2048, 1536, 201, 403
    A = WL.make_decay(m, n, seed=11, rank_cap=800, dtype=np.float32)
    A[0] = 0.0
    Ad = _dev(A)
    planes = [None, Ad[1], Ad[2], Ad[3]]
    qs = pkg.QSketch(m, n, s, l, emb="rademacher", prec="bf16x3", seed=13, pure=True)
    qs.update(planes, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    err = float(qs.error(planes).item())
    assert qs.device_status() == 0
    Om, Psi = _emb(n, s, l, m, 13, O.EMB_RADEMACHER)
    A64 = Ad.double().cpu().numpy()
    ref = O.onepass(A64, Om, Psi, "pseudo_qr", 3)
    assert rel(qs.get("Y").cpu().numpy(), ref["Y"]) < 1e-5
    assert rel(qs.get("W").cpu().numpy(), ref["W"]) < 1e-5
    assert abs(err - ref["err"]) <= 1e-3 * ref["err"], (err, ref["err"])


def test_tc_c5_shaped_tall_pipeline(pkg):
    """The c5 shape class (tall and narrow pure quaternion A, Gaussian test matrices, s = 41,
    l = 83) at 65536 x 256: sketch parity and the final error within 1e-3 of the oracle's."""
    m, n, s, l = 65536, 256, 41, 83
    A = WL.make_decay(m, n, seed=17, rank_cap=256, dtype=np.float32)
    A[0] = 0.0
    Ad = torch.as_tensor(A, device="cuda")
    planes = [None, Ad[1], Ad[2], Ad[3]]
    qs = pkg.QSketch(m, n, s, l, emb="gaussian", prec="bf16x3", seed=19, pure=True)
    qs.update(planes, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    err = float(qs.error(planes).item())
    assert qs.device_status() == 0
    Om, Psi = _emb(n, s, l, m, 19)
    ref = O.onepass(A.astype(np.float64), Om, Psi, "pseudo_qr", 3)
    assert rel(qs.get("Y").cpu().numpy(), ref["Y"]) < 1e-5
    assert rel(qs.get("W").cpu().numpy(), ref["W"]) < 1e-5
    assert abs(err - ref["err"]) <= 1e-3 * ref["err"], (err, ref["err"])
