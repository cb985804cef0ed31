"""Edge cases of the tensor-core path against the FP64 oracle.

* s = 256: the largest sketch width the fused kernel takes (NS = 256, one Y plane per TMEM
  half, Omega staged in two row halves); s = 257 is refused with QS_ERR_UNSUPPORTED.
* l = min(m, n) (the method's bound, Sec. 4.1) with a ragged last column tile: the whole path,
  final error within 1% of the oracle's.
Split-BF16 sketches at the 1e-5 relative tolerance.
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


def _dev(A):
    m, n = A.shape[1], A.shape[2]
    buf = torch.zeros((4, m, (n + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    buf[:, :, :n] = torch.as_tensor(A, device="cuda")
    return buf[:, :, :n]


def test_tc_sketch_at_maximum_width(pkg):
    m, n, s, l = 300, 260, 256, 256
    A = WL.make_gaussian(m, n, seed=11).astype(np.float32)
    qs = pkg.QSketch(m, n, s, l, emb="gaussian", prec="bf16x3", seed=12)
    qs.update(_dev(A), theta=0.0)
    torch.cuda.synchronize()
    assert qs.device_status() == 0
    Om = O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, 12)
    Psi = O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, 12)
    Y, W = O.sketch(A.astype(np.float64), Om, Psi)
    assert rel(qs.get("Y").cpu().numpy(), Y) < 1e-5
    assert rel(qs.get("W").cpu().numpy(), W) < 1e-5
    wide = pkg.QSketch(m, n, 257, 257, emb="gaussian", prec="bf16x3", seed=12)
    with pytest.raises(pkg.QSError):
        wide.update(_dev(A), theta=0.0)


def test_tc_path_with_l_at_its_bound(pkg):
    m, n, s, l = 300, 100, 40, 100
    A = WL.make_decay(m, n, seed=13, rank_cap=100, dtype=np.float32)
    Ad = _dev(A)
    qs = pkg.QSketch(m, n, s, l, emb="gaussian", prec="bf16x3", seed=14)
    qs.update(Ad, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    err = float(qs.error(Ad).item())
    assert qs.device_status() == 0
    Om = O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, 14)
    Psi = O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, 14)
    ref = O.onepass(A.astype(np.float64), Om, Psi, "pseudo_qr", 3)
    assert rel(qs.get("Y").cpu().numpy(), ref["Y"]) < 1e-5
    assert rel(qs.get("W").cpu().numpy(), ref["W"]) < 1e-5
    assert abs(err - ref["err"]) <= 0.01 * ref["err"], (err, ref["err"])
