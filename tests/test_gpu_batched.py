"""Batched sketches (qsketch_update_batched) through the C ABI: several independent matrices
of different shapes in one call, as in the batch workload (m, n in [256, 4096], k in [8, 64],
s = 2k + 1, l = 2s + 1, Rademacher test matrices, split-BF16).  Each result matches the
oracle's sketch of its own matrix (1e-5 relative, the split-BF16 tolerance) and the
single-matrix entry point on the same inputs.
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


def test_batched_matches_oracle_and_single_updates(pkg):
    shapes = [(300, 260, 8), (512, 384, 16), (640, 1024, 64)]   # (m, n, k)
    sk, sk1, mats, host = [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        s = 2 * k + 1
        l = 2 * s + 1
        A = WL.make_decay(m, n, seed=20 + i, rank_cap=min(m, n, 320), dtype=np.float32)
        host.append(A)
        mats.append(_dev(A))
        sk.append(pkg.QSketch(m, n, s, l, emb="rademacher", prec="bf16x3", seed=100 + i))
        sk1.append(pkg.QSketch(m, n, s, l, emb="rademacher", prec="bf16x3", seed=100 + i))
    pkg.update_batched(sk, mats)
    for q, A in zip(sk1, mats):
        q.update(A, theta=0.0)
    torch.cuda.synchronize()
    for i, ((m, n, k), A) in enumerate(zip(shapes, host)):
        s = 2 * k + 1
        l = 2 * s + 1
        assert sk[i].device_status() == 0
        Om = O.draw_embedding(n, s, O.EMB_RADEMACHER, O.STREAM_OMEGA, 100 + i)
        Psi = O.draw_embedding(l, m, O.EMB_RADEMACHER, O.STREAM_PSI, 100 + i)
        Y, W = O.sketch(A.astype(np.float64), Om, Psi)
        assert rel(sk[i].get("Y").cpu().numpy(), Y) < 1e-5
        assert rel(sk[i].get("W").cpu().numpy(), W) < 1e-5
        assert rel(sk[i].get("Y").cpu().numpy(), sk1[i].get("Y").cpu().numpy()) < 1e-6
        assert rel(sk[i].get("W").cpu().numpy(), sk1[i].get("W").cpu().numpy()) < 1e-6


def test_batched_rejects_before_enqueueing(pkg):
    """A bad item (row pitch not a multiple of 4 elements) fails the whole batch on the host."""
    good = _dev(WL.make_gaussian(128, 96, seed=1).astype(np.float32))
    bad = torch.zeros((4, 64, 70), dtype=torch.float32, device="cuda")[:, :, :66]
    q1 = pkg.QSketch(128, 96, 9, 19, prec="bf16x3", seed=1)
    q2 = pkg.QSketch(64, 66, 9, 19, prec="bf16x3", seed=2)
    before = pkg.launch_count()
    with pytest.raises(pkg.QSError):
        pkg.update_batched([q1, q2], [good, bad])
    assert pkg.launch_count() == before
