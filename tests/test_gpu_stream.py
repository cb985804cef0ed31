"""Streamed update from host memory (qsketch_update_host) through the C ABI: row blocks of a
pinned host matrix copied on the handle's copy stream while the previous block is sketched.

The result is the sketch of the whole matrix (linear updates, Sec. 4): it matches the oracle
at the tolerance of the arithmetic (1e-12 FP64, 1e-5 split-BF16) and the one-call device
update to summation order (1e-6 relative in the FP32 modes).  In resident mode the staging
buffer ends as a full device copy of A.
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


@pytest.mark.parametrize("prec,mode,tol", [("bf16x3", "ring", 1e-5), ("bf16x3", "resident", 1e-5),
                                           ("fp64", "ring", 1e-12)])
def test_streamed_update_matches_oracle_and_device_update(pkg, prec, mode, tol):
    m, n, s, l = 1000, 700, 21, 43                     # 7 blocks of 150 rows, the last ragged
    A = WL.make_gaussian(m, n, seed=31)
    dt = torch.float64 if prec == "fp64" else torch.float32
    A_host = torch.as_tensor(A, dtype=dt).pin_memory()
    qs = pkg.QSketch(m, n, s, l, prec=prec, seed=33)
    if mode == "resident":
        staging = torch.empty(qs.staging_shape(), dtype=dt, device="cuda")
    else:
        staging = torch.empty((2, 4, 150, qs.staging_shape()[2]), dtype=dt, device="cuda")
    qs.update_host(A_host, staging, block_rows=150, theta=0.0)
    torch.cuda.synchronize()
    assert qs.device_status() == 0
    Om = O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, 33)
    Psi = O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, 33)
    A64 = A_host.double().numpy()
    Y, W = O.sketch(A64, Om, Psi)
    assert rel(qs.get("Y").cpu().numpy(), Y) < tol
    assert rel(qs.get("W").cpu().numpy(), W) < tol
    ref = pkg.QSketch(m, n, s, l, prec=prec, seed=33)
    ref.update(A_host.to("cuda"), theta=0.0)
    assert rel(qs.get("Y").cpu().numpy(), ref.get("Y").cpu().numpy()) < max(tol, 1e-6)
    assert rel(qs.get("W").cpu().numpy(), ref.get("W").cpu().numpy()) < max(tol, 1e-6)
    if mode == "resident":
        np.testing.assert_array_equal(staging[:, :, :n].cpu().numpy(), A_host.numpy())


def test_streamed_update_pure_and_staging_checks(pkg):
    m, n, s, l = 320, 256, 9, 19
    A = WL.make_gaussian(m, n, seed=4).astype(np.float32)
    A[0] = 0.0
    A_host = torch.as_tensor(A).pin_memory()
    qs = pkg.QSketch(m, n, s, l, prec="bf16x3", seed=3, pure=True)
    staging = torch.empty((2, 4, 64, qs.staging_shape()[2]), dtype=torch.float32, device="cuda")
    qs.update_host([None, A_host[1], A_host[2], A_host[3]], staging, block_rows=64, theta=0.0)
    Om = O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, 3)
    Psi = O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, 3)
    Y, W = O.sketch(A.astype(np.float64), Om, Psi)
    assert rel(qs.get("Y").cpu().numpy(), Y) < 1e-5
    assert rel(qs.get("W").cpu().numpy(), W) < 1e-5
    small = torch.empty((4, 64, qs.staging_shape()[2]), dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.QSError):               # one slot only: neither ring nor resident
        qs.update_host(A_host, small, block_rows=64)


def _aligned_block(Ad, r0, r1, c0, c1):
    """Copy of a block in a fresh buffer whose rows are 16-byte aligned (pitch a multiple of 4)."""
    nb = c1 - c0
    buf = torch.zeros(4, r1 - r0, (nb + 3) // 4 * 4, dtype=Ad.dtype, device=Ad.device)
    buf[:, :, :nb] = Ad[:, r0:r1, c0:c1]
    return buf[:, :, :nb]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_tc_block_updates_at_unaligned_offsets(pkg, prec):
    """Row offsets not a multiple of 8 (the tiles start 8-aligned, the A tile loads zero rows
    before the block), a column offset of 4 mod 8 (shifted tile), a column offset of 3 mod 4
    (FP32 kernels) and ragged tails: the sum of the block updates is the full sketch."""
    m, n, s, l = 1000, 700, 21, 43
    A = WL.make_gaussian(m, n, seed=17).astype(np.float32)
    Ad = torch.as_tensor(A, device="cuda")
    qs = pkg.QSketch(m, n, s, l, prec=prec, seed=5)
    full = pkg.QSketch(m, n, s, l, prec=prec, seed=5)
    full.update(Ad, theta=0.0)
    qs.update(Ad[:, :8, :8].contiguous(), theta=0.0, eta=0.0)           # zero Y and W
    for r0, r1 in ((0, 150), (150, 333), (333, 1000)):
        for c0, c1 in ((0, 4), (4, 203), (203, 700)):
            qs.update(_aligned_block(Ad, r0, r1, c0, c1), row0=r0, col0=c0)
    torch.cuda.synchronize()
    assert qs.device_status() == 0
    Om = O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, 5)
    Psi = O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, 5)
    Y, W = O.sketch(A.astype(np.float64), Om, Psi)
    tol = 1e-5 if prec == "bf16x3" else 1e-2          # one BF16 product: 2^-8 per factor
    assert rel(qs.get("Y").cpu().numpy(), Y) < tol
    assert rel(qs.get("W").cpu().numpy(), W) < tol
    assert rel(qs.get("Y").cpu().numpy(), full.get("Y").cpu().numpy()) < tol
    assert rel(qs.get("W").cpu().numpy(), full.get("W").cpu().numpy()) < tol


def test_double_buffered_stream_of_matrices(pkg):
    """Three matrices in turn through two resident staging buffers, each with an event after the
    error pass that read it last: the copies of matrix i+1 may run while matrix i is processed,
    and every sketch and error equals the device-resident computation."""
    m, n, s, l = 640, 512, 17, 35
    mats = [torch.as_tensor(WL.make_decay(m, n, seed=40 + i, rank_cap=64, dtype=np.float32)).pin_memory()
            for i in range(3)]
    qs = pkg.QSketch(m, n, s, l, prec="bf16x3", seed=8)
    staging = [torch.empty(qs.staging_shape(), dtype=torch.float32, device="cuda") for _ in range(2)]
    freed = [torch.cuda.Event(), torch.cuda.Event()]
    got = []
    for i, Ah in enumerate(mats):
        j = i & 1
        qs.update_host(Ah, staging[j], block_rows=128, theta=0.0,
                       staging_free=freed[j] if i >= 2 else None)
        Y, W = qs.get("Y").clone(), qs.get("W").clone()
        qs.rangefinder("pseudo_qr", 3)
        qs.core()
        err = qs.error(staging[j][:, :, :n]).clone()
        freed[j].record()
        got.append((Y, W, err))
    torch.cuda.synchronize()
    assert qs.device_status() == 0
    for Ah, (Y, W, err) in zip(mats, got):
        ref = pkg.QSketch(m, n, s, l, prec="bf16x3", seed=8)
        Ad = Ah.to("cuda")
        ref.update(Ad, theta=0.0)
        assert rel(Y.cpu().numpy(), ref.get("Y").cpu().numpy()) < 1e-6
        assert rel(W.cpu().numpy(), ref.get("W").cpu().numpy()) < 1e-6
        ref.rangefinder("pseudo_qr", 3)
        ref.core()
        e_ref = float(ref.error(Ad).item())
        assert abs(float(err.item()) - e_ref) <= 1e-3 * e_ref
