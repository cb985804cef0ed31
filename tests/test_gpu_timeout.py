"""Failure path of the bounded device waits, through the C ABI.

QS_FLAG_TEST_WITHHOLD_COPY makes the tensor-core sketch withhold the copy of its first A
tile, so every wait on it expires (2 s of %globaltimer).  The kernel must record
QS_ERR_TIMEOUT in the status word, wait for its own copies and MMAs, free its TMEM and
return -- no hang, no fault -- and the context must stay usable: a normal sketch afterwards
is exact.
"""
import time

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


def test_withheld_copy_times_out_and_context_survives(pkg):
    from paper_2404_14783_gb300.qsketch import QS_ERR_TIMEOUT, QS_FLAG_TEST_WITHHOLD_COPY
    m, n, s, l = 256, 128, 9, 19
    A = WL.make_gaussian(m, n, seed=3).astype(np.float32)
    Ad = torch.as_tensor(A, device="cuda")
    qs = pkg.QSketch(m, n, s, l, prec="bf16x3", seed=4, flags=QS_FLAG_TEST_WITHHOLD_COPY)
    t0 = time.time()
    qs.update(Ad, theta=0.0)
    status = qs.device_status()            # synchronises the stream
    elapsed = time.time() - t0
    assert status == QS_ERR_TIMEOUT
    assert 1.5 < elapsed < 30.0
    # the context is usable and the same kernel is exact without the switch
    ok = pkg.QSketch(m, n, s, l, prec="bf16x3", seed=4)
    ok.update(Ad, theta=0.0)
    assert ok.device_status() == 0
    Om = O.draw_embedding(n, s, O.EMB_GAUSSIAN, O.STREAM_OMEGA, 4)
    Psi = O.draw_embedding(l, m, O.EMB_GAUSSIAN, O.STREAM_PSI, 4)
    Y, W = O.sketch(A.astype(np.float64), Om, Psi)
    assert rel(ok.get("Y").cpu().numpy(), Y) < 1e-5
    assert rel(ok.get("W").cpu().numpy(), W) < 1e-5
