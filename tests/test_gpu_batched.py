"""Batched sketches (qsketch_update_batched) through the C ABI: several independent matrices
of different shapes in one call, as in the batch workload (m, n in [256, 4096], k in [8, 64],
s = 2k + 1, l = 2s + 1, Rademacher test matrices, split-BF16).  Each result matches the
oracle's sketch of its own matrix (1e-5 relative, the split-BF16 tolerance) and the
single-matrix entry point on the same inputs.  The tensor-core items of a call share
persistent launches of up to 32 matrices; the call replays from a captured CUDA graph.
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


def _batch(pkg, count, seed):
    """count small matrices of mixed shapes, embeddings, precisions and purity."""
    rng = np.random.default_rng(seed)
    sk, sk1, mats, host, meta = [], [], [], [], []
    for i in range(count):
        m, n = (int(v) for v in rng.integers(64, 400, size=2))
        k = int(rng.integers(2, 9))
        s = 2 * k + 1
        l = min(2 * s + 1, m, n)
        emb = "rademacher" if i % 3 else "gaussian"
        prec = ("bf16x3", "bf16x3", "bf16", "fp32")[i % 4]
        pure = i % 5 == 4
        A = WL.make_decay(m, n, seed=seed + i, rank_cap=min(m, n, 64), dtype=np.float32)
        if pure:
            A[0] = 0.0
        host.append(A)
        d = _dev(A)
        mats.append([None, d[1], d[2], d[3]] if pure else d)
        kw = dict(emb=emb, prec=prec, seed=1000 + i, pure=pure)
        sk.append(pkg.QSketch(m, n, s, l, **kw))
        sk1.append(pkg.QSketch(m, n, s, l, **kw))
        meta.append((m, n, s, l, emb, prec))
    return sk, sk1, mats, host, meta


def _check_batch(sk, sk1, host, meta, tol_single, seeds=None):
    for i, (A, (m, n, s, l, emb, prec)) in enumerate(zip(host, meta)):
        seed = 1000 + (i if seeds is None else seeds[i])
        assert sk[i].device_status() == 0
        Y, W = sk[i].get("Y").cpu().numpy(), sk[i].get("W").cpu().numpy()
        assert rel(Y, sk1[i].get("Y").cpu().numpy()) < tol_single, i
        assert rel(W, sk1[i].get("W").cpu().numpy()) < tol_single, i
        if i % 7 == 0:       # a sample against the oracle
            kind = O.EMB_RADEMACHER if emb == "rademacher" else O.EMB_GAUSSIAN
            Om = O.draw_embedding(n, s, kind, O.STREAM_OMEGA, seed)
            Psi = O.draw_embedding(l, m, kind, O.STREAM_PSI, seed)
            Yr, Wr = O.sketch(A.astype(np.float64), Om, Psi)
            tol = 8e-3 if prec == "bf16" else 1e-5
            assert rel(Y, Yr) < tol and rel(W, Wr) < tol, i


def test_batched_persistent_launches(pkg):
    """48 items: the 36 in the tensor-core modes run as two persistent launches (32 + 4 items,
    each after a launch that zeroes their sketches); the FP32 ones one update each.  Each item
    equals its single update (1e-6: only the order of the L2 reductions differs) and, on a
    sample, the oracle (1e-5 split-BF16, 8e-3 BF16)."""
    sk, sk1, mats, host, meta = _batch(pkg, 48, seed=50)
    n_tc = sum(1 for mt in meta if mt[5] != "fp32")
    before = pkg.launch_count()
    pkg.update_batched(sk, mats)
    launched = pkg.launch_count() - before
    n_fp32 = len(meta) - n_tc
    prepare = (n_tc + 31) // 32
    assert prepare == 2
    assert launched <= 2 * prepare + n_fp32 * 8, launched
    for q, A in zip(sk1, mats):
        q.update(A, theta=0.0)
    torch.cuda.synchronize()
    _check_batch(sk, sk1, host, meta, 1e-6)


def test_batched_update_replays_from_a_cuda_graph(pkg):
    """The batched call captured once in a CUDA graph and replayed (the sketches cleared in
    between) gives the eager results."""
    sk, sk1, mats, host, meta = _batch(pkg, 12, seed=90)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        pkg.update_batched(sk, mats)          # eager run on a side stream (first-call set-up)
    torch.cuda.current_stream().wait_stream(side)
    for q, A in zip(sk1, mats):
        q.update(A, theta=0.0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pkg.update_batched(sk, mats)
    for rep in range(2):
        for q in sk:
            q.get("Y").fill_(float("nan"))
            q.get("W").fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        _check_batch(sk, sk1, host, meta, 1e-6)


def test_tuned_batched_plan(pkg):
    """qsketch_tune_batched times the candidate plans (32 items per launch or one launch with
    the descriptors in the workspaces, item order, persistent grid) on the batch -- every plan
    form runs -- and the batched call then runs the kept plan: same sketches as single
    updates."""
    sk, sk1, mats, host, meta = _batch(pkg, 20, seed=130)
    tc = [i for i, mt in enumerate(meta) if mt[5] != "fp32"]
    pkg.tune_batched([sk[i] for i in tc], [mats[i] for i in tc], reps=2)
    for q in sk:
        q.get("Y").fill_(float("nan"))
        q.get("W").fill_(float("nan"))
    pkg.update_batched([sk[i] for i in tc], [mats[i] for i in tc])
    for i in tc:
        sk1[i].update(mats[i], theta=0.0)
    torch.cuda.synchronize()
    _check_batch([sk[i] for i in tc], [sk1[i] for i in tc], [host[i] for i in tc],
                 [meta[i] for i in tc], 1e-6, seeds=tc)
