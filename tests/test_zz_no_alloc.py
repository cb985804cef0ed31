"""The allocation-free error entry point (qs_reconstruct_error_static) against the handle's
error pass (qreconstruct_error), through the C ABI.

In the FP64 and FP32 modes both run the same per-tile arithmetic of the SIMT product's error
epilogue; only the order in which the tile sums are added differs (atomics versus a
fixed-order reduction), so the two agree to FP64 summation rounding: 1e-12 relative.  In the
split-BF16 mode the handle's pass runs on the tensor cores (H X from BF16 hi/lo pairs), which
moves the error by at most 2^-15 ||M||_F / ||A||_F, M = |H| |X| over the Hamilton terms.
The static path is deterministic, so two calls in a row return the same bits; the second
call also shows that no state left in the static scratch by the first one leaks into the
result.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def _pipeline(pkg, m, n, s, l, prec, pure=False, seed=5):
    A = WL.make_decay(m, n, seed=seed, rank_cap=min(m, n), dtype=np.float32)
    if pure:
        A[0] = 0.0
    qs = pkg.QSketch(m, n, s, l, prec=prec, seed=seed, pure=pure)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ad = torch.as_tensor(A, dtype=dt, device="cuda")
    planes = [None, Ad[1], Ad[2], Ad[3]] if pure else Ad
    qs.update(planes, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    ref = float(qs.error(planes).item())
    return qs, planes, ref


_PLANE = [[0, 1, 2, 3], [1, 0, 3, 2], [2, 3, 0, 1], [3, 2, 1, 0]]


def _split_bf16_bound(planes, H, X):
    Hn = H.double().cpu().numpy()
    Xn = X.double().cpu().numpy()
    An = np.stack([np.zeros(Hn.shape[1:2] + Xn.shape[2:]) if p is None else p.double().cpu().numpy()
                   for p in planes])
    M = np.stack([sum(np.abs(Hn[_PLANE[q][b]]) @ np.abs(Xn[b]) for b in range(4)) for q in range(4)])
    return 2.0 ** -15 * np.linalg.norm(M) / np.linalg.norm(An)


def _static_twice(pkg, planes, H, X):
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    r1 = float(pkg.reconstruct_error_static(planes, H, X, out).item())
    r2 = float(pkg.reconstruct_error_static(planes, H, X, out).item())
    return r1, r2


@pytest.mark.parametrize("m,n,s,l,prec", [(600, 500, 21, 43, "fp64"),
                                          (1000, 700, 37, 75, "bf16x3"),
                                          (64, 64, 1, 1, "fp32")])
def test_static_error_matches_handle_error(pkg, m, n, s, l, prec):
    qs, planes, ref = _pipeline(pkg, m, n, s, l, prec)
    r1, r2 = _static_twice(pkg, planes, qs.get("H"), qs.get("X"))
    assert ref > 0
    tol = 1e-12 * ref
    if prec == "bf16x3":
        tol += _split_bf16_bound(planes, qs.get("H"), qs.get("X"))
    assert abs(r1 - ref) <= tol, (r1, ref, tol)
    assert r2 == r1


def test_static_error_pure_quaternion_and_strided_factors(pkg):
    m, n, s, l = 300, 257, 13, 29
    qs, planes, ref = _pipeline(pkg, m, n, s, l, "fp64", pure=True)
    # H with leading dimension s + 7, X with leading dimension n + 3
    Hw = torch.zeros(4, m, s + 7, dtype=torch.float64, device="cuda")
    Xw = torch.zeros(4, s, n + 3, dtype=torch.float64, device="cuda")
    Hw[:, :, :s] = qs.get("H")
    Xw[:, :, :n] = qs.get("X")
    H = [Hw[p, :, :s] for p in range(4)]
    X = [Xw[p, :, :n] for p in range(4)]
    r1, r2 = _static_twice(pkg, planes, H, X)
    assert abs(r1 - ref) <= 1e-12 * ref, (r1, ref)
    assert r2 == r1


def test_static_error_rejects_sizes_beyond_its_scratch(pkg):
    lib = pkg.load_library()
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    planes = (ctypes.c_void_p * 4)(p, p, p, p)
    side = 64 * 257                      # 257^2 tiles > QS_STATIC_ERR_MAX_TILES = 65536
    before = pkg.launch_count()
    st = lib.qs_reconstruct_error_static(side, side, 1, 0, planes, side, planes, 1, planes, side,
                                         ctypes.c_void_p(out.data_ptr()), None)
    assert st == 7                       # QS_ERR_UNSUPPORTED
    assert pkg.launch_count() == before
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
