"""The allocation-free error entry point (qs_reconstruct_error_static) against the handle's
error pass (qreconstruct_error), through the C ABI.

In the FP64 and FP32 modes both run the same per-tile arithmetic of the SIMT product's error
epilogue; only the order in which the tile sums are added differs (atomics versus a
fixed-order reduction), so the two agree to FP64 summation rounding: 1e-12 relative.  In the
split-BF16 mode the handle's pass runs on the tensor cores (H X from BF16 hi/lo pairs), which
moves the error by at most 2^-15 ||M||_F / ||A||_F, M = |H| |X| over the Hamilton terms.
The handles run with rf_prec = mixed in the FP32-storage modes, which keeps H and X in FP32,
so that both entry points see the same factor values.  Both are also compared with the
oracle's error of those factors (FP64): 1e-12 relative in FP64; in FP32 the product H X is
accumulated in FP32, which moves the error by at most 2 s 2^-24 ||M||_F / ||A||_F.

The static path is deterministic, so two calls in a row return the same bits.  A large call
followed by a smaller one shows that what the first leaves in the static scratch does not
leak into the second, and the device's free memory is the same before and after a call.
"""
import ctypes

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


def _pipeline(pkg, m, n, s, l, prec, pure=False, seed=5):
    A = WL.make_decay(m, n, seed=seed, rank_cap=min(m, n), dtype=np.float32)
    if pure:
        A[0] = 0.0
    qs = pkg.QSketch(m, n, s, l, prec=prec, seed=seed, pure=pure,
                     rf_prec="df64" if prec == "fp64" else "mixed")
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ad = torch.as_tensor(A, dtype=dt, device="cuda")
    planes = [None, Ad[1], Ad[2], Ad[3]] if pure else Ad
    qs.update(planes, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    ref = float(qs.error(planes).item())
    return qs, planes, ref


_PLANE = [[0, 1, 2, 3], [1, 0, 3, 2], [2, 3, 0, 1], [3, 2, 1, 0]]


def _np_planes(planes, H, X):
    Hn = H.double().cpu().numpy()
    Xn = X.double().cpu().numpy()
    An = np.stack([np.zeros(Hn.shape[1:2] + Xn.shape[2:]) if p is None else p.double().cpu().numpy()
                   for p in planes])
    return An, Hn, Xn


def _abs_product_bound(planes, H, X, unit):
    """unit * ||M||_F / ||A||_F, M = |H| |X| summed over the Hamilton terms."""
    An, Hn, Xn = _np_planes(planes, H, X)
    M = np.stack([sum(np.abs(Hn[_PLANE[q][b]]) @ np.abs(Xn[b]) for b in range(4)) for q in range(4)])
    return unit * np.linalg.norm(M) / np.linalg.norm(An)


def _split_bf16_bound(planes, H, X):
    return _abs_product_bound(planes, H, X, 2.0 ** -15)


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
    # against the oracle's error of the same factors
    An, Hn, Xn = _np_planes(planes, qs.get("H"), qs.get("X"))
    exact = O.rel_error(An, Hn, Xn)
    tol_o = 1e-12 * exact if prec == "fp64" else _abs_product_bound(planes, qs.get("H"), qs.get("X"),
                                                                    2 * s * 2.0 ** -24)
    assert abs(r1 - exact) <= tol_o, (r1, exact, tol_o)


def test_static_error_large_then_small_call_and_no_allocation(pkg):
    """A 1000 x 700 call, then a 64 x 64 one: the second equals its own handle's error (the
    first call's scratch contents do not leak); the device's free memory does not move."""
    big, bplanes, _ = _pipeline(pkg, 1000, 700, 37, 75, "fp64", seed=8)
    small, splanes, sref = _pipeline(pkg, 64, 64, 5, 11, "fp64", seed=9)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    pkg.reconstruct_error_static(bplanes, big.get("H"), big.get("X"), out)   # warm-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    reserved0 = torch.cuda.memory_reserved()
    pkg.reconstruct_error_static(bplanes, big.get("H"), big.get("X"), out)
    r = float(pkg.reconstruct_error_static(splanes, small.get("H"), small.get("X"), out).item())
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    assert abs(r - sref) <= 1e-12 * sref, (r, sref)


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
