"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads,
exports every function include/qsketch.h declares, and validates arguments on the host
before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_14783_gb300 import build as b
    b.build()
    import paper_2404_14783_gb300 as pkg
    return pkg.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "qsketch.h")).read()
    return re.findall(r"QS_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)


def test_header_declares_abi():
    names = _declared()
    import paper_2404_14783_gb300 as pkg
    assert sorted(names) == sorted(pkg.ABI_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_only_abi_symbols_exported(lib):
    import subprocess
    import paper_2404_14783_gb300 as pkg
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True,
                         text=True).stdout
    text_syms = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert text_syms == set(pkg.ABI_SYMBOLS)


def _cfg(**kw):
    from paper_2404_14783_gb300 import QSConfig
    d = dict(m=100, n=80, s=5, l=11, emb=0, prec=0, seed=1, pure=0, flags=0)
    d.update(kw)
    return QSConfig(**d)


def test_workspace_bytes_and_validation(lib):
    good = lib.qsketch_workspace_bytes(ctypes.byref(_cfg()))
    assert good > 0 and good % 256 == 0
    # FP32 storage with native-FP64 stages stores half-size objects; with the default
    # double-float stages the workspace adds the scratch of the sliced tensor-core products
    f32_fp64 = lib.qsketch_workspace_bytes(ctypes.byref(_cfg(prec=1, rf_prec=1)))
    assert f32_fp64 < good
    assert lib.qsketch_workspace_bytes(ctypes.byref(_cfg(prec=1))) > f32_fp64
    for bad in (dict(s=0), dict(l=4), dict(l=81), dict(m=0), dict(emb=2), dict(prec=9),
                dict(flags=1), dict(pure=3), dict(s=2000, l=2000, m=5000, n=5000),
                dict(rf_prec=3), dict(rf_prec=-1), dict(reserved=1)):
        assert lib.qsketch_workspace_bytes(ctypes.byref(_cfg(**bad))) == 0, bad


def test_host_validation_before_launch(lib):
    from paper_2404_14783_gb300.qsketch import QS_ERR_INVALID, QS_ERR_NOMEM
    h = ctypes.c_void_p()
    # invalid config, null workspace, misaligned workspace, too-small workspace
    assert lib.qsketch_create(ctypes.byref(_cfg(s=0)), ctypes.c_void_p(256), 1 << 30, None,
                              ctypes.byref(h)) == QS_ERR_INVALID
    assert lib.qsketch_create(ctypes.byref(_cfg()), None, 1 << 30, None,
                              ctypes.byref(h)) == QS_ERR_INVALID
    assert lib.qsketch_create(ctypes.byref(_cfg()), ctypes.c_void_p(256 + 8), 1 << 30, None,
                              ctypes.byref(h)) == QS_ERR_INVALID
    assert lib.qsketch_create(ctypes.byref(_cfg()), ctypes.c_void_p(256), 16, None,
                              ctypes.byref(h)) == QS_ERR_NOMEM
    assert not h.value
    planes = (ctypes.c_void_p * 4)()
    assert lib.qsketch_update(None, planes, 10, 0, 0, 1, 1, 1.0, 1.0, None) == QS_ERR_INVALID
    assert lib.qrangefinder(None, 0, 3, None) == QS_ERR_INVALID
    assert lib.qonepass_core(None, None) == QS_ERR_INVALID
    assert lib.qreconstruct_error(None, planes, 10, None, None) == QS_ERR_INVALID
    assert lib.qsketch_destroy(None) == QS_ERR_INVALID
    assert lib.qs_status_string(0) == b"ok"
    assert lib.qs_version() >= 100


def test_batched_update_host_validation(lib):
    """qsketch_update_batched validates every item before any CUDA call."""
    from paper_2404_14783_gb300.qsketch import QS_ERR_INVALID, QS_OK
    VP, I64 = ctypes.c_void_p, ctypes.c_int64
    assert lib.qsketch_update_batched(0, None, None, None, None) == QS_OK
    assert lib.qsketch_update_batched(-1, None, None, None, None) == QS_ERR_INVALID
    hs = (VP * 1)(None)
    ptrs = (VP * 4)(None, None, None, None)
    lds = (I64 * 1)(8)
    assert lib.qsketch_update_batched(1, hs, ptrs, lds, None) == QS_ERR_INVALID
    assert lib.qsketch_update_batched(1, None, ptrs, lds, None) == QS_ERR_INVALID


def test_test_flag_only_in_tensor_core_modes(lib):
    # the withhold switch is valid with the tensor-core precisions only
    assert lib.qsketch_workspace_bytes(ctypes.byref(_cfg(flags=1, prec=3))) > 0
    assert lib.qsketch_workspace_bytes(ctypes.byref(_cfg(flags=1, prec=1))) == 0
    assert lib.qsketch_workspace_bytes(ctypes.byref(_cfg(flags=2, prec=3))) == 0


def test_rf_precision_sets_the_storage_of_h_and_x(lib):
    """FP32-storage modes keep H and X in FP64 unless the stages after the sketch run mixed;
    the double-float and mixed stages add the scratch of the sliced tensor-core products."""
    fp32_df = lib.qsketch_workspace_bytes(ctypes.byref(_cfg(prec=1, rf_prec=0)))
    fp32_64 = lib.qsketch_workspace_bytes(ctypes.byref(_cfg(prec=1, rf_prec=1)))
    fp32_mx = lib.qsketch_workspace_bytes(ctypes.byref(_cfg(prec=1, rf_prec=2)))
    m, n, s = 100, 80, 5
    hx_fp32_saving = 4 * (m * s + s * n) * 4      # H and X in FP32 instead of FP64
    assert fp32_df > fp32_64 > 0 and fp32_df > fp32_mx > 0
    assert fp32_df - fp32_mx >= hx_fp32_saving - 2 * 256


def test_static_error_binding_checks_shapes_before_any_launch(lib):
    """reconstruct_error_static refuses operands of the wrong shape, mixed row strides or a
    bad output before it reaches the C ABI (nothing launched)."""
    import torch
    import paper_2404_14783_gb300 as pkg
    m, n, s = 40, 30, 5
    A = torch.zeros(4, m, n, dtype=torch.float64)
    H = torch.zeros(4, m, s, dtype=torch.float64)
    X = torch.zeros(4, s, n, dtype=torch.float64)
    out = torch.zeros(1, dtype=torch.float64)
    before = pkg.launch_count()
    bad_cases = [
        (torch.zeros(4, m, n - 1, dtype=torch.float64), H, X, out),     # A too narrow
        (torch.zeros(4, m - 1, n, dtype=torch.float64), H, X, out),     # A too short
        (A, H, torch.zeros(4, s - 1, n, dtype=torch.float64), out),     # X too short for H
        (A, [H[0], H[1], H[2], None], X, out),                           # H plane missing
        ([A[0], A[1], A[2], torch.zeros(m, n + 3, dtype=torch.float64)[:, :n]], H, X, out),
        (A, H, X, out),                                                  # out on the host
    ]
    for a, h, x, o in bad_cases:
        with pytest.raises(ValueError):
            pkg.reconstruct_error_static(a, h, x, o)
    assert pkg.launch_count() == before
