"""ctypes binding of libqsketch.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module only converts Python
arguments to the C ABI declared in include/qsketch.h.  PyTorch provides device memory and
streams.  If the shared library is missing the binding raises: there is no CPU fallback.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqsketch.so")

QS_OK, QS_ERR_INVALID, QS_ERR_NOMEM, QS_ERR_CUDA, QS_ERR_RANK, QS_ERR_NUMERIC, \
    QS_ERR_TIMEOUT, QS_ERR_UNSUPPORTED = range(8)
QS_EMB_GAUSSIAN, QS_EMB_RADEMACHER = 0, 1
QS_PREC_FP64, QS_PREC_FP32, QS_PREC_BF16, QS_PREC_BF16X3 = 0, 1, 2, 3
QS_RF_PSEUDO_QR, QS_RF_PSEUDO_SVD = 0, 1
QS_RF_PREC_DF64, QS_RF_PREC_FP64, QS_RF_PREC_MIXED = 0, 1, 2
QS_OBJ_Y, QS_OBJ_W, QS_OBJ_OMEGA, QS_OBJ_PSI, QS_OBJ_H, QS_OBJ_X, QS_OBJ_PSIH, \
    QS_OBJ_SCALARS, QS_OBJ_HR, QS_OBJ_XR, QS_OBJ_SIGMA = range(11)
QS_DT_F64, QS_DT_F32 = 0, 1
QS_FLAG_TEST_WITHHOLD_COPY = 1

PRECISIONS = {"fp64": QS_PREC_FP64, "fp32": QS_PREC_FP32, "bf16": QS_PREC_BF16,
              "bf16x3": QS_PREC_BF16X3}
EMBEDDINGS = {"gaussian": QS_EMB_GAUSSIAN, "rademacher": QS_EMB_RADEMACHER}
QS_RF_PSEUDO_QR_HOUSEHOLDER, QS_RF_PSEUDO_SVD_HOUSEHOLDER = 2, 3
RANGEFINDERS = {"pseudo_qr": QS_RF_PSEUDO_QR, "pseudo_svd": QS_RF_PSEUDO_SVD,
                "pseudo_qr_householder": QS_RF_PSEUDO_QR_HOUSEHOLDER,
                "pseudo_svd_householder": QS_RF_PSEUDO_SVD_HOUSEHOLDER}
RF_PRECISIONS = {"df64": QS_RF_PREC_DF64, "fp64": QS_RF_PREC_FP64, "mixed": QS_RF_PREC_MIXED}

ABI_SYMBOLS = ("qsketch_workspace_bytes", "qsketch_create", "qsketch_update", "qrangefinder",
               "qonepass_core", "qreconstruct_error", "qsketch_get", "qs_last_device_error",
               "qsketch_destroy", "qs_status_string", "qs_launch_count", "qs_version",
               "qs_reconstruct_error_static", "qsketch_update_batched", "qtruncate",
               "qsketch_update_host", "qsketch_tune_batched", "qs_lorenz4d")


class QSConfig(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("s", ctypes.c_int64),
                ("l", ctypes.c_int64), ("emb", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("pure", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("rf_prec", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class QSError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: status {code} ({_status_string(code)})")


_lib = None


def load_library(path=LIB_PATH):
    """Load libqsketch.so and declare the ABI.  Raises OSError when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libqsketch.so not built at {path}; run paper_2404_14783_gb300.build")
    lib = ctypes.CDLL(path)
    P, I64, I32, D, VP = ctypes.POINTER, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
    planes = VP * 4
    lib.qsketch_workspace_bytes.argtypes = [P(QSConfig)]
    lib.qsketch_workspace_bytes.restype = ctypes.c_size_t
    lib.qsketch_create.argtypes = [P(QSConfig), VP, ctypes.c_size_t, VP, P(VP)]
    lib.qsketch_update.argtypes = [VP, planes, I64, I64, I64, I64, I64, D, D, VP]
    lib.qrangefinder.argtypes = [VP, I32, I32, VP]
    lib.qonepass_core.argtypes = [VP, VP]
    lib.qreconstruct_error.argtypes = [VP, planes, I64, VP, VP]
    lib.qsketch_get.argtypes = [VP, I32, P(VP), P(I64), P(I64), P(I32)]
    lib.qs_last_device_error.argtypes = [VP, VP]
    lib.qsketch_destroy.argtypes = [VP]
    lib.qs_status_string.argtypes = [I32]
    lib.qs_status_string.restype = ctypes.c_char_p
    lib.qs_version.restype = I32
    lib.qs_launch_count.restype = I64
    lib.qs_reconstruct_error_static.argtypes = [I64, I64, I64, I32, planes, I64, planes, I64,
                                                planes, I64, VP, VP]
    lib.qsketch_update_batched.argtypes = [I32, P(VP), P(VP), P(I64), VP]
    lib.qsketch_tune_batched.argtypes = [I32, P(VP), P(VP), P(I64), I32, VP]
    lib.qs_lorenz4d.argtypes = [VP, I64, I64, D, D, D, D, planes, I32, I64, VP]
    lib.qtruncate.argtypes = [VP, I64, VP]
    lib.qsketch_update_host.argtypes = [VP, planes, I64, I64, VP, ctypes.c_size_t, VP, D, D, VP]
    for name in ("qsketch_create", "qsketch_update", "qrangefinder", "qonepass_core",
                 "qreconstruct_error", "qsketch_get", "qs_last_device_error", "qsketch_destroy",
                 "qs_reconstruct_error_static", "qsketch_update_batched", "qtruncate",
                 "qsketch_update_host", "qsketch_tune_batched", "qs_lorenz4d"):
        getattr(lib, name).restype = I32
    _lib = lib
    return lib


def launch_count():
    """Kernel launches the library has enqueued in this process."""
    return int(load_library().qs_launch_count())


def reconstruct_error_static(A, H, X, out, stream=None):
    """||A - H X||_F / ||A||_F through qs_reconstruct_error_static (no handle, no workspace).

    A (m x n), H (m x s), X (s x n): (4, rows, cols) CUDA tensors or lists of four planes
    (A's first plane may be None), all float64 or all float32, row-major planes, the planes
    of one operand with one row stride.  `out` is a 1-element CUDA float64 tensor the result
    is written to on `stream`; the caller provides it so that the call itself allocates
    nothing.  Shapes, dtypes, devices and strides are checked here, before the C call, so
    that no launch reads past a caller's buffer (ValueError otherwise)."""
    lib = load_library()
    f64 = _dtype_of(H) == torch.float64
    m, s = _shape_of(H)
    s2, n = _shape_of(X)
    if s2 != s:
        raise ValueError(f"X has {s2} rows, H has {s} columns")
    for name, M_, shape, may_skip_w in (("A", A, (m, n), True), ("H", H, (m, s), False),
                                        ("X", X, (s, n), False)):
        mats = [M_[p] for p in range(4)] if isinstance(M_, torch.Tensor) else list(M_)
        if len(mats) != 4:
            raise ValueError(f"{name} must have four planes")
        strides = set()
        for p, t in enumerate(mats):
            if t is None:
                if p == 0 and may_skip_w:
                    continue
                raise ValueError(f"plane {p} of {name} is missing")
            if tuple(t.shape) != shape:
                raise ValueError(f"plane {p} of {name} is {tuple(t.shape)}, expected {shape}")
            strides.add(t.stride(0) if t.shape[0] > 1 else t.shape[1])
        if len(strides) != 1:
            raise ValueError(f"the planes of {name} have different row strides {sorted(strides)}")
    if (not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.float64
            or out.numel() < 1):
        raise ValueError("out must be a CUDA float64 tensor with at least one element")
    for M_ in (A, H, X):
        for t in ([M_[p] for p in range(4)] if isinstance(M_, torch.Tensor) else list(M_)):
            if t is not None and t.device != out.device:
                raise ValueError(f"every plane must be on {out.device}")
    a_ptrs, lda = _planes(A, f64)
    h_ptrs, ldh = _planes(H, f64)
    x_ptrs, ldx = _planes(X, f64)
    _check(lib.qs_reconstruct_error_static(m, n, s, QS_DT_F64 if f64 else QS_DT_F32, a_ptrs, lda,
                                           h_ptrs, ldh, x_ptrs, ldx,
                                           ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
           "qs_reconstruct_error_static")
    return out


def _batch_args(sketches, matrices):
    count = len(sketches)
    hs = (ctypes.c_void_p * max(count, 1))()
    ptrs = (ctypes.c_void_p * max(4 * count, 1))()
    lds = (ctypes.c_int64 * max(count, 1))()
    for i, (qs, A) in enumerate(zip(sketches, matrices)):
        p4, ld = _planes(A, qs.f64)
        hs[i] = qs.handle
        for q in range(4):
            ptrs[4 * i + q] = p4[q]
        lds[i] = ld
    return count, hs, ptrs, lds


def tune_batched(sketches, matrices, reps=3, stream=None):
    """qsketch_tune_batched: time the candidate plans of the batched sketch on this batch and
    keep the fastest for batches of the same signature (synchronises the stream)."""
    lib = load_library()
    count, hs, ptrs, lds = _batch_args(sketches, matrices)
    return _check(lib.qsketch_tune_batched(count, hs, ptrs, lds, int(reps), _stream_ptr(stream)),
                  "qsketch_tune_batched")


def lorenz4d(u0, steps, dt, a=15.0, b=2.0, c=28.0, dtype=torch.float32, stream=None):
    """qs_lorenz4d: RK4 trajectories of the 4D Lorenz-type system from the initial states u0
    (a (4, cols) CUDA float64 tensor); returns the (4, steps, cols) quaternion matrix of the
    states after each step (leading dimension padded to a multiple of 4), viewed as
    (4, steps, cols)."""
    lib = load_library()
    if not (u0.is_cuda and u0.dtype == torch.float64 and u0.dim() == 2 and u0.shape[0] == 4):
        raise ValueError("u0 must be a (4, cols) CUDA float64 tensor")
    u0 = u0.contiguous()
    cols = int(u0.shape[1])
    ldo = (cols + 3) // 4 * 4
    out = torch.empty((4, steps, ldo), dtype=dtype, device=u0.device)
    ptrs = (ctypes.c_void_p * 4)(*[out[p].data_ptr() for p in range(4)])
    _check(lib.qs_lorenz4d(ctypes.c_void_p(u0.data_ptr()), cols, int(steps), float(dt), float(a),
                           float(b), float(c), ptrs, QS_DT_F64 if dtype == torch.float64 else QS_DT_F32,
                           ldo, _stream_ptr(stream)), "qs_lorenz4d")
    return out[:, :, :cols]


def update_batched(sketches, matrices, stream=None):
    """Y_i = A_i Omega_i and W_i = Psi_i A_i for each (QSketch, A_i) pair in one call
    (qsketch_update_batched); A_i as for QSketch.update, the whole matrix."""
    lib = load_library()
    count = len(sketches)
    hs = (ctypes.c_void_p * max(count, 1))()
    ptrs = (ctypes.c_void_p * max(4 * count, 1))()
    lds = (ctypes.c_int64 * max(count, 1))()
    for i, (qs, A) in enumerate(zip(sketches, matrices)):
        p4, ld = _planes(A, qs.f64)
        hs[i] = qs.handle
        for q in range(4):
            ptrs[4 * i + q] = p4[q]
        lds[i] = ld
    return _check(lib.qsketch_update_batched(count, hs, ptrs, lds, _stream_ptr(stream)),
                  "qsketch_update_batched")


def _dtype_of(M):
    return M.dtype if isinstance(M, torch.Tensor) else next(t for t in M if t is not None).dtype


def _shape_of(M):
    if isinstance(M, torch.Tensor):
        return int(M.shape[1]), int(M.shape[2])
    ref = next(t for t in M if t is not None)
    return int(ref.shape[0]), int(ref.shape[1])


def _status_string(code):
    try:
        return load_library().qs_status_string(int(code)).decode()
    except OSError:
        return "?"


def _check(code, what, allow=(QS_OK,)):
    if code not in allow:
        raise QSError(code, what)
    return code


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _planes(A, f64):
    """Four plane pointers from a (4, rows, cols) tensor or a list of 4 tensors/None."""
    want = torch.float64 if f64 else torch.float32
    if isinstance(A, torch.Tensor):
        assert A.dim() == 3 and A.shape[0] == 4, "A must be (4, rows, cols)"
        mats = [A[p] for p in range(4)]
    else:
        mats = list(A)
    ptrs = (ctypes.c_void_p * 4)()
    ld = None
    for p, t in enumerate(mats):
        if t is None:
            ptrs[p] = None
            continue
        if not t.is_cuda or t.dtype != want or t.stride(1) != 1:
            raise ValueError(f"plane {p} must be a CUDA {want} row-major matrix")
        ld = t.stride(0) if t.shape[0] > 1 else t.shape[1]
        ptrs[p] = t.data_ptr()
    return ptrs, ld


class QSketch:
    """One sketch state (Omega, Psi, Y, W and the results) in a caller-owned workspace."""

    def __init__(self, m, n, s, l, emb="gaussian", prec="fp64", seed=0, pure=False,
                 device="cuda", stream=None, flags=0, rf_prec="df64"):
        self.lib = load_library()
        self.cfg = QSConfig(m, n, s, l, EMBEDDINGS.get(emb, emb), PRECISIONS.get(prec, prec),
                            seed, int(bool(pure)), int(flags), RF_PRECISIONS.get(rf_prec, rf_prec), 0)
        self.f64 = self.cfg.prec == QS_PREC_FP64
        nbytes = self.lib.qsketch_workspace_bytes(ctypes.byref(self.cfg))
        if nbytes == 0:
            raise QSError(QS_ERR_INVALID, "qsketch_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.handle = ctypes.c_void_p()
        _check(self.lib.qsketch_create(ctypes.byref(self.cfg), ctypes.c_void_p(self.workspace.data_ptr()),
                                       nbytes, _stream_ptr(stream), ctypes.byref(self.handle)),
               "qsketch_create")

    def reset(self, seed=None, stream=None):
        """Re-run qsketch_create on the same workspace: redraw Omega and Psi (same seed unless
        given) and zero Y and W."""
        if seed is not None:
            self.cfg.seed = seed
        if self.handle:
            self.lib.qsketch_destroy(self.handle)
        self.handle = ctypes.c_void_p()
        _check(self.lib.qsketch_create(ctypes.byref(self.cfg), ctypes.c_void_p(self.workspace.data_ptr()),
                                       self.workspace.numel(), _stream_ptr(stream),
                                       ctypes.byref(self.handle)), "qsketch_create")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.qsketch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- calls
    def update(self, A, row0=0, col0=0, theta=1.0, eta=1.0, stream=None):
        """Linear update with the block A (tensor (4, mb, nb) or 4 planes, plane 0 may be None)."""
        ptrs, ld = _planes(A, self.f64)
        if isinstance(A, torch.Tensor):
            mb, nb = A.shape[1], A.shape[2]
        else:
            ref = next(t for t in A if t is not None)
            mb, nb = ref.shape
        return _check(self.lib.qsketch_update(self.handle, ptrs, ld, row0, col0, mb, nb, theta, eta,
                                              _stream_ptr(stream)), "qsketch_update")

    def rangefinder(self, kind="pseudo_qr", n_correction=3, stream=None):
        return _check(self.lib.qrangefinder(self.handle, RANGEFINDERS.get(kind, kind), n_correction,
                                            _stream_ptr(stream)), "qrangefinder")

    def core(self, stream=None):
        return _check(self.lib.qonepass_core(self.handle, _stream_ptr(stream)), "qonepass_core")

    def error(self, A, out=None, stream=None):
        """Relative error ||A - HX||_F/||A||_F; returns a 1-element CUDA float64 tensor."""
        ptrs, ld = _planes(A, self.f64)
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=self.workspace.device)
        _check(self.lib.qreconstruct_error(self.handle, ptrs, ld, ctypes.c_void_p(out.data_ptr()),
                                           _stream_ptr(stream)), "qreconstruct_error")
        return out

    def staging_shape(self):
        """(4, m, ldd) of a resident staging copy for update_host (ldd = ceil(n / 4) * 4)."""
        c = self.cfg
        return (4, c.m, (c.n + 3) // 4 * 4)

    def update_host(self, A_host, staging, block_rows=1024, theta=0.0, eta=1.0, staging_free=None,
                    stream=None):
        """Full-matrix update from host memory (qsketch_update_host).  A_host: (4, m, n) CPU
        tensor (pinned for overlap) or a list of four planes (the first may be None when
        pure); staging: CUDA tensor -- a resident copy of shape staging_shape() (A stays on
        the device afterwards) or at least two blocks of block_rows rows; staging_free: a
        recorded torch.cuda.Event after which staging may be overwritten (default: all work
        enqueued on the stream so far)."""
        want = torch.float64 if self.f64 else torch.float32
        mats = [A_host[p] for p in range(4)] if isinstance(A_host, torch.Tensor) else list(A_host)
        ptrs = (ctypes.c_void_p * 4)()
        ld = None
        for p, t in enumerate(mats):
            if t is None:
                ptrs[p] = None
                continue
            if t.is_cuda or t.dtype != want or t.stride(1) != 1:
                raise ValueError(f"host plane {p} must be a CPU {want} row-major matrix")
            ld = t.stride(0)
            ptrs[p] = t.data_ptr()
        nbytes = staging.numel() * staging.element_size()
        ev = ctypes.c_void_p(staging_free.cuda_event) if staging_free is not None else None
        return _check(self.lib.qsketch_update_host(self.handle, ptrs, ld, int(block_rows),
                                                   ctypes.c_void_p(staging.data_ptr()), nbytes, ev,
                                                   theta, eta, _stream_ptr(stream)),
                      "qsketch_update_host")

    def truncate(self, r, stream=None):
        """Truncation stage (Alg. 4): rank-r H_r, X_r = Sigma_r V_r* and Sigma_r, read with
        get("Hr"), get("Xr"), get("sigma")."""
        _check(self.lib.qtruncate(self.handle, int(r), _stream_ptr(stream)), "qtruncate")
        self.trunc_r = int(r)

    def device_status(self, stream=None):
        return self.lib.qs_last_device_error(self.handle, _stream_ptr(stream))

    def get(self, which):
        """Tensor view (4, rows, cols) of a workspace object (no copy)."""
        names = {"Y": QS_OBJ_Y, "W": QS_OBJ_W, "Omega": QS_OBJ_OMEGA, "Psi": QS_OBJ_PSI,
                 "H": QS_OBJ_H, "X": QS_OBJ_X, "PsiH": QS_OBJ_PSIH, "scalars": QS_OBJ_SCALARS,
                 "Hr": QS_OBJ_HR, "Xr": QS_OBJ_XR, "sigma": QS_OBJ_SIGMA}
        code = names.get(which, which)
        ptr, ld, ps, dt = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(self.lib.qsketch_get(self.handle, code, ctypes.byref(ptr), ctypes.byref(ld),
                                    ctypes.byref(ps), ctypes.byref(dt)), "qsketch_get")
        c = self.cfg
        r = getattr(self, "trunc_r", 0)
        shapes = {QS_OBJ_Y: (c.m, c.s), QS_OBJ_W: (c.l, c.n), QS_OBJ_OMEGA: (c.n, c.s),
                  QS_OBJ_PSI: (c.l, c.m), QS_OBJ_H: (c.m, c.s), QS_OBJ_X: (c.s, c.n),
                  QS_OBJ_PSIH: (c.l, c.s), QS_OBJ_HR: (c.m, r), QS_OBJ_XR: (r, c.n)}
        dtype = torch.float64 if dt.value == QS_DT_F64 else torch.float32
        esize = 8 if dtype == torch.float64 else 4
        off = ptr.value - self.workspace.data_ptr()
        if code == QS_OBJ_SCALARS:
            return self.workspace[off:off + 16 * 8].view(torch.float64)
        if code == QS_OBJ_SIGMA:
            return self.workspace[off:off + ld.value * 8].view(torch.float64)
        rows, cols = shapes[code]
        nel = 3 * ps.value + (rows - 1) * ld.value + cols
        flat = self.workspace[off:off + nel * esize].view(dtype)
        return flat.as_strided((4, rows, cols), (ps.value, ld.value, 1))
