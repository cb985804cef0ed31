"""Plain FP64 CPU oracle for the one-pass randomized quaternion low-rank approximation.

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg and the reference arm (``--impl reference``) of ``bench.py`` may import it.  The CUDA product path never imports,
links or executes anything here, and nothing here imports the CUDA path: the two share
no code.  The only common dependency is ``workloads`` (seeded synthetic inputs, which
holds none of the method's arithmetic).

Every function follows the paper (Chang & Yang, "Randomized large-scale quaternion
matrix approximation: practical rangefinders and one-pass algorithm", arXiv 2404.14783)
step by step, in double precision, with numpy primitives (matmul, complex QR, SVD,
linear solves) as the only library calls.  Citations name the paper's section, equation
or algorithm.

Quaternion matrices are numpy arrays of shape ``(4, rows, cols)``: the four real
component planes ``Q_w, Q_x, Q_y, Q_z`` of ``Q = Q_w + Q_x i + Q_y j + Q_z k``.

What pins each function to the paper (not to itself) is in ``tests/test_oracle_pins.py``.
No function here is "parity unpinned".
"""
from .quaternion import (qmatmul, qconjT, chi, comp, from_comp, upsilon, qnorm, qeye,
                         qzeros, qpinv, qscalar_mul_chi)
from .philox import (philox4x32_10, draw_embedding, draw_uniform_f, EMB_GAUSSIAN,
                     EMB_RADEMACHER, STREAM_OMEGA, STREAM_PSI, STREAM_PSVD_F)
from .method import (sketch, thin_qr_complex, pseudo_qr, correction_step, epsilon_rule,
                     pseudo_svd, classify_pairs, qls_solve, qb_core, rel_error,
                     qmgs2, qsvd_dense, onepass, truncate, truncated_core)
from .lorenz import lorenz4d_rhs, rk4_step, lorenz4d_snapshots

__all__ = [n for n in dir() if not n.startswith("_")]
