"""GB300 (sm_103a) one-pass randomized quaternion low-rank approximation.

The compute path is the CUDA library libqsketch.so (C ABI in include/qsketch.h); this
package is its thin Python binding.  See ``QSketch`` for the calls:

    qs = QSketch(m, n, s, l, emb="gaussian", prec="bf16x3", seed=0)
    qs.update(A)                 # Y = A Omega, W = Psi A   (Sec. 4.1)
    qs.rangefinder("pseudo_qr")  # H with R(H) = R(Y)       (Alg. 1 / Alg. 2)
    qs.core()                    # X = (Psi H)^dagger W     (Alg. 3)
    qs.error(A)                  # ||A - HX||_F / ||A||_F   (Sec. 5)
"""
from .qsketch import (QSketch, QSError, QSConfig, load_library, ABI_SYMBOLS, LIB_PATH,
                      PRECISIONS, EMBEDDINGS, RANGEFINDERS, launch_count,
                      reconstruct_error_static, update_batched, tune_batched, RF_PRECISIONS,
                      lorenz4d)

__all__ = ["QSketch", "QSError", "QSConfig", "load_library", "ABI_SYMBOLS", "LIB_PATH",
           "PRECISIONS", "EMBEDDINGS", "RANGEFINDERS", "launch_count", "reconstruct_error_static",
           "update_batched", "tune_batched", "RF_PRECISIONS", "lorenz4d"]
