"""The paper's hyperchaotic-system example (Sec. 5, 4D Lorenz-type system) through the C ABI.

  * The GPU generator (qs_lorenz4d: RK4 in FP64, one trajectory per thread) against the
    oracle's RK4 of the same system on 64 trajectories x 300 steps of 1e-3: the two differ
    only by rounding (FMA contraction), which the chaotic flow amplifies little over t = 0.3:
    1e-10 relative.
  * The one-pass method on snapshots of the system (2000 time instances x 1000 initial states,
    built by the oracle's integrator, so no oracle input comes from the GPU): final relative
    error against the oracle's with the same test matrices: 1e-6 relative (FP64 path),
    1% (split-BF16 sketch, double-float stages).
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


def test_generator_matches_oracle_rk4(pkg):
    u0 = WL.lorenz_initial_states(64, seed=3)
    A = pkg.lorenz4d(torch.as_tensor(u0, device="cuda"), 300, 1e-3, dtype=torch.float64)
    ref = O.lorenz4d_snapshots(u0, 300, 1e-3)
    got = A.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("bf16x3", 1e-2)])
def test_onepass_on_lorenz_snapshots(pkg, prec, tol):
    m, n, s, l = 2000, 1000, 41, 83
    A = O.lorenz4d_snapshots(WL.lorenz_initial_states(n, seed=4), m, 1e-3)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ad = torch.as_tensor(A, dtype=dt, device="cuda").contiguous()
    qs = pkg.QSketch(m, n, s, l, emb="gaussian", prec=prec, seed=5)
    qs.update(Ad, theta=0.0)
    qs.rangefinder("pseudo_qr", 3)
    qs.core()
    err = float(qs.error(Ad).item())
    assert qs.device_status() == 0
    Om = qs.get("Omega").cpu().double().numpy()
    Psi = qs.get("Psi").cpu().double().numpy()
    ref = O.onepass(Ad.double().cpu().numpy(), Om, Psi, "pseudo_qr", 3)
    assert abs(err - ref["err"]) <= tol * ref["err"], (err, ref["err"])
