"""GPU tests of the mixed-precision path (SWM_BF16): E = Z M^-1 rounded to complex bfloat16 feeds
the inner GMRES products, and float64 iterative refinement with complex64-valued residuals brings
the currents to the accuracy of the complex64 system, far below the bfloat16 rounding (2^-9).
Every path is compared with the float64 oracle."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import K, assert_rcs_db, run_gpu
from synth import cloud_uniform_cube, observations_phi_cut

pytestmark = pytest.mark.gpu

C128, C64, BF16 = 0, 1, 2


def _err(out, X):
    return np.linalg.norm(out["currents"] - X) / np.linalg.norm(X)


@pytest.mark.parametrize("path", ["persistent", "per_kernel", "split"])
def test_bf16_refinement_reaches_complex64_accuracy(monkeypatch, path):
    from paper_2410_03060_gb300 import swm

    if path == "per_kernel":
        monkeypatch.setenv("SWM_PERSIST", "0")
    if path == "split":
        monkeypatch.setenv("SWM_SPLIT_ROWS", "0")
    cl = cloud_uniform_cube(150, 6.0, seed=71)
    inc = np.array([[0.0, 0.0, 0.0], [1.1, 0.4, 0.3], [2.0, 3.0, 1.0]])
    obs = observations_phi_cut(90)
    X = O.solve_lu(O.assemble(cl, K, 2.0, sparse=False), O.rhs(cl, K, inc))
    s_ref = O.rcs_bistatic(cl, K, X, obs)
    outs = {}
    for prec in (BF16, C64):
        outs[prec] = run_gpu(cl, K, 2.0, prec, inc, obs=obs, tol=1e-9, restart=30)
    try:
        bf, c64 = outs[BF16], outs[C64]
        assert bf["rc"] == 0 and bf["stats"]["converged"] == 1
        assert bf["stats"]["restarts"] >= 2  # more than one refinement step was needed
        e_bf, e_c64 = _err(bf, X), _err(c64, X)
        # both reach the accuracy of the float32-evaluated blocks, far below bfloat16 rounding
        assert e_bf < 1e-4 and e_c64 < 1e-4
        assert np.linalg.norm(bf["currents"] - c64["currents"]) / np.linalg.norm(X) < 1e-5
        for i in range(inc.shape[0]):
            assert_rcs_db(bf["sigma"][i, :, 0], s_ref[i, :, 0], db=0.1)
    finally:
        for o in outs.values():
            swm.swm_destroy(o["ctx"])


def test_bf16_stops_at_tolerance_and_reports_not_converged():
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(80, 5.0, seed=72)
    inc = np.array([[0.3, 0.2, 0.0]])
    X = O.solve_lu(O.assemble(cl, K, 2.0, sparse=False), O.rhs(cl, K, inc))
    out = run_gpu(cl, K, 2.0, BF16, inc, tol=1e-6, restart=30)
    try:
        assert out["rc"] == 0 and out["stats"]["rel_residual"] <= 1e-6
        assert _err(out, X) < 5e-5
    finally:
        swm.swm_destroy(out["ctx"])
    out = run_gpu(cl, K, 2.0, BF16, inc, tol=1e-12, restart=30, max_iter=3)
    try:
        assert out["rc"] == swm.SWM_ENOTCONV and out["stats"]["converged"] == 0
    finally:
        swm.swm_destroy(out["ctx"])
