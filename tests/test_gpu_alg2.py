"""ALG2 of Sec. 5.2 (Table 4, column G): Algorithm 2 with the dual step length tau = 1
instead of 1.9, on both paths, against the oracle run with the same tau.

* FP64: lock-step with the sigma rule (identical penalty schedule, iterates to
  rounding) and a whole solve to eta_dot <= 1e-6 with the oracle's stopping iteration;
* mixed: lock-step within FP32 noise, and a whole solve whose objective is within
  1e-6 relative of the FP64 oracle's continued to eta_dot <= 1e-7.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import ensure_built, oracle_mixture, pair, rel_err

pytestmark = pytest.mark.gpu

TAU = 1.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_alg2_lockstep(prec, bound):
    rng = np.random.default_rng(1300)
    r0 = np.where(rng.random(120) < 0.2, 0.0, rng.random(120))
    r1 = rng.random(120) + 0.01
    g, prob, gpu = pair(2, 8, [12, 10], r0, r1, prec=prec, check_every=10, tau=TAU)
    st = O.State.zeros(g)
    O.solve(prob, st, tol=0.0, maxit=60, check_every=10, tau=TAU)
    gpu.dot_solve(tol=0.0, maxit=60)
    q2, al2, b2, s2, it = gpu.dot_get_state()
    gpu.close()
    assert it == 60 and s2 == st.sigma
    assert rel_err(q2, st.q) < bound and rel_err(al2, st.alpha) < bound and rel_err(b2, st.beta) < bound


def test_alg2_whole_solve():
    """16^2 x 8 Gaussian mixture (seed 4100) with tau = 1.  FP64 to eta_dot <= 1e-6: the
    oracle's stopping iteration and objective.  Mixed to 1e-6: objective within 1e-6
    relative of the oracle's at the same tolerance (same schedule, so the difference is
    precision); continued to 1e-7: within 1e-6 relative of the oracle's at 1e-7 (the
    objective itself still moves by a few 1e-6 between the two tolerances)."""
    r0, r1, mask, g, prob, st, res = oracle_mixture(8, 16, 4100, tol=1e-6, tau=TAU)
    w_o = O.w2_squared(g, res["primal_obj"])
    gpu = pair(2, 8, [16, 16], r0, r1, prec="fp64", tau=TAU)[2]
    assert gpu.dot_solve(1e-6, 60000) == 0
    rho, m, phi, obj, kk = gpu.dot_get()
    gpu.close()
    assert int(kk["iterations"]) == res["iterations"]
    assert abs(obj - w_o) <= 1e-9 * abs(obj)
    rho_o = O.density_slices(g, st)
    assert np.abs(rho - rho_o).max() <= 1e-8 * rho_o.max()
    ref = oracle_mixture(8, 16, 4100, tol=1e-7, tau=TAU)
    w_ref = O.w2_squared(g, ref[6]["primal_obj"])
    gpu = pair(2, 8, [16, 16], r0, r1, prec="mixed", tau=TAU)[2]
    assert gpu.dot_solve(1e-6, 60000) == 0
    obj6, kk6 = gpu.dot_get()[3:]
    assert gpu.dot_solve(1e-7, 200000) == 0
    obj7, kk7 = gpu.dot_get()[3:]
    gpu.close()
    print("ALG2 mixed", kk6["iterations"], kk7["iterations"], "oracle", res["iterations"], ref[6]["iterations"],
          "rel at 1e-6", abs(obj6 - w_o) / w_o, "rel at 1e-7", abs(obj7 - w_ref) / w_ref)
    assert kk6["eta_dot"] <= 1e-6 and kk7["eta_dot"] <= 1e-7
    assert abs(obj6 - w_o) <= 1e-6 * w_o
    assert abs(obj7 - w_ref) <= 1e-6 * w_ref
