"""The multilevel strategy (Sec. 5) on the GPU: coarse levels solved and
interpolated onto the caller's grid, which then converges to the same solution
as a cold start and as the FP64 oracle solved from zero to eta_dot <= 1e-7."""
import numpy as np
import pytest

import oracle as O
from gpu_util import ensure_built, oracle_mixture
from paper_2505_05424_gb300 import workloads as W
from paper_2505_05424_gb300.solver import DotError, DotSolver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.mark.parametrize("prec,masked", [("mixed", False), ("mixed", True), ("fp64", False)])
def test_multilevel_reaches_the_cold_start_solution(prec, masked):
    spec = W.GridSpec(2, 16, 32)
    r0, r1, mask = W.mixture_pair(spec, 4100 + masked, obstacles=masked)
    cold = DotSolver(2, 16, 32, r0, r1, mask=mask, prec=prec)
    assert cold.dot_solve(1e-6, 40000) == 0
    _, _, phi_c, obj_c, kk_c = cold.dot_get()
    cold.close()
    warm = DotSolver(2, 16, 32, r0, r1, mask=mask, prec=prec)
    rc, iters = warm.dot_solve_multilevel(2, 1e-6, 40000)
    assert rc == 0 and len(iters) == 3 and min(iters) > 0
    rho, m, phi_w, obj_w, kk_w = warm.dot_get()
    warm.close()
    print(prec, masked, "cold", kk_c["iterations"], "multilevel (fine, 1/2, 1/4)", iters, obj_c, obj_w)
    assert kk_w["eta_dot"] <= 1e-6
    assert kk_w["iterations"] == iters[0]
    # two solves that each stop at eta <= 1e-6 agree on the objective to ~1e-5
    assert abs(obj_w - obj_c) <= 2e-5 * abs(obj_c)


def test_multilevel_rejects_indivisible_grids():
    r = np.ones(30 * 30)
    s = DotSolver(2, 16, 30, r, r, prec="mixed")
    with pytest.raises(DotError):
        s.dot_solve_multilevel(2)       # 30 is not divisible by 4
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("masked", [False, True])
def test_multilevel_matches_oracle(prec, masked):
    """16^2 x 8 mixtures (seed 4100, with and without obstacles), two coarse levels
    (8^2 x 4, 4^2 x 2), solved to eta_dot <= 1e-7 and compared with the oracle's cold
    solve to the same tolerance: the objective within 1e-6 relative, the densities
    within 1% of their maximum (measured differences are printed).  At 1e-6 the
    objective itself still differs from its 1e-7 value by a few 1e-6 on this grid."""
    tol = 1e-7
    r0, r1, mask, g, prob, st, res = oracle_mixture(8, 16, 4100 + masked, masked=masked, tol=1e-7)
    w_ref = O.w2_squared(g, res["primal_obj"])
    rho_o = O.density_slices(g, st)
    s = DotSolver(2, 8, 16, r0, r1, mask=mask, prec=prec)
    rc, iters = s.dot_solve_multilevel(2, tol, 200000)
    rho, m, phi, obj, kk = s.dot_get()
    s.close()
    d_rho = np.abs(rho - rho_o).max() / rho_o.max()
    print(prec, masked, "levels (fine, 1/2, 1/4)", iters, "oracle", res["iterations"], "obj", obj, "ref", w_ref,
          "rel", abs(obj - w_ref) / w_ref, "max|rho - rho_o| / max", d_rho)
    assert rc == 0 and kk["eta_dot"] <= tol
    assert abs(obj - w_ref) <= 1e-6 * w_ref
    assert d_rho <= 1e-2
