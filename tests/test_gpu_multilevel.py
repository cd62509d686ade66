"""The multilevel strategy (Sec. 5) on the GPU: coarse levels solved and
interpolated onto the caller's grid, which then converges to the same solution
as a cold start."""
import numpy as np
import pytest

from gpu_util import ensure_built
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
