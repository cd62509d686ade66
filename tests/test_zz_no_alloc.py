"""The allocation-free Poisson entry point against the existing one.

dot_poisson_f32_noalloc serves callers that cannot allocate device memory (plugins
of hosts that forbid allocation on their worker threads, processes whose device
memory another allocator has reserved); its scratch lives in a fixed device array
of the library.  It must return what dot_poisson returns for a DOT_MIXED context on
the same right-hand side, call after call, although the array keeps the previous
call's contents, and agree with the oracle's Poisson solve (Sec. 4, DCT
diagonalisation of A^*A).  This file is collected last so that a failure here
leaves every other test already run.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import ensure_built, rel_err
from test_gpu_parity_mixed import refined_tol
from paper_2505_05424_gb300.solver import DotError, DotSolver, dot_poisson_f32_noalloc

pytestmark = pytest.mark.gpu

# one grid whose spatial axes run on the tensor cores, one on the SIMT passes, a 3D
# grid, and a time axis near the largest the entry point accepts (151 of 160 nodes)
GRIDS = [(2, 16, [64, 48]), (2, 9, [30, 22]), (3, 7, [16, 12, 20]), (2, 150, [64, 64])]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def centred(v):
    v = np.asarray(v, dtype=np.float64).ravel()
    return v - v.mean()


@pytest.mark.parametrize("D,T,N", GRIDS)
def test_noalloc_matches_dot_poisson_twice(D, T, N):
    import torch
    n = (T + 1) * int(np.prod(N))
    rng = np.random.default_rng(900 + T)
    r0 = rng.random(int(np.prod(N))) + 0.1
    ctx = DotSolver(D, T, N, r0, r0, prec="mixed")
    for call in range(2):
        b = (rng.standard_normal(n) + 0.3 * call).astype(np.float32)
        ref = ctx.dot_poisson(b.astype(np.float64))
        bd = torch.from_numpy(b).cuda()
        out = torch.full((2 * n,), float("nan"), dtype=torch.float32, device="cuda")
        dot_poisson_f32_noalloc(D, T, N, bd, out)
        pair = out.cpu().numpy().astype(np.float64).reshape(n, 2)
        phi = pair[:, 0] + pair[:, 1]
        # same refined solve on the same input (the time axis may run the other
        # time pass): agreement within the bar the refined solve is held to
        tol = refined_tol(T, N)
        assert rel_err(centred(phi), centred(ref)) < tol, call
        # and the oracle's solve of the same FP32 right-hand side, at the bar the
        # refined mixed solve is held to
        g = O.Grid(D, T, N)
        want = O.poisson(g, b.astype(np.float64))
        assert rel_err(centred(phi), centred(want)) < tol, call
    ctx.close()


def test_noalloc_rejects_grids_beyond_its_limit():
    import torch
    b = torch.zeros(4, dtype=torch.float32, device="cuda")
    phi = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(DotError) as e:
        dot_poisson_f32_noalloc(2, 64, [256, 256], b, phi)     # 4.26M nodes > 2^20
    assert "at most" in str(e.value)
    with pytest.raises(DotError):
        dot_poisson_f32_noalloc(2, 8, [300, 8], b, phi)        # axis longer than 256
    with pytest.raises(DotError) as e:
        dot_poisson_f32_noalloc(2, 160, [8, 8], b, phi)        # 161 time nodes > 160
    assert "160" in str(e.value)


def test_noalloc_accepts_largest_time_axis():
    """T + 1 = 160, the largest accepted, against the oracle."""
    import torch
    D, T, N = 2, 159, [16, 20]
    n = (T + 1) * int(np.prod(N))
    b = np.random.default_rng(77).standard_normal(n).astype(np.float32)
    out = torch.full((2 * n,), float("nan"), dtype=torch.float32, device="cuda")
    dot_poisson_f32_noalloc(D, T, N, torch.from_numpy(b).cuda(), out)
    pair = out.cpu().numpy().astype(np.float64).reshape(n, 2)
    want = O.poisson(O.Grid(D, T, N), b.astype(np.float64))
    assert rel_err(centred(pair[:, 0] + pair[:, 1]), centred(want)) < refined_tol(T, N)
