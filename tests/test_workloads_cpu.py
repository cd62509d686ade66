"""The analytic examples Ex-1 .. Ex-4 of Sec. 5 as sampled by workloads.paper_example."""
import numpy as np
import pytest

from paper_2505_05424_gb300 import workloads as W


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("delta", [0.0, 0.05])
def test_unit_mass_plus_floor(k, delta):
    N = 40
    r0, r1 = W.paper_example(k, N, delta)
    for r in (r0, r1):
        assert r.shape == (N * N,)
        # mass 1 on the unit square before the floor: mean of the samples is 1 + delta
        assert abs(r.mean() - (1.0 + delta)) < 1e-12
        assert r.min() >= delta


def test_ex1_is_a_mirror_image():
    # rho_1(x1, x2) = rho_0(x2, x1): the Gaussian at (0.25, 0.75) moves to (0.75, 0.25)
    N = 32
    r0, r1 = W.paper_example(1, N)
    np.testing.assert_array_equal(r1.reshape(N, N), r0.reshape(N, N).T)
    i = np.argmax(r0.reshape(N, N))
    assert np.unravel_index(i, (N, N)) in {(N // 4 - 1, 3 * N // 4 - 1), (N // 4, 3 * N // 4)}


def test_ex2_to_ex4_share_the_four_gaussian_target():
    N = 36
    targets = [W.paper_example(k, N)[1] for k in (2, 3, 4)]
    np.testing.assert_array_equal(targets[0], targets[1])
    np.testing.assert_array_equal(targets[0], targets[2])
    t = targets[0].reshape(N, N)
    # symmetric under both reflections of the square, four maxima at the quarter points
    np.testing.assert_allclose(t, t[::-1, :], rtol=1e-12)
    np.testing.assert_allclose(t, t[:, ::-1], rtol=1e-12)
    np.testing.assert_allclose(t, t.T, rtol=1e-12)


def test_ex4_source_vanishes_at_the_centre_only():
    N = 64
    r0 = W.paper_example(4, N)[0].reshape(N, N)
    # (x1 - 1/2)^4 + (x2 - 1/2)^4: minimal at the four centre cells, largest at the corners
    c = r0[N // 2 - 1:N // 2 + 1, N // 2 - 1:N // 2 + 1]
    assert np.allclose(c, r0.min())
    assert r0[0, 0] == r0.max()


def test_named_workloads():
    for name in ("ex1", "ex2", "ex3", "ex4"):
        spec, r0, r1, mask = W.workload(name)
        assert (spec.D, spec.T, spec.N) == (2, 32, 128)
        assert mask is None and r0.size == r1.size == 128 * 128
