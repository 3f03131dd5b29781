"""Host part of the trajectory mode: the finite differences behind the
critical-point estimate from d<H>/d lambda and d^2<H>/d lambda^2 (Sec. 3.2).
Pinned by closed forms: three-point differences are exact on quadratics, the
first derivative converges at second order inside the grid, and the largest
|y''| of a smoothed kink sits at the kink."""
import numpy as np
import pytest

import paper_1910_08020_gb300 as z2


def test_exact_on_quadratics_on_uneven_grids():
    rng = np.random.default_rng(7)
    for _ in range(20):
        x = np.cumsum(rng.uniform(0.05, 0.5, size=9))
        a, b, c = rng.normal(size=3)
        dy, d2y, _ = z2.finite_differences(x, a * x * x + b * x + c)
        assert np.max(np.abs(dy - (2 * a * x + b))) < 1e-10 * (1 + abs(a) + abs(b))
        assert np.max(np.abs(d2y - 2 * a)) < 1e-9 * (1 + abs(a))


def test_second_order_inside_the_grid():
    errs = []
    for n in (21, 41, 81):
        x = np.linspace(0.0, 2.0, n)
        dy, _, _ = z2.finite_differences(x, np.sin(x))
        errs.append(np.max(np.abs(dy[1:-1] - np.cos(x[1:-1]))))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_critical_point_at_the_kink():
    # E(lambda) = -sqrt(1 + ((lambda - lc) / w)^2): |E''| peaks at lambda = lc
    lc, w = 3.04, 0.2
    x = np.linspace(2.0, 4.0, 201)
    _, _, xc = z2.finite_differences(x, -np.sqrt(1 + ((x - lc) / w) ** 2))
    assert abs(xc - lc) <= 0.01


@pytest.mark.parametrize("x,y", [([0, 1], [0, 1]), ([0, 1, 1], [0, 1, 2]), ([0, 2, 1], [0, 1, 2]),
                                 ([0, 1, 2], [0, 1])])
def test_rejects_bad_grids(x, y):
    with pytest.raises(ValueError):
        z2.finite_differences(x, y)
