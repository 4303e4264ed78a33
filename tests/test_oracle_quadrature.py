"""Pins of the consistent loads, P_h and the element-quadrature L2 norm (Sec. 2.1, Sec. 5)."""
import numpy as np
import pytest

from oracle import fem, quadrature, solver
from paper_2412_01138_gb300 import inputs as I


def test_gauss_rule_exact_degree():
    for qp in (1, 2, 3, 5):
        s, w = quadrature.gauss_legendre(qp)
        for k in range(2 * qp):
            assert np.sum(w * s ** k) == pytest.approx(1.0 / (k + 1), rel=1e-14)


def test_load_1d_polynomials():
    """F_k = int g phi_k: g = 1 -> h; g = x -> h x_k; g = x^2 -> h x_k^2 + h^3/6."""
    lo, hi, n = 0.2, 1.7, 9
    h, x = fem.axis_grid(lo, hi, n)
    np.testing.assert_allclose(quadrature.load_1d(lambda t: np.ones_like(t), lo, hi, n, 2), h * np.ones(n), rtol=1e-14)
    np.testing.assert_allclose(quadrature.load_1d(lambda t: t, lo, hi, n, 2), h * x, rtol=1e-14)
    np.testing.assert_allclose(quadrature.load_1d(lambda t: t * t, lo, hi, n, 2), h * x * x + h ** 3 / 6, rtol=1e-14)


@pytest.mark.parametrize("n", [(5, 4), (3, 4, 2)])
def test_full_load_equals_separable_outer_product(n):
    d = len(n)
    box = tuple((0.1 * a, 1.0 + 0.2 * a) for a in range(d))
    bumps = I.gaussian_bumps(I.SplitMix64(3), d, 2, width=(0.2, 0.3))
    for term in bumps:
        full = quadrature.load_full((term,), 0.37, n, box, 3)
        sep = term.amp * quadrature.eval_time(term, 0.37) * fem.outer_all(
            quadrature.separable_load_factors(term, n, box, 3))
        np.testing.assert_allclose(full, sep, rtol=1e-13, atol=1e-16)


def test_projection_is_L2_orthogonal():
    """(u - P_h u, phi_k) = 0 for every hat, checked with an independent 8-point rule."""
    n, lo, hi = 7, 0.0, 1.0
    g = lambda x: np.exp(x) * np.sin(3 * x)
    h, x = fem.axis_grid(lo, hi, n)
    basis = fem.ClosedFormBasis((n,), ((lo, hi),), 1.0)
    c = basis.to_modal_from_load(quadrature.load_1d(g, lo, hi, n, 6))
    uh = basis.to_nodal(c)
    V = np.concatenate([[0.0], uh, [0.0]])
    s, w = np.polynomial.legendre.leggauss(8)
    s, w = 0.5 * (s + 1), 0.5 * w
    resid = np.zeros(n + 2)
    for e in range(n + 1):
        xq = lo + (e + s) * h
        r = g(xq) - (V[e] * (1 - s) + V[e + 1] * s)
        resid[e] += h * np.sum(w * r * (1 - s))
        resid[e + 1] += h * np.sum(w * r * s)
    assert np.abs(resid[1:-1]).max() < 1e-12


def test_l2_norm_of_fe_function_matches_mass_matrix():
    n, box = (4, 3), ((0.0, 1.0), (0.0, 2.0))
    rng = np.random.default_rng(0)
    u = rng.standard_normal(n)
    M, _ = fem.assemble(n, box, 1.0)
    zero = (I.Term(0.0, (I.Factor(I.S_ONE), I.Factor(I.S_ONE))),)
    got = quadrature.l2_error_full(u, zero, 0.0, n, box, 5)
    assert got == pytest.approx(np.sqrt(u.reshape(-1) @ (M @ u.reshape(-1))), rel=1e-13)


def test_moving_hat_load_matches_fine_quadrature():
    """The 3-point element rule on the moving hat against a 400-point rule (kinks make it inexact:
    the two differ by O(h^3) per element near the kinks only)."""
    prob = I.example4(32, 0.01, 1.0)
    term = prob.forcing[0]
    for t in (0.0, 0.13, 0.61):
        F3 = quadrature.load_full(prob.forcing, t, prob.n, prob.box, 3)
        F400 = quadrature.load_full(prob.forcing, t, prob.n, prob.box, 400)
        assert np.abs(F3 - F400).max() <= 0.05 * np.abs(F400).max()
        assert np.abs(F400.sum() - term.amp * 0.05) < 1e-6  # integral of the hat times sum of hats = area
