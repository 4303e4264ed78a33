"""Pins of the phi_j functions and the weights b_i of Eq. (3-12).

Independent routes: an arbitrary-precision quadrature of the integral
definitions (mpmath, where installed), exact rational integration of the
Lagrange basis at z = 0 (the Newton-Cotes weights), and closed forms.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import phi
from paper_2412_01138_gb300 import inputs as I

Z_GRID = -np.logspace(-14, 4, 61)


def _lagrange_coeffs_exact(c):
    """Monomial coefficients of each Lagrange basis polynomial, exactly (Fractions)."""
    s = len(c)
    out = []
    for i in range(s):
        poly = [Fraction(1)]
        for m in range(s):
            if m == i:
                continue
            den = c[i] - c[m]
            # multiply by (theta - c_m)/den
            new = [Fraction(0)] * (len(poly) + 1)
            for k, a in enumerate(poly):
                new[k + 1] += a / den
                new[k] -= a * c[m] / den
            poly = new
        out.append(poly)
    return out


@pytest.mark.parametrize("nodes", [(0, Fraction(1, 2)), (0, Fraction(1, 3), Fraction(2, 3)),
                                   (0, Fraction(1, 4), Fraction(1, 2), Fraction(3, 4)),
                                   (0, 1), (Fraction(1, 5), Fraction(7, 10))])
def test_b_at_zero_is_newton_cotes(nodes):
    """b_i(0) = int_0^1 l_i: exact rational integration of the Lagrange basis."""
    exact = [float(sum(a / (k + 1) for k, a in enumerate(poly))) for poly in _lagrange_coeffs_exact(list(nodes))]
    got = phi.b_weights(np.array([0.0]), [float(c) for c in nodes])[:, 0]
    np.testing.assert_allclose(got, exact, rtol=0, atol=2e-15)


def test_newton_cotes_known_values():
    """The limits quoted for the tableaux used by the benchmark workloads."""
    z0 = np.array([0.0])
    np.testing.assert_allclose(phi.b_weights(z0, [0, 0.5])[:, 0], [0, 1], atol=1e-15)
    np.testing.assert_allclose(phi.b_weights(z0, [0, 1 / 3, 2 / 3])[:, 0], [0.25, 0, 0.75], atol=1e-15)
    np.testing.assert_allclose(phi.b_weights(z0, [0, 0.25, 0.5, 0.75])[:, 0], [0, 2 / 3, -1 / 3, 2 / 3], atol=1e-15)
    np.testing.assert_allclose(phi.b_weights(z0, [0, 1])[:, 0], [0.5, 0.5], atol=1e-15)


def test_phi_at_zero():
    v = phi.phi_functions(np.array([0.0]), 6)[:, 0]
    np.testing.assert_allclose(v, [1 / math.factorial(j) for j in range(1, 7)], rtol=1e-16)


def test_phi_closed_forms():
    """phi_1 = (e^z - 1)/z, phi_2 = (e^z - 1 - z)/z^2 where these are well conditioned."""
    z = -np.array([3.0, 7.5, 40.0, 1e3, 1.2e4])
    v = phi.phi_functions(z, 2)
    np.testing.assert_allclose(v[0], (np.exp(z) - 1) / z, rtol=1e-15)
    np.testing.assert_allclose(v[1], (np.exp(z) - 1 - z) / z ** 2, rtol=1e-14)


@pytest.mark.parametrize("nodes", [I.uniform_nodes(2), I.uniform_nodes(3), I.uniform_nodes(4),
                                   I.draw_random_nodes(2, 2), I.draw_random_nodes(4, 17)])
def test_b_phi_identity(nodes):
    """sum_i b_i c_i^{j-1}/(j-1)! = phi_j for 1 <= j <= s (Theorem 3.1's proof)."""
    s = len(nodes)
    b = phi.b_weights(Z_GRID, nodes)
    ph = phi.phi_functions(Z_GRID, s)
    for j in range(1, s + 1):
        lhs = sum(b[i] * nodes[i] ** (j - 1) for i in range(s)) / math.factorial(j - 1)
        np.testing.assert_allclose(lhs, ph[j - 1], rtol=1e-12, atol=0)


def test_phi_against_arbitrary_precision():
    """phi_j(z), j <= 4, to ~1e-15 against 40-digit quadrature of its integral definition."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    zs = -np.logspace(-14, 4, 37)
    got = phi.phi_functions(zs, 4)
    for zi, z in enumerate(zs):
        zm = mp.mpf(float(z))
        pts = [0, 1] if abs(z) < 50 else [0, 1 - 50 / abs(z), 1]
        for j in range(1, 5):
            ref = mp.quad(lambda t: mp.e ** (zm * (1 - t)) * t ** (j - 1) / mp.factorial(j - 1), pts)
            assert abs((mp.mpf(float(got[j - 1, zi])) - ref) / ref) < 2e-15


@pytest.mark.parametrize("nodes", [I.uniform_nodes(2), I.uniform_nodes(4), I.draw_random_nodes(2, 2)])
def test_b_against_direct_integral(nodes):
    """b_i(z) against 40-digit quadrature of Eq. (3-12) itself (no phi, no Vandermonde)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    c = [mp.mpf(float(v)) for v in nodes]
    s = len(c)
    zs = -np.array([1e-12, 1e-6, 1e-3, 0.077, 0.5, 1.9, 2.1, 9.7, 383.0, 1.2e4])
    got = phi.b_weights(zs, nodes)
    for zi, z in enumerate(zs):
        zm = mp.mpf(float(z))
        pts = [0, 1] if abs(z) < 50 else [0, 1 - 50 / abs(z), 1]
        for i in range(s):
            def li(t, i=i):
                out = mp.mpf(1)
                for m in range(s):
                    if m != i:
                        out *= (t - c[m]) / (c[i] - c[m])
                return out
            ref = mp.quad(lambda t: mp.e ** (zm * (1 - t)) * li(t), pts)
            scale = max(abs(ref), mp.mpf(1) / (1 + abs(zm)))
            assert abs(mp.mpf(float(got[i, zi])) - ref) / scale < 1e-13


def test_duplicate_nodes_rejected():
    with pytest.raises(ValueError):
        phi.b_weights(np.array([-1.0]), [0.5, 0.5])
