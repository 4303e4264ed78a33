"""phi_j functions and the exponential Runge-Kutta weights b_i of Eq. (3-12).

Test infrastructure only (see ``oracle/__init__``).

Eq. (3-12): b_i(z) = int_0^1 e^{z(1-theta)} l_i(theta) dtheta with l_i the
Lagrange basis on distinct nodes c_1..c_s in [0,1].  The proof of
Theorem 3.1 defines phi_j(z) = int_0^1 e^{z(1-theta)} theta^{j-1}/(j-1)! dtheta
and shows sum_i b_i c_i^{j-1}/(j-1)! = phi_j for 1 <= j <= s.  The oracle
takes exactly that identity as the definition of the weights: it solves the
s x s (transposed Vandermonde) system sum_i b_i c_i^m = m! phi_{m+1}(z),
m = 0..s-1.

phi_j is evaluated in float64 by the Taylor series
phi_j(z) = sum_{k>=0} z^k/(k+j)! for |z| < PHI_SERIES_RADIUS and by the
recurrence phi_1 = expm1(z)/z, phi_{j+1} = (phi_j - 1/j!)/z beyond it.
Pinned in tests against an arbitrary-precision quadrature of the integral
definitions, phi_j(0) = 1/j! and the Newton-Cotes limits of b_i.
"""
from __future__ import annotations

import math

import numpy as np

#: |z| below which the Taylor series is used (chosen by the precision test
#: against the arbitrary-precision reference over z in -logspace(-14, 6)).
PHI_SERIES_RADIUS = 2.0
_SERIES_TERMS = 30


def phi_functions(z, s: int) -> np.ndarray:
    """phi_1(z) .. phi_s(z) for real z (any sign); returns shape (s,) + z.shape."""
    z = np.asarray(z, dtype=np.float64)
    out = np.empty((s,) + z.shape, dtype=np.float64)
    small = np.abs(z) < PHI_SERIES_RADIUS
    zs = np.where(small, z, 0.0)
    for j in range(1, s + 1):
        acc = np.zeros_like(z)
        # Horner on sum_{k=0}^{K} z^k/(k+j)!
        for k in range(_SERIES_TERMS, -1, -1):
            acc = acc * zs + 1.0 / math.factorial(k + j)
        out[j - 1] = acc
    zl = np.where(small, 1.0, z)
    rec = np.expm1(zl) / zl
    big = ~small
    out[0] = np.where(big, rec, out[0])
    for j in range(1, s):
        rec = (rec - 1.0 / math.factorial(j)) / zl
        out[j] = np.where(big, rec, out[j])
    return out


def b_weights(z, nodes) -> np.ndarray:
    """b_i(z), i = 1..s, for the nodes c_i; returns shape (s,) + z.shape.

    Solves sum_i b_i c_i^m = m! phi_{m+1}(z), m = 0..s-1 (the identity of
    Theorem 3.1's proof, equivalent to Eq. (3-12)).
    """
    c = np.asarray(nodes, dtype=np.float64)
    s = len(c)
    if len(set(c.tolist())) != s:
        raise ValueError("interpolation nodes must be distinct")
    z = np.asarray(z, dtype=np.float64)
    ph = phi_functions(z, s)
    rhs = np.stack([math.factorial(m) * ph[m] for m in range(s)], axis=0).reshape(s, -1)
    V = np.array([[ci ** m for ci in c] for m in range(s)])  # V[m, i] = c_i^m
    b = np.linalg.solve(V, rhs)
    return b.reshape((s,) + z.shape)
