"""Non-homogeneous Dirichlet data by lifting (the extension the paper calls straightforward).

Test infrastructure only (see ``oracle/__init__``).

The paper treats u = 0 on the boundary and remarks (openings of Sec. 3 and
Sec. 4) that its results extend to non-homogeneous Dirichlet data, without
formulas.  The reading used here: the data are given as separable terms
g(t, x) on the closed box; the lifting is their Q1 interpolant I_h g on ALL nodes (boundary nodes take
the data, interior nodes the interpolated values), and the unknown is
w = u_h - I_h g, which vanishes on the boundary.  Testing the weak form with the
interior hat functions phi_i gives the homogeneous problem of Sec. 2.1 with the
extra load

    r_i(t) = -( M_full d/dt(I_h g)(t) + K_full (I_h g)(t) )_i ,

where M_full, K_full are the Q1 mass and stiffness matrices of the whole grid
(boundary nodes included, rows restricted to interior nodes).  The initial value
is w(t0) = P_h(u0 - I_h g(t0)) (the L2 projection of the lifted data), and the
discrete solution on interior nodes is u_h = w + I_h g.

Here M_full and K_full are assembled as explicit Kronecker products of the 1D
rectangular blocks (interior rows, all columns) and applied to the full nodal
vector of I_h g: no separable shortcut is taken.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import quadrature


def full_axis(lo: float, hi: float, n: int):
    """Mesh size and coordinates of all n + 2 nodes of one axis (boundary included)."""
    h = (hi - lo) / (n + 1)
    return h, lo + h * np.arange(0, n + 2, dtype=np.float64)


def rows_mass_1d(n: int, h: float) -> sp.csr_matrix:
    """Interior rows of the 1D P1 mass matrix of the full grid: (h/6) [1 4 1] per row."""
    A = sp.lil_matrix((n, n + 2))
    for k in range(n):
        A[k, k] = h / 6.0
        A[k, k + 1] = 4.0 * h / 6.0
        A[k, k + 2] = h / 6.0
    return A.tocsr()


def rows_stiffness_1d(n: int, h: float) -> sp.csr_matrix:
    """Interior rows of the 1D P1 stiffness matrix of the full grid: (1/h) [-1 2 -1] per row."""
    A = sp.lil_matrix((n, n + 2))
    for k in range(n):
        A[k, k] = -1.0 / h
        A[k, k + 1] = 2.0 / h
        A[k, k + 2] = -1.0 / h
    return A.tocsr()


def eval_time_derivative(term, t: float) -> float:
    """d/dt of a term's time factor (exp(a t) or sin(w t + phi)), written out."""
    a, b = term.tp
    if term.tkind == 1:  # T_SIN
        return a * np.cos(a * t + b)
    return a * np.exp(a * t)


class DirichletLift:
    """The lifting of separable boundary data on one grid (C-ordered arrays)."""

    def __init__(self, prob):
        self.prob = prob
        d = prob.d
        Ms, Ks, self.coords = [], [], []
        for a in range(d):
            h, x = full_axis(prob.box[a][0], prob.box[a][1], prob.n[a])
            Ms.append(rows_mass_1d(prob.n[a], h))
            Ks.append(rows_stiffness_1d(prob.n[a], h))
            self.coords.append(x)

        def kron_all(mats):
            out = mats[0]
            for m in mats[1:]:
                out = sp.kron(out, m, format="csr")
            return out

        self.M_rows = kron_all(Ms)
        K = None
        for a in range(d):
            term = kron_all([Ks[b] if b == a else Ms[b] for b in range(d)])
            K = term if K is None else K + term
        self.K_rows = (prob.D * K).tocsr()

    def full_values(self, t: float, derivative: bool = False) -> np.ndarray:
        """Nodal values of I_h g(t) (or of its time derivative) on the full grid, flattened."""
        out = np.zeros(tuple(len(x) for x in self.coords))
        for term in self.prob.boundary:
            vals = [quadrature.eval_factor(f, x) for f, x in zip(term.factors, self.coords)]
            prod = vals[0]
            for v in vals[1:]:
                prod = np.multiply.outer(prod, v)
            tf = eval_time_derivative(term, t) if derivative else quadrature.eval_time(term, t)
            out = out + term.amp * tf * prod
        return out.reshape(-1)

    def interior(self, t: float) -> np.ndarray:
        """I_h g(t) on the interior nodes, shape n."""
        full = self.full_values(t).reshape(tuple(len(x) for x in self.coords))
        return full[tuple(slice(1, -1) for _ in self.coords)]

    def extra_load(self, t: float) -> np.ndarray:
        """r(t) = -(M_full dI_h g/dt + K_full I_h g) on interior rows, shape n."""
        r = -(self.M_rows @ self.full_values(t, derivative=True) + self.K_rows @ self.full_values(t))
        return r.reshape(self.prob.n)

    def lift_load(self, t: float) -> np.ndarray:
        """(I_h g(t), phi_i) = (M_full I_h g(t))_i, shape n (its L2 projection's load)."""
        return (self.M_rows @ self.full_values(t)).reshape(self.prob.n)
