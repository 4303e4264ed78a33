"""Pins of the oracle's non-homogeneous Dirichlet lifting (oracle/dirichlet.py).

* A multilinear function is discretely harmonic (its Q1 stiffness rows vanish on
  interior nodes), so with f = 0, u0 = g and time-constant data the solution stays
  g exactly, in 1D, 2D and 3D.
* For time-constant data the lifted problem is affine and EIFE integrates constant
  forcing exactly; the result must equal the exact solution of the eliminated
  system M_ii c' + K_ii c = -K_ib g_b (boundary nodes moved to the right-hand
  side), computed here by a dense matrix exponential -- a different formulation.
* u = e^{a t} q with q multilinear and f = a u: the lifted unknown w is identically
  zero, which holds only if the d/dt(I_h g) mass term cancels f exactly.
* Oscillating, non-harmonic data with f = 0: the error against a 512-substep run
  falls at the tableau's order.
* 1D heat with constant end values alpha, beta: u = alpha + (beta - alpha) x +
  e^{-D pi^2 t} sin(pi x); the error is O(h^2).
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import dirichlet, quadrature
from oracle import solver as osolver
from paper_2412_01138_gb300 import inputs as I


def _poly(c0, c1, c2=0.0):
    return I.Factor(I.S_POLY, (c0, c1, c2, 0.0))


def _problem(d, n, boundary, u0, forcing, D=0.3, N=4, M=8, q=3, T=1.0):
    box = ((0.0, 1.0), (0.0, 2.0), (0.0, 1.5))[:d]
    return I.Problem(d, tuple(n), box, D, 0.0, T, N, M, I.uniform_nodes(q), I.uniform_nodes(2),
                     tuple(u0), tuple(forcing), 3, 1e-12, None, "dirichlet", tuple(boundary))


@pytest.mark.parametrize("d,n", [(1, (17,)), (2, (9, 11)), (3, (5, 6, 7))])
def test_harmonic_data_is_stationary(d, n):
    facs = tuple(_poly(1.0 + a, 2.0 - 0.5 * a) for a in range(d))
    g = (I.Term(1.7, facs, I.T_EXP, (0.0, 0.0)),)
    prob = _problem(d, n, g, (I.Term(1.7, facs),), ())
    sys_ = osolver.ModalSystem(prob)
    out = osolver.sequential_fine(sys_)
    lift = dirichlet.DirichletLift(prob)
    for k in range(prob.N + 1):
        t = prob.t0 + k * prob.T / prob.N
        u = sys_.solution_nodal(out[k], t)
        assert np.abs(u - lift.interior(t)).max() <= 1e-13 * np.abs(lift.interior(t)).max()


def _full_matrices(prob):
    Ms, Ks, nfull = [], [], []
    for a in range(prob.d):
        na = prob.n[a]
        h = (prob.box[a][1] - prob.box[a][0]) / (na + 1)
        m = (h / 6.0) * (np.diag(np.r_[2.0, 4.0 * np.ones(na), 2.0]) + np.eye(na + 2, k=1) + np.eye(na + 2, k=-1))
        kk = (1.0 / h) * (np.diag(np.r_[1.0, 2.0 * np.ones(na), 1.0]) - np.eye(na + 2, k=1) - np.eye(na + 2, k=-1))
        Ms.append(m)
        Ks.append(kk)
        nfull.append(na + 2)

    def kron_all(mats):
        out = mats[0]
        for x in mats[1:]:
            out = np.kron(out, x)
        return out

    M = kron_all(Ms)
    K = sum(kron_all([Ks[b] if b == a else Ms[b] for b in range(prob.d)]) for a in range(prob.d))
    inner = np.zeros(nfull, dtype=bool)
    inner[tuple(slice(1, -1) for _ in nfull)] = True
    return M, prob.D * K, inner.reshape(-1), nfull


def test_time_constant_data_matches_eliminated_system():
    prob = _problem(2, (6, 7), (I.Term(1.0, (I.Factor(I.S_SIN, (1.3, 0.4)), _poly(0.5, 1.0, -0.7)),
                                         I.T_EXP, (0.0, 0.0)),),
                    (I.Term(1.0, (I.Factor(I.S_SIN, (math.pi, 0.0)), I.Factor(I.S_SIN, (math.pi / 2, 0.0)))),),
                    (), D=0.2, N=3, M=5)
    sys_ = osolver.ModalSystem(prob, basis="dense")
    out = osolver.sequential_fine(sys_)
    M, K, inner, nfull = _full_matrices(prob)
    bd = ~inner
    lift = dirichlet.DirichletLift(prob)
    gfull = lift.full_values(0.0)
    Mii, Kii, Kib = M[np.ix_(inner, inner)], K[np.ix_(inner, inner)], K[np.ix_(inner, bd)]
    rhs = -Kib @ gfull[bd]
    steady = np.linalg.solve(Kii, rhs)
    # initial interior values: P_h(u0 - I_h g) + I_h g on interior nodes
    F0 = quadrature.load_full(prob.u0, None, prob.n, prob.box, prob.quad_pts).reshape(-1)
    w0 = np.linalg.solve(Mii, F0 - (M[inner] @ gfull))
    c0 = w0 + gfull[inner]
    A = np.linalg.solve(Mii, Kii)
    for k in range(prob.N + 1):
        t = k * prob.T / prob.N
        exact = steady + scipy.linalg.expm(-A * t) @ (c0 - steady)
        got = sys_.solution_nodal(out[k], t).reshape(-1)
        assert np.abs(got - exact).max() <= 1e-12 * np.abs(exact).max(), k


def _exp_problem(M, q):
    a = -0.8
    facs = (_poly(1.0, 2.0), _poly(3.0, -1.0))
    g = (I.Term(1.0, facs, I.T_EXP, (a, 0.0)),)
    f = (I.Term(a, facs, I.T_EXP, (a, 0.0)),)  # u_t - D lap u = a u for multilinear u
    return _problem(2, (7, 9), g, (I.Term(1.0, facs),), f, D=0.5, N=2, M=M, q=q), a, facs


def test_exponential_data_is_reproduced_exactly():
    """u = e^{a t} q: the lifted unknown w stays 0 only if the d/dt(I_h g) term cancels f."""
    prob, a, facs = _exp_problem(6, 3)
    sys_ = osolver.ModalSystem(prob)
    out = osolver.sequential_fine(sys_)
    lift = dirichlet.DirichletLift(prob)
    for k in range(prob.N + 1):
        t = k * prob.T / prob.N
        exact = math.exp(a * t) * lift.interior(0.0)
        assert np.abs(sys_.solution_nodal(out[k], t) - exact).max() <= 1e-13 * np.abs(exact).max()


@pytest.mark.parametrize("q", [2, 3])
def test_time_dependent_data_converges_at_tableau_order(q):
    """f = 0, u0 = 0 inside, oscillating non-harmonic data: self-convergence in the substep count."""
    g = (I.Term(1.0, (I.Factor(I.S_SIN, (2.0, 0.3)), _poly(1.0, 0.0, 1.0)), I.T_SIN, (3.0, 0.2)),)

    def run(M):
        prob = _problem(2, (7, 9), g, (), (), D=0.5, N=2, M=M, q=q)
        sys_ = osolver.ModalSystem(prob)
        return sys_.solution_nodal(osolver.sequential_fine(sys_)[-1], prob.T)

    ref = run(512)
    errs = [np.abs(run(M) - ref).max() for M in (8, 16, 32)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - q) < 0.3 for r in rates), (errs, rates)


def test_heat_with_constant_end_values_is_second_order():
    D, alpha, beta = 0.4, 1.5, -0.5
    errs = []
    for nx in (16, 32, 64):
        box = ((0.0, 1.0),)
        g = (I.Term(1.0, (_poly(alpha, beta - alpha),), I.T_EXP, (0.0, 0.0)),)
        u0 = (I.Term(1.0, (_poly(alpha, beta - alpha),)), I.Term(1.0, (I.Factor(I.S_SIN, (math.pi, 0.0)),)))
        prob = I.Problem(1, (nx - 1,), box, D, 0.0, 0.5, 4, 32, I.uniform_nodes(4), I.uniform_nodes(2),
                         u0, (), 3, 1e-12, None, "heat", g)
        sys_ = osolver.ModalSystem(prob)
        out = osolver.sequential_fine(sys_)
        u = sys_.solution_nodal(out[-1], prob.T)
        x = np.linspace(0.0, 1.0, nx + 1)[1:-1]
        ue = alpha + (beta - alpha) * x + math.exp(-D * math.pi ** 2 * prob.T) * np.sin(math.pi * x)
        errs.append(np.abs(u - ue).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - 2.0) < 0.2 for r in rates), (errs, rates)
