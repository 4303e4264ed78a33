"""Pins of the oracle's periodic axes (circulant Q1 matrices diagonalised by the DHT).

* The discrete Hartley matrix is symmetric and an involution.
* H M H and H K H of the assembled circulant matrices are diagonal with the closed-form
  periodic spectra (theta_j = 2 pi j / n).
* The dense generalized eigensolve route and the closed-form route give the same solution.
* With every axis periodic and f = 0 the integral of u_h is conserved (the constant mode
  has lam = 0) exactly.
* Fourier-mode exact solutions (1D periodic; 2D periodic x Dirichlet) converge at O(h^2).
* The separable 1D loads and the full d-D element quadrature agree on periodic axes.
"""
import math

import numpy as np
import pytest

from oracle import fem, quadrature
from oracle import solver as osolver
from paper_2412_01138_gb300 import inputs as I


@pytest.mark.parametrize("n", [1, 2, 7, 16, 33])
def test_dht_is_a_symmetric_involution(n):
    H = fem.dht_matrix(n)
    assert np.abs(H - H.T).max() <= 1e-15
    assert np.abs(H @ H - np.eye(n)).max() <= 1e-13


@pytest.mark.parametrize("n,L", [(8, 1.0), (15, 2.5), (32, 0.7)])
def test_circulant_spectra(n, L):
    h = L / n
    H = fem.dht_matrix(n)
    muM, muK = fem.axis_eigenvalues_periodic(n, h)
    for A, mu in ((fem.mass_1d_periodic(n, h), muM), (fem.stiffness_1d_periodic(n, h), muK)):
        B = H @ A @ H
        assert np.abs(B - np.diag(np.diag(B))).max() <= 1e-12 * np.abs(A).max()
        assert np.allclose(np.diag(B), mu, rtol=0, atol=1e-12 * np.abs(A).max())


def _problem(n, periodic, box, D=0.2, N=3, M=5, forcing=True, q=3):
    d = len(n)
    u0 = (I.Term(1.0, tuple(I.Factor(I.S_SIN, (2 * math.pi * (a + 1) / (box[a][1] - box[a][0]), 0.3))
                            for a in range(d))),
          I.Term(0.7, tuple(I.Factor(I.S_POLY, (1.0, 0.2, -0.1, 0.0)) for a in range(d))))
    f = ()
    if forcing:
        f = (I.Term(0.5, tuple(I.Factor(I.S_GAUSS, (0.4 * (box[a][1] - box[a][0]) + box[a][0], 0.15))
                               for a in range(d)), I.T_SIN, (3.0, 0.2)),)
    return I.Problem(d, tuple(n), tuple(box), D, 0.0, 1.0, N, M, I.uniform_nodes(q), I.uniform_nodes(2),
                     u0, f, 3, 1e-12, None, "periodic", (), tuple(periodic))


@pytest.mark.parametrize("n,periodic", [((9,), (True,)), ((6, 7), (True, False)), ((5, 4, 6), (True, True, False)),
                                        ((6, 5), (True, True))])
def test_dense_and_closed_form_routes_agree(n, periodic):
    box = ((0.0, 1.0), (-0.5, 1.0), (0.0, 2.0))[:len(n)]
    prob = _problem(n, periodic, box)
    a = osolver.ModalSystem(prob)
    b = osolver.ModalSystem(prob, basis="dense")
    ua = a.to_nodal(osolver.sequential_fine(a)[-1])
    ub = b.to_nodal(osolver.sequential_fine(b)[-1])
    assert np.abs(ua - ub).max() <= 1e-12 * np.abs(ua).max()


def test_integral_is_conserved_when_every_axis_is_periodic():
    box = ((0.0, 1.0), (0.0, 2.0))
    prob = _problem((12, 10), (True, True), box, forcing=False, N=4, M=8)
    sys_ = osolver.ModalSystem(prob)
    out = osolver.sequential_fine(sys_)
    M, _ = fem.assemble(prob.n, box, prob.D, prob.periodic)
    ones = np.ones(prob.ndof)
    mass = [ones @ (M @ sys_.to_nodal(c).reshape(-1)) for c in out]
    assert np.abs(np.array(mass) - mass[0]).max() <= 1e-13 * abs(mass[0])
    assert np.abs(sys_.lam.reshape(-1)[0]) == 0.0


def _fourier_error(nx, two_d):
    D, T, L = 0.3, 0.4, 2.0
    kx = 2 * math.pi * 2 / L
    if two_d:
        box = ((0.0, L), (0.0, 1.0))
        n, per = (nx, nx - 1), (True, False)
        u0 = (I.Term(1.0, (I.Factor(I.S_SIN, (kx, math.pi / 2)), I.Factor(I.S_SIN, (math.pi, 0.0)))),)
        rate = D * (kx ** 2 + math.pi ** 2)
    else:
        box = ((0.0, L),)
        n, per = (nx,), (True,)
        u0 = (I.Term(1.0, (I.Factor(I.S_SIN, (kx, math.pi / 2)),)),)
        rate = D * kx ** 2
    prob = I.Problem(len(n), n, box, D, 0.0, T, 2, 64, I.uniform_nodes(4), I.uniform_nodes(2), u0, (), 3, 1e-12,
                     None, "fourier", (), per)
    sys_ = osolver.ModalSystem(prob)
    u = sys_.to_nodal(osolver.sequential_fine(sys_)[-1])
    _, x = fem.axis_grid(0.0, L, nx, True)
    exact = math.exp(-rate * T) * np.cos(kx * x)
    if two_d:
        _, y = fem.axis_grid(0.0, 1.0, nx - 1)
        exact = np.multiply.outer(exact, np.sin(math.pi * y))
    return np.abs(u - exact).max()


@pytest.mark.parametrize("two_d", [False, True])
def test_fourier_mode_converges_second_order(two_d):
    errs = [_fourier_error(nx, two_d) for nx in (16, 32, 64)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - 2.0) < 0.15 for r in rates), (errs, rates)


@pytest.mark.parametrize("n,periodic", [((11,), (True,)), ((7, 9), (True, False)), ((6, 5), (True, True))])
def test_separable_and_full_loads_agree(n, periodic):
    box = ((0.0, 1.0), (0.0, 1.3))[:len(n)]
    prob = _problem(n, periodic, box)
    term = prob.forcing[0]
    loads = quadrature.separable_load_factors(term, prob.n, box, 3, periodic)
    sep = term.amp * fem.outer_all(loads)
    full = quadrature.load_full((I.Term(term.amp, term.factors),), None, prob.n, box, 3, periodic)
    assert np.abs(sep - full).max() <= 1e-14 * np.abs(full).max()
