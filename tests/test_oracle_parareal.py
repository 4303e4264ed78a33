"""Pins of the EIFE stepping and of Algorithm 1 (Sec. 2.2-2.3, Theorems 3.1 and 4.3)."""
import math

import numpy as np
import pytest

from oracle import fem, quadrature, solver
from paper_2412_01138_gb300 import inputs as I


def _bump_problem(N=6, M=5, seed=7):
    rng = I.SplitMix64(seed)
    box = ((0.0, 1.0), (0.0, 1.0))
    u0, f, _ = I.sin_mode(2, box, 0.2)
    bumps = I.gaussian_bumps(rng, 2, 4)
    return I.Problem(2, (15, 11), box, 0.2, 0.0, 1.0, N, M, I.uniform_nodes(4), I.draw_random_nodes(2, seed),
                     u0, f + bumps, 3)


def _rel(a, b, sys):
    return sys.norm(a - b) / sys.norm(b)


def test_k0_is_sequential_coarse():
    prob = _bump_problem()
    sys = solver.ModalSystem(prob)
    res = solver.parareal(sys, tol=0.0, k_max=0)
    c = solver.sequential_eife(sys, prob.N, prob.coarse_nodes)
    assert _rel(res.U[-1], c, sys) < 1e-15


def test_iterate_k_exact_for_first_k_slices_and_at_k_equals_N():
    """Theorem 4.3: U^{n,(k)} equals the sequential fine solution for n <= k, and k = N is exact."""
    prob = _bump_problem()
    sys = solver.ModalSystem(prob)
    fine = solver.sequential_fine(sys)
    res = solver.parareal(sys, tol=0.0, k_max=prob.N)
    for k, U in enumerate(res.history):
        for n in range(min(k, prob.N) + 1):
            assert _rel(U[n], fine[n], sys) < 1e-13
    for n in range(prob.N + 1):
        assert _rel(res.U[n], fine[n], sys) < 1e-13


def test_one_iteration_reaches_fine_solution():
    """G and F share the exact homogeneous propagator, so F - G is affine-free and k = 1 suffices."""
    prob = _bump_problem()
    sys = solver.ModalSystem(prob)
    fine = solver.sequential_fine(sys)
    res = solver.parareal(sys, tol=0.0, k_max=2)
    for n in range(prob.N + 1):
        assert _rel(res.history[1][n], fine[n], sys) < 1e-13
    assert res.residuals[0] > 1e-6          # the coarse solution is visibly worse
    assert res.residuals[1] < 1e-13         # the second iteration only confirms


def test_stopping_rule_config1():
    prob = I.config1()
    sys = solver.ModalSystem(prob)
    res = solver.parareal(sys, tol=prob.tol)
    assert res.k == 2 and res.residuals[-1] <= prob.tol
    fine = solver.sequential_fine(sys)
    assert _rel(res.U[-1], fine[-1], sys) < 1e-14


def test_stepper_against_exact_scalar_solution():
    """For f = a e^{r t} on one mode the EIFE step with s nodes has error O(tau^{s+1}) per step.

    The exact mode solution is e^{-lam tau} c + a (e^{r(t+tau)} - e^{-lam tau} e^{r t})/(lam + r).
    """
    lam, a, r = np.array([3.0]), 1.7, -0.6
    for s in (2, 3, 4):
        errs = []
        for tau in (0.2, 0.1, 0.05):
            st = solver.Stepper(lam, tau, I.uniform_nodes(s))
            c = st.step(np.array([0.4]), 0.3, lambda t: a * math.exp(r * t) * np.ones(1))
            ex = math.exp(-lam[0] * tau) * 0.4 + a * (math.exp(r * (0.3 + tau)) - math.exp(-lam[0] * tau) * math.exp(r * 0.3)) / (lam[0] + r)
            errs.append(abs(c[0] - ex))
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert min(rates) > s + 1 - 0.3


@pytest.mark.parametrize("q", [2, 3, 4])
def test_temporal_order_theorem_3_1(q):
    """||u_h(T) - u_h^N|| = O(dt^q) against a far-finer EIFE reference (Theorem 3.1)."""
    rng = I.SplitMix64(31)
    box = ((0.0, 1.0),)
    u0, f, _ = I.sin_mode(1, box, 0.5)
    bumps = I.gaussian_bumps(rng, 1, 3, omega=(1.0, 4.0), width=(0.1, 0.2))
    prob = I.Problem(1, (63,), box, 0.5, 0.0, 1.0, 1, 1, I.uniform_nodes(q), I.uniform_nodes(q), u0, f + bumps, 3)
    sys = solver.ModalSystem(prob)
    ref = solver.sequential_eife(sys, 512, I.uniform_nodes(4))
    errs = [sys.norm(solver.sequential_eife(sys, nt, prob.fine_nodes) - ref) for nt in (4, 8, 16)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > q - 0.35


@pytest.mark.parametrize("d", [1, 2])
def test_spatial_order_lemma_3_1(d):
    """Manufactured u = e^{-t} prod sin(pi x): L2 error ratio about 4 per halving of h (Lemma 3.1)."""
    box = ((0.0, 1.0),) * d
    errs = []
    for nx in (8, 16, 32):
        u0, f, ex = I.sin_mode(d, box, 0.3)
        prob = I.Problem(d, (nx - 1,) * d, box, 0.3, 0.0, 0.5, 2, 32, I.uniform_nodes(4), I.uniform_nodes(2),
                         u0, f, 3, 0.0, ex)
        sys = solver.ModalSystem(prob)
        c = solver.sequential_eife(sys, 64, prob.fine_nodes)
        errs.append(quadrature.l2_error_full(sys.to_nodal(c), ex, 0.5, prob.n, box, 5))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.7 < r < 4.3 for r in ratios)


def test_semigroup_contraction():
    """0 < e^{-lam dt} <= 1 for every mode (Lemma 4.1: the discrete semigroup is bounded by 1)."""
    sys = solver.ModalSystem(I.scaled(I.config3(), (7, 6, 5)))
    st = solver.Stepper(sys.lam, 1e-3, I.uniform_nodes(4))
    assert np.all(st.E > 0) and np.all(st.E <= 1)


def test_mode_subset_equals_full_run():
    prob = _bump_problem()
    full = solver.ModalSystem(prob)
    idx = np.array([0, 5, 17, 100, prob.ndof - 1])
    sub = solver.ModalSystem(prob, modes=idx)
    a = solver.parareal(full, tol=0.0, k_max=2).U[-1][idx]
    b = solver.parareal(sub, tol=0.0, k_max=2).U[-1]
    np.testing.assert_allclose(b, a, rtol=1e-15, atol=0)


def test_zero_initial_data_is_the_zero_function():
    """No u0 terms means u0 = 0: the oracle's U^0 is the zero vector of the right length, and the
    solve is driven by the source alone (the coarse sweep of a zero state under zero forcing is zero)."""
    import numpy as np

    from oracle import solver as osolver
    from paper_2412_01138_gb300 import inputs as I

    box = ((0.0, 1.0),)
    prob = I.Problem(1, (15,), box, 0.5, 0.0, 1.0, 3, 2, I.uniform_nodes(2), I.uniform_nodes(2), (), (), 3, 1e-12)
    sys_ = osolver.ModalSystem(prob)
    assert isinstance(sys_.c0, np.ndarray) and sys_.c0.shape == (15,) and not sys_.c0.any()
    ref = osolver.parareal(sys_, tol=0.0, k_max=1)
    assert all(not u.any() for u in ref.U)
