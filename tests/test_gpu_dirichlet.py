"""GPU parity of non-homogeneous Dirichlet data (pe_set_dirichlet, the lifting w = u_h - I_h g).

The library forms the lifting's extra load from per-axis stencils of the data's factors
and the tensor DST-I; the oracle assembles the full-grid mass and stiffness rows as
Kronecker products and applies them to the nodal lifting (oracle/dirichlet.py).  Float64
bound 1e-12 (modal w and nodal u_h at every slice), mixed 1e-6.
"""

import numpy as np
import pytest

from oracle import solver as osolver
from paper_2412_01138_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_01138_gb300 import pe as _pe

    _pe.lib()
    return _pe


def _rel(a, b, w=None):
    w = np.ones_like(b) if w is None else w
    return float(np.sqrt(np.sum(w * (a - b) ** 2)) / np.sqrt(np.sum(w * b * b)))


def _poly(c0, c1, c2=0.0):
    return I.Factor(I.S_POLY, (c0, c1, c2, 0.0))


def _problem(d, n, N=4, M=6, seed=5):
    box = ((0.0, 1.0), (0.0, 1.5), (0.0, 0.8))[:d]
    D = 0.15
    u0, f, _ = I.sin_mode(d, box, D)
    rng = I.SplitMix64(seed)
    bumps = I.gaussian_bumps(rng, d, 3)
    g1 = I.Term(0.8, tuple(_poly(1.0 + 0.3 * a, 0.5 - a, 0.2) for a in range(d)), I.T_EXP, (-0.7, 0.0))
    g2 = I.Term(-0.4, tuple(I.Factor(I.S_SIN, (1.7 + a, 0.3)) for a in range(d)), I.T_SIN, (4.0, 0.6))
    g3 = I.Term(0.25, tuple(I.Factor(I.S_GAUSS, (0.3, 0.4)) if a == 0 else _poly(1.0, 0.0) for a in range(d)),
                I.T_EXP, (0.0, 0.0))
    return I.Problem(d, tuple(n), box, D, 0.1, 1.0, N, M, I.uniform_nodes(4), I.draw_random_nodes(2, seed),
                     u0, f + bumps, 3, 1e-12, None, "dirichlet", (g1, g2, g3))


@pytest.mark.parametrize("d,n", [(1, (200,)), (2, (23, 30)), (3, (9, 12, 7))])
def test_dirichlet_iterates_match_oracle(pe, d, n):
    prob = _problem(d, n)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    dT = prob.T / prob.N
    with pe.Solver(prob) as s:
        s.set_problem()
        for n_ in range(prob.N + 1):
            assert _rel(s.modal(n_), ref.history[0][n_], sys_.norm_w) <= 1e-12, ("k=0", n_)
        for k in (1, 2):
            s.iterate()
            for n_ in range(1, prob.N + 1):
                assert _rel(s.modal(n_), ref.history[k][n_], sys_.norm_w) <= 1e-12, (k, n_)
        for n_ in range(prob.N + 1):
            got = s.solution(n_).reshape(prob.n)
            want = sys_.solution_nodal(ref.U[n_], prob.t0 + n_ * dT)
            assert _rel(got, want) <= 1e-12, n_


def test_dirichlet_mixed_and_nodal_initial_data(pe):
    prob = _problem(2, (31, 26))
    sys_ = osolver.ModalSystem(prob)
    fine = osolver.sequential_fine(sys_)
    want = sys_.solution_nodal(fine[-1], prob.t0 + prob.T)
    with pe.Solver(prob, precision=pe.PE_MIXED) as s:
        s.solve(tol=1e-6)
        assert _rel(s.solution(prob.N).reshape(prob.n), want) <= 1e-6
    # nodal initial data: the interior values of u_h(t0) = P_h(u0 - I_h g) + I_h g
    u0_nodal = sys_.solution_nodal(sys_.c0, prob.t0).reshape(-1).copy()
    with pe.Solver(prob) as s:
        s.solve(tol=1e-12, u0_kind=pe.PE_FIELD_NODAL, nodal=u0_nodal)
        assert _rel(s.solution(prob.N).reshape(prob.n), want) <= 1e-12


def test_harmonic_data_stays(pe):
    facs = (_poly(1.0, 2.0), _poly(3.0, -1.0))
    g = (I.Term(1.3, facs, I.T_EXP, (0.0, 0.0)),)
    prob = I.Problem(2, (40, 33), ((0.0, 1.0), (0.0, 1.0)), 0.3, 0.0, 1.0, 4, 8, I.uniform_nodes(3),
                     I.uniform_nodes(2), (I.Term(1.3, facs),), (), 3, 1e-12, None, "harmonic", g)
    x = np.linspace(0.0, 1.0, 42)[1:-1]
    y = np.linspace(0.0, 1.0, 35)[1:-1]
    want = 1.3 * np.multiply.outer(1.0 + 2.0 * x, 3.0 - y)
    with pe.Solver(prob) as s:
        s.solve(tol=1e-12)
        for n_ in range(prob.N + 1):
            assert np.abs(s.solution(n_).reshape(prob.n) - want).max() <= 1e-12 * np.abs(want).max()


def test_dirichlet_rejections(pe):
    prob = _problem(2, (9, 9))
    with pytest.raises(pe.PEError):
        pe.Solver(prob, forcing_path=pe.PE_FORCING_GENERAL)
    many = tuple(prob.boundary) * 4  # 12 data terms x 3 = 36 forcing terms > 32
    with pe.Solver(prob) as s:
        s.set_dirichlet(many)
        with pytest.raises(pe.PEError):
            s.set_problem()
    # the data can be cleared again
    with pe.Solver(prob) as s:
        s.set_dirichlet(())
        s.solve(tol=1e-10)
