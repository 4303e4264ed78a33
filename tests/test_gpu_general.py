"""GPU parity of the general forcing path (consistent load + tensor DST-I at every stage time).

The oracle's counterpart assembles the d-D consistent load by direct element
quadrature of f(t, x) at every stage time and transforms it (``forcing_route='full'``).
Float64 bound 1e-12; mixed 1e-6.
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


def _rel(a, b, w):
    return float(np.sqrt(np.sum(w * (a - b) ** 2)) / np.sqrt(np.sum(w * b * b)))


@pytest.mark.parametrize("alpha,freq,q,p", [(0.01, 1.0, 2, 2), (0.01, 10.0, 3, 2), (0.1, 10.0, 3, 3)])
def test_example4_moving_hat(pe, alpha, freq, q, p):
    """Example 4 of Sec. 5 (oscillating hat source), N_x = 128, 4 x 16, k = 4 iterations."""
    prob = I.example4(128, alpha, freq, 4, 16, q, p)
    sys_ = osolver.ModalSystem(prob, forcing_route="full")
    ref = osolver.parareal(sys_, tol=0.0, k_max=4)
    with pe.Solver(prob, forcing_path=pe.PE_FORCING_GENERAL) as s:
        s.set_problem()
        for n in range(prob.N + 1):
            assert _rel(s.modal(n), ref.history[0][n], sys_.norm_w) <= 1e-12
        for _ in range(4):
            s.iterate()
        for n in range(1, prob.N + 1):
            assert _rel(s.modal(n), ref.U[n], sys_.norm_w) <= 1e-12, n
        nodal = s.solution(prob.N)
    ref_nodal = sys_.to_nodal(ref.U[-1]).reshape(-1)
    assert np.abs(nodal - ref_nodal).max() <= 1e-12 * np.abs(ref_nodal).max()


@pytest.mark.parametrize("alpha,freq", [(0.01, 1.0), (0.01, 10.0), (0.1, 1.0), (0.1, 10.0)])
def test_example4_paper_size(pe, alpha, freq):
    """Example 4 at the paper's size: N_x = 1024 (1023 interior nodes), 4 x 16, k = 4 iterations,
    every (alpha, f) pair the paper runs, float64 and mixed."""
    prob = I.example4(1024, alpha, freq, 4, 16, 3, 3)
    sys_ = osolver.ModalSystem(prob, forcing_route="full")
    ref = osolver.parareal(sys_, tol=0.0, k_max=4)
    for prec, bound in ((pe.PE_FP64, 1e-12), (pe.PE_MIXED, 1e-6)):
        with pe.Solver(prob, precision=prec, forcing_path=pe.PE_FORCING_GENERAL) as s:
            s.set_problem()
            for _ in range(4):
                s.iterate()
            for n in range(1, prob.N + 1):
                assert _rel(s.modal(n), ref.U[n], sys_.norm_w) <= bound, (prec, n)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_moving_hat_2d(pe, precision):
    prob = I.moving_hat_2d()
    sys_ = osolver.ModalSystem(prob, forcing_route="full")
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    prec = pe.PE_FP64 if precision == "fp64" else pe.PE_MIXED
    bound = 1e-12 if precision == "fp64" else 1e-6
    with pe.Solver(prob, precision=prec, forcing_path=pe.PE_FORCING_GENERAL) as s:
        info = s.solve(tol=1e-6)
        assert info["k"] == 2
        for n in range(1, prob.N + 1):
            assert _rel(s.modal(n), ref.U[n], sys_.norm_w) <= bound, n


@pytest.mark.parametrize("n", [(63, 50), (31, 17, 9)])
def test_general_equals_separable_on_separable_sources(pe, n):
    base = I.config2() if len(n) == 2 else I.config3()
    prob = I.scaled(base, n, N=6, M=8)
    with pe.Solver(prob) as a:
        a.solve(tol=0.0)
        ua = [a.modal(k) for k in range(prob.N + 1)]
    with pe.Solver(prob, forcing_path=pe.PE_FORCING_GENERAL) as b:
        b.solve(tol=0.0)
        ub = [b.modal(k) for k in range(prob.N + 1)]
    w = np.ones(prob.ndof)
    for k in range(1, prob.N + 1):
        assert _rel(ub[k], ua[k], w) <= 1e-12


def test_general_full_size_config2_mixed(pe):
    """The 2D 255^2 workload through the general path (a DST per stage time), sampled modes."""
    prob = I.config2()
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, prob.ndof - 1], rng.integers(0, prob.ndof, 300)]))
    sys_ = osolver.ModalSystem(prob, modes=idx)
    ref = osolver.parareal(sys_, tol=0.0, k_max=1)
    with pe.Solver(prob, precision=pe.PE_MIXED, forcing_path=pe.PE_FORCING_GENERAL) as s:
        info = s.solve(tol=1e-6)
        assert info["k"] == 2
        for n in (1, prob.N):
            assert _rel(s.modal(n)[idx], ref.U[n], sys_.norm_w) <= 1e-6, n


def test_moving_source_rejected_on_separable_path(pe):
    prob = I.example4(32, 0.01, 1.0)
    with pe.Solver(prob) as s:
        with pytest.raises(pe.PEError) as ei:
            s.set_problem()
        assert ei.value.status == pe.PE_EINVAL
