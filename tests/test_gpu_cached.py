"""GPU tests of the cached forced part (pe_options.cache_forced).

The fine propagator is affine in its start value, F^M(v) = exp(-lam M dt) v + F^M(0),
so keeping F^M(0) of every slice after the first sweep changes no iterate beyond
rounding: float64 iterates match the oracle to 1e-12, mixed ones match the uncached
mixed run exactly, and only one fine sweep runs per problem and precision.
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


def _prob():
    return I.scaled(I.config2(), (37, 45), N=6, M=9)


def test_cached_float64_iterates_match_oracle(pe):
    prob = _prob()
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=3)
    with pe.Solver(prob, cache_forced=True) as s:
        s.set_problem()
        for k in range(1, 4):
            s.iterate()
            for n in range(1, prob.N + 1):
                assert _rel(s.modal(n), ref.history[k][n], sys_.norm_w) <= 1e-12, (k, n)
        info = s.solve(tol=1e-10)
        assert info["k"] == 2 and info["fine_sweeps"] == 1


def test_cached_mixed_equals_uncached_and_refines(pe):
    prob = _prob()
    sys_ = osolver.ModalSystem(prob)
    fine = osolver.sequential_fine(sys_)
    with pe.Solver(prob, precision=pe.PE_MIXED) as a, pe.Solver(prob, precision=pe.PE_MIXED, cache_forced=True) as b:
        ia, ib = a.solve(tol=1e-6), b.solve(tol=1e-6)
        assert ia["k"] == ib["k"] == 2 and ia["fine_sweeps"] == 2 and ib["fine_sweeps"] == 1
        for n in range(prob.N + 1):
            np.testing.assert_array_equal(a.modal(n), b.modal(n))
        b.refine()  # float64 sweep: makes its own float64 forced parts
        for n in range(1, prob.N + 1):
            assert _rel(b.modal(n), fine[n], sys_.norm_w) <= 1e-12, n


def test_cached_general_path_rejected(pe):
    prob = I.example4(32, 0.01, 1.0)
    with pytest.raises(pe.PEError):
        pe.Solver(prob, forcing_path=pe.PE_FORCING_GENERAL, cache_forced=True)
