"""GPU parity of periodic axes (pe_options.periodic_mask: circulant Q1 matrices, DHT basis).

Float64 bound 1e-12 against the oracle (oracle/fem.py dht_matrix, periodic loads), mixed
1e-6; the general forcing path (per-stage loads and transforms) on periodic axes; the
constant mode of an all-periodic problem (lam = 0) keeps its coefficient.
"""
import math

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


def _problem(n, periodic, N=4, M=6, seed=8, forcing=True):
    d = len(n)
    box = ((0.0, 1.0), (-0.5, 1.0), (0.0, 2.0))[:d]
    u0 = (I.Term(1.0, tuple(I.Factor(I.S_SIN, (2 * math.pi / (box[a][1] - box[a][0]), 0.3 + a)) for a in range(d))),
          I.Term(0.5, tuple(I.Factor(I.S_POLY, (1.0, 0.1, 0.0, 0.0)) for a in range(d))))
    f = ()
    if forcing:
        rng = I.SplitMix64(seed)
        f = I.gaussian_bumps(rng, d, 3) + (I.Term(0.4, tuple(I.Factor(I.S_SIN, (4 * math.pi / (box[a][1] - box[a][0]), 0.1))
                                                            for a in range(d)), I.T_EXP, (-0.5, 0.0)),)
    return I.Problem(d, tuple(n), box, 0.12, 0.0, 1.0, N, M, I.uniform_nodes(4), I.draw_random_nodes(2, seed),
                     u0, f, 3, 1e-12, None, "periodic", (), tuple(periodic))


# n = 128 .. 1024 periodic axes run the DHT through the FFT kernels (contiguous and strided);
# other sizes through the DHT matrix
CASES = [((64,), (True,)), ((37,), (True,)), ((32, 27), (True, False)), ((20, 31), (False, True)),
         ((24, 18), (True, True)), ((8, 9, 10), (True, False, True)), ((256,), (True,)),
         ((128, 40), (True, False)), ((13, 512), (False, True)), ((1024,), (True,))]


@pytest.mark.parametrize("n,periodic", CASES)
def test_periodic_iterates_match_oracle(pe, n, periodic):
    prob = _problem(n, periodic)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    with pe.Solver(prob) as s:
        s.set_problem()
        for n_ in range(prob.N + 1):
            assert _rel(s.modal(n_), ref.history[0][n_], sys_.norm_w) <= 1e-12, ("k=0", n_)
        for k in (1, 2):
            s.iterate()
            for n_ in range(1, prob.N + 1):
                assert _rel(s.modal(n_), ref.history[k][n_], sys_.norm_w) <= 1e-12, (k, n_)
        got = s.solution(prob.N).reshape(prob.n)
    assert _rel(got, sys_.to_nodal(ref.U[-1])) <= 1e-12


@pytest.mark.parametrize("n", [(48, 33), (256, 33)])
def test_periodic_mixed_precision(pe, n):
    prob = _problem(n, (True, False))
    sys_ = osolver.ModalSystem(prob)
    fine = osolver.sequential_fine(sys_)
    with pe.Solver(prob, precision=pe.PE_MIXED) as s:
        s.solve(tol=1e-6)
        for n_ in range(1, prob.N + 1):
            assert _rel(s.modal(n_), fine[n_], sys_.norm_w) <= 1e-6, n_


@pytest.mark.parametrize("nx,precision", [(24, "fp64"), (128, "fp64"), (128, "mixed")])
def test_periodic_general_path_moving_hat(pe, nx, precision):
    box = ((0.0, 1.0), (0.0, 1.0))
    hat = I.Term(2.0, (I.Factor(I.S_MOVING_HAT, (0.5, 0.45, 1.0, 0.1)), I.Factor(I.S_SIN, (math.pi, 0.0))))
    u0 = (I.Term(1.0, (I.Factor(I.S_SIN, (2 * math.pi, 0.2)), I.Factor(I.S_SIN, (math.pi, 0.0)))),)
    prob = I.Problem(2, (nx, 19), box, 0.1, 0.0, 1.0, 3, 4, I.uniform_nodes(3), I.uniform_nodes(2), u0, (hat,),
                     3, 1e-12, None, "periodic_hat", (), (True, False))
    sys_ = osolver.ModalSystem(prob, forcing_route="full")
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    prec, bound = (pe.PE_FP64, 1e-12) if precision == "fp64" else (pe.PE_MIXED, 1e-6)
    with pe.Solver(prob, precision=prec, forcing_path=pe.PE_FORCING_GENERAL) as s:
        s.set_problem()
        for _ in range(2):
            s.iterate()
        for n_ in range(1, prob.N + 1):
            assert _rel(s.modal(n_), ref.U[n_], sys_.norm_w) <= bound, n_


def test_constant_mode_is_kept_when_every_axis_is_periodic(pe):
    prob = _problem((16, 12), (True, True), forcing=False)
    with pe.Solver(prob) as s:
        s.solve(tol=1e-12)
        c0 = [s.modal(n_)[0] for n_ in range(prob.N + 1)]
    assert np.abs(np.array(c0) - c0[0]).max() <= 1e-13 * abs(c0[0])


def test_periodic_rejections(pe):
    prob = _problem((16, 12), (True, False))
    with pe.Solver(prob) as s:
        with pytest.raises(pe.PEError):
            s.set_dirichlet((I.Term(1.0, (I.Factor(I.S_POLY, (1.0, 0.0, 0.0, 0.0)),) * 2),))
