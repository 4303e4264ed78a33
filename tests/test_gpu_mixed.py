"""GPU parity of the mixed-precision form (float32 fine stages) against the float64 oracle.

Bound: relative L2 <= 1e-6 (the precision workload's stated bound before
float64 refinement).
"""
import math

import numpy as np
import pytest

from oracle import solver as osolver
from paper_2412_01138_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


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


@pytest.mark.parametrize("which", ["c3_small", "c2_small", "c5_small"])
def test_mixed_small_all_modes(pe, which):
    if which == "c3_small":
        prob = I.scaled(I.config3(), (15, 13, 17), N=16, M=32)
    elif which == "c2_small":
        prob = I.scaled(I.config2(), (63, 50), N=8, M=64)
    else:
        prob = I.scaled(I.config5(), (63, 63), N=16, M=32)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    with pe.Solver(prob, precision=pe.PE_MIXED) as s:
        info = s.solve(tol=1e-6)
        assert info["k"] == 2
        for n in range(1, prob.N + 1):
            assert _rel(s.modal(n), ref.U[n], sys_.norm_w) <= TOL_MIXED, n


def test_mixed_config3_full_size_sampled(pe):
    """Config 3 at full size (127^3, 64 x 32, RK4, R = 17), sampled modes."""
    prob = I.config3()
    rng = np.random.default_rng(3)
    idx = np.unique(np.concatenate([[0, 1, 127, prob.ndof - 1], rng.integers(0, prob.ndof, 300)]))
    sys_ = osolver.ModalSystem(prob, modes=idx)
    ref = osolver.parareal(sys_, tol=0.0, k_max=1)
    with pe.Solver(prob, precision=pe.PE_MIXED) as s:
        info = s.solve(tol=1e-6)
        assert info["k"] == 2 and info["residual"] <= 1e-6
        for n in (1, prob.N // 2, prob.N):
            assert _rel(s.modal(n)[idx], ref.U[n], sys_.norm_w) <= TOL_MIXED, n


@pytest.mark.parametrize("which", ["c3_small", "c2_small"])
def test_float64_refinement_reaches_float64_parity(pe, which):
    """One float64 iteration from the mixed iterate gives the float64 fine solution (<= 1e-12)."""
    if which == "c3_small":
        prob = I.scaled(I.config3(), (15, 13, 17), N=16, M=32)
    else:
        prob = I.scaled(I.config2(), (63, 50), N=8, M=64)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    with pe.Solver(prob, precision=pe.PE_MIXED) as s:
        s.solve(tol=1e-6)
        mixed = [s.modal(n) for n in range(1, prob.N + 1)]
        before = max(_rel(m, ref.U[n + 1], sys_.norm_w) for n, m in enumerate(mixed))
        r = s.refine()
        after = max(_rel(s.modal(n), ref.U[n], sys_.norm_w) for n in range(1, prob.N + 1))
    assert 1e-12 < before <= TOL_MIXED
    assert after <= 1e-12
    # the refinement's residual measures the change it made, i.e. the mixed iterate's error over
    # every slice (the refined iterate being the float64 one to 1e-12): the same number
    w = sys_.norm_w
    num = sum(float(np.sum(w * (m - ref.U[n + 1]) ** 2)) for n, m in enumerate(mixed))
    den = sum(float(np.sum(w * ref.U[n] ** 2)) for n in range(1, prob.N + 1))
    err_all = math.sqrt(num / den)
    assert abs(r - err_all) <= 1e-3 * err_all, (r, err_all)


def _term_mix(kinds, seed):
    """Separable terms with the given time kinds ('e' exponential, 's' sinusoid), drawn from a
    SplitMix64 stream (frequencies up to 200, several turns per substep)."""
    rng = I.SplitMix64(seed)
    out = []
    for k in kinds:
        facs = (I.Factor(I.S_SIN, (math.pi * (1 + int(4 * rng.uniform())), 0.0)),
                I.Factor(I.S_GAUSS, (rng.uniform(), 0.05 + 0.1 * rng.uniform())))
        amp = 2.0 * rng.uniform() - 1.0
        if k == "e":
            out.append(I.Term(amp, facs, I.T_EXP, (8.0 * rng.uniform() - 6.0, 0.0)))
        else:
            out.append(I.Term(amp, facs, I.T_SIN, (200.0 * rng.uniform(), 2.0 * math.pi * rng.uniform())))
    return tuple(out)


# (time kinds, substeps): K = 1, 2, 3, 26, 64, 50 columns.  Two [M][KC] float blocks of at most
# 48 KB run in the persistent kernel (cp.async double buffer over (tile, slice) items); the last
# two cases (M * KC = 6208 and 13000 floats) take the chunked per-slice kernel.
@pytest.mark.parametrize("kinds,M", [("e", 7), ("s", 9), ("es", 64), ("esse" * 4 + "s", 33), ("s" * 32, 97),
                                     ("ses" * 10, 250)])
def test_mixed_stage_contraction_column_classes(pe, kinds, M):
    box = ((0.0, 1.0), (0.0, 1.0))
    u0, _, _ = I.sin_mode(2, box, 0.05)
    prob = I.Problem(2, (47, 61), box, 0.05, 0.1, 0.6, 5, M, I.draw_random_nodes(5, 77), I.uniform_nodes(2), u0,
                     _term_mix(kinds, len(kinds)), 3, 1e-12)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    with pe.Solver(prob, precision=pe.PE_MIXED) as s:
        s.set_problem()
        for k in range(1, 3):
            s.iterate()
            for n in range(1, prob.N + 1):
                assert _rel(s.modal(n), ref.history[k][n], sys_.norm_w) <= TOL_MIXED, (k, n)
