"""GPU parity of the tensor-core engine of the mixed fine sweep (pe_options.fine_engine = PE_FINE_TC)
against the float64 oracle.

The stage contraction runs on tcgen05 with three-term bfloat16 splits of both operands and six
products accumulated in float32, so the engine keeps the mixed form's bound: relative L2
<= 1e-6 against the oracle on the workloads, and no more than the float32 form's own error on
stress mixes of many high-frequency terms.  Cases span every column padding (K = 1 .. 64:
16, 32 and 64 columns, 32-, 64- and 128-byte swizzled operand rows), substep counts 16 .. 128
(slice groups of 1 .. 16 slices, the last group ragged), mode counts that leave a partial
tile, and the cached forced part.
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


# Stress mixes: with 17 or more random terms the float32 form itself (either engine) ends up
# to about 1.5e-6 from the oracle, so these cases check the engine against the SIMT float32
# form slice by slice (no more than 10% above its error) under a 2e-6 cap; the 1e-6 bound is
# checked on the workloads below.
# (time kinds, substeps, slices): K = 1, 2, 28, 34, 40, 64, 61, 18 columns (paddings 16, 16, 32, 64,
# 64, 64, 64, 32); M = 16 (16 slices per group), 32 (8, or 4 at padding 64), 64 (4), 96 (1 at
# padding 64), 48 (2), 128 (1); N chosen so that the last slice group is partial.
@pytest.mark.parametrize("kinds,M,N", [("e", 16, 21), ("s", 32, 9), ("esses" * 3 + "ss", 64, 7),
                                       ("esse" * 4 + "s" * 5, 96, 5), ("s" * 20, 48, 11),
                                       ("s" * 32, 128, 3), ("s" * 30 + "e", 32, 6), ("s" * 9, 32, 7)])
def test_tc_engine_column_paddings_and_groups(pe, kinds, M, N):
    box = ((0.0, 1.0), (0.0, 1.0))
    u0, _, _ = I.sin_mode(2, box, 0.05)
    prob = I.Problem(2, (47, 61), box, 0.05, 0.1, 0.6, N, M, I.draw_random_nodes(4, 78), I.uniform_nodes(2), u0,
                     _term_mix(kinds, len(kinds) + 3), 3, 1e-12)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    err = {}
    for eng in (pe.PE_FINE_SIMT, pe.PE_FINE_TC):
        with pe.Solver(prob, precision=pe.PE_MIXED, fine_engine=eng) as s:
            s.set_problem()
            e = []
            for k in range(1, 3):
                s.iterate()
                e.append([_rel(s.modal(n), ref.history[k][n], sys_.norm_w) for n in range(1, prob.N + 1)])
        err[eng] = np.array(e)
    tc, simt = err[pe.PE_FINE_TC], err[pe.PE_FINE_SIMT]
    assert tc.max() <= 2e-6, tc.max()
    assert np.all(tc <= 1.1 * simt + 1e-8), (tc, simt)


@pytest.mark.parametrize("which", ["c3_small", "c2_small"])
def test_tc_engine_matches_simt_mixed(pe, which):
    """The two engines of the mixed form agree far inside the mixed bound, and the tensor-core
    iterate meets the oracle's bound at every slice."""
    if which == "c3_small":
        prob = I.scaled(I.config3(), (15, 13, 17), N=16, M=32)
    else:
        prob = I.scaled(I.config2(), (63, 50), N=8, M=64)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    outs = {}
    for eng in (pe.PE_FINE_SIMT, pe.PE_FINE_TC):
        with pe.Solver(prob, precision=pe.PE_MIXED, fine_engine=eng) as s:
            info = s.solve(tol=1e-6)
            outs[eng] = ([s.modal(n) for n in range(prob.N + 1)], info)
    (tc, itc), (simt, isimt) = outs[pe.PE_FINE_TC], outs[pe.PE_FINE_SIMT]
    assert itc["k"] == isimt["k"]
    for n in range(1, prob.N + 1):
        assert _rel(tc[n], ref.U[n], sys_.norm_w) <= TOL_MIXED, n
        assert _rel(tc[n], simt[n], sys_.norm_w) <= 5e-7, n


def test_tc_engine_config2_full_size_sampled(pe):
    """The 255^2 workload (32 x 64, RK4, K = 17) at full size, sampled modes."""
    prob = I.config2()
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, 1, 255, prob.ndof - 1], rng.integers(0, prob.ndof, 400)]))
    sys_ = osolver.ModalSystem(prob, modes=idx)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    with pe.Solver(prob, precision=pe.PE_MIXED, fine_engine=pe.PE_FINE_TC) as s:
        info = s.solve(tol=1e-6)
        assert info["k"] == 2
        for n in (1, prob.N // 2, prob.N):
            assert _rel(s.modal(n)[idx], ref.U[n], sys_.norm_w) <= TOL_MIXED, n


def test_tc_engine_cached_forced_part(pe):
    """cache_forced: the tensor-core sweep from zero, later iterations E^M U + F^M(0)."""
    prob = I.scaled(I.config2(), (63, 50), N=8, M=64)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=3)
    with pe.Solver(prob, precision=pe.PE_MIXED, fine_engine=pe.PE_FINE_TC, cache_forced=True) as s:
        s.set_problem()
        for k in range(1, 4):
            s.iterate()
        for n in range(1, prob.N + 1):
            assert _rel(s.modal(n), ref.history[3][n], sys_.norm_w) <= TOL_MIXED, n


def test_tc_engine_rejections(pe):
    prob = I.scaled(I.config2(), (31, 30), N=4, M=64)
    with pytest.raises(pe.PEError) as ei:
        pe.Solver(prob, precision=pe.PE_FP64, fine_engine=pe.PE_FINE_TC)
    assert ei.value.status == pe.PE_EINVAL
    with pytest.raises(pe.PEError) as ei:
        pe.Solver(I.scaled(I.config2(), (31, 30), N=4, M=24), precision=pe.PE_MIXED, fine_engine=pe.PE_FINE_TC)
    assert ei.value.status == pe.PE_EINVAL
    with pytest.raises(pe.PEError) as ei:
        pe.Solver(I.scaled(I.config2(), (31, 30), N=4, M=256), precision=pe.PE_MIXED, fine_engine=pe.PE_FINE_TC)
    assert ei.value.status == pe.PE_EINVAL
    with pytest.raises(pe.PEError) as ei:
        pe.Solver(prob, precision=pe.PE_MIXED, fine_engine=pe.PE_FINE_TC, forcing_path=pe.PE_FORCING_GENERAL)
    assert ei.value.status == pe.PE_EINVAL


def _builder(module):
    import importlib.util
    import os

    spec = importlib.util.spec_from_file_location(module, os.path.join(os.path.dirname(__file__), module + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod._problem


@pytest.mark.parametrize("which", ["periodic", "dirichlet", "c3_small"])
def test_tc_engine_other_separable_problems(pe, which):
    """Periodic axes (DHT), non-homogeneous Dirichlet data (lifted forcing terms) and a 3D grid
    through the tensor-core engine: the converged iterate against the oracle's sequential fine
    solution (the Parareal fixed point), bound 1e-6."""
    if which == "periodic":
        prob = _builder("test_gpu_periodic")((128, 27), (True, False), N=4, M=16)
    elif which == "dirichlet":
        prob = _builder("test_gpu_dirichlet")(2, (23, 30), N=4, M=16)
    else:
        prob = I.scaled(I.config3(), (15, 13, 17), N=8, M=32)
    sys_ = osolver.ModalSystem(prob)
    fine = osolver.sequential_fine(sys_)
    with pe.Solver(prob, precision=pe.PE_MIXED, fine_engine=pe.PE_FINE_TC) as s:
        s.solve(tol=1e-6)
        for n in range(1, prob.N + 1):
            assert _rel(s.modal(n), fine[n], sys_.norm_w) <= TOL_MIXED, n
