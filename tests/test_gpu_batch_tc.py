"""GPU parity of the batched solver with its stage contraction on the tensor cores
(pe_options.fine_engine = PE_FINE_TC in pe_setup_batch).

Work items are (problem, slice group, 128-mode tile) of many problems at once, one persistent
launch per column padding (16, 32, 64).  Each problem must match the oracle to the mixed bound
1e-6 (relative L2) and the batched SIMT float32 engine closely; the batch mixes dimensions,
column counts in every padding class, substep counts 16..128 (slice groups of 1..16 slices, the
last one partial) and grids that leave a partial tile.
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


def _tc_batch():
    """Uneven problems with M a multiple of 16: d = 1, 2, 3; K from 1 to 39 (paddings 16, 32, 64)."""
    probs = []
    for i, M in enumerate((16, 32, 48, 64, 96, 128, 32, 16)):
        p = I.config4_problem(3 * i + 1)
        probs.append(I.scaled(p, (9 + 13 * i, 41 - 3 * i), N=3 + i, M=M))
    rng = I.SplitMix64(91)
    box1 = ((0.0, 2.0),)
    u0, f, _ = I.sin_mode(1, box1, 0.4)
    probs.append(I.Problem(1, (300,), box1, 0.4, 0.1, 0.9, 5, 32, I.uniform_nodes(3), I.draw_random_nodes(2, 3),
                           u0, f + I.gaussian_bumps(rng, 1, 19), 3, 1e-12))  # K = 39: padding 64
    box3 = ((0.0, 1.0), (0.0, 0.5), (0.0, 1.5))
    u0, f, _ = I.sin_mode(3, box3, 0.2)
    probs.append(I.Problem(3, (9, 6, 11), box3, 0.2, 0.0, 1.0, 4, 16, I.uniform_nodes(4), I.uniform_nodes(2),
                           u0, f + I.gaussian_bumps(rng, 3, 3), 3, 1e-12))
    probs.append(I.Problem(2, (5, 5), ((0.0, 1.0),) * 2, 1.0, 0.0, 1.0, 1, 16, I.uniform_nodes(2),
                           I.uniform_nodes(1), I.sin_mode(2, ((0.0, 1.0),) * 2, 1.0)[0], (), 3, 1e-12))  # K = 1
    return probs


def test_batch_tc_matches_oracle_and_simt_per_problem(pe):
    probs = _tc_batch()
    out = {}
    for eng in (pe.PE_FINE_SIMT, pe.PE_FINE_TC):
        with pe.BatchSolver(probs, precision=pe.PE_MIXED, fine_engine=eng) as b:
            b.autotune(None)
            info = b.solve(tol=1e-6)
            r, k = b.status()
            out[eng] = ([[b.modal(i, n) for n in range(p.N + 1)] for i, p in enumerate(probs)], k, info,
                        [b.solution(i) for i in range(len(probs))])
    (tc, ktc, itc, ntc), (simt, ksimt, isimt, nsimt) = out[pe.PE_FINE_TC], out[pe.PE_FINE_SIMT]
    assert list(ktc) == list(ksimt)
    assert itc["fine_dof_substeps"] == isimt["fine_dof_substeps"]
    for i, prob in enumerate(probs):
        sys_ = osolver.ModalSystem(prob)
        fine = osolver.sequential_fine(sys_)  # the Parareal fixed point
        for n in range(1, prob.N + 1):
            assert _rel(tc[i][n], fine[n], sys_.norm_w) <= 1e-6, (i, n)
            assert _rel(tc[i][n], simt[i][n], sys_.norm_w) <= 1e-6, (i, n)
        ref_nodal = sys_.to_nodal(fine[-1]).reshape(-1)
        assert np.abs(ntc[i] - ref_nodal).max() <= 1e-6 * np.abs(ref_nodal).max(), i


def test_batch_tc_config4_subset_sampled(pe):
    """The first 24 problems of the 512-problem batched workload (n 31..511, 16-64 slices x 32
    substeps, 4-16 bumps) through the tensor-core engine, sampled modes of every problem."""
    probs = I.config4(count=24)
    with pe.BatchSolver(probs, precision=pe.PE_MIXED, fine_engine=pe.PE_FINE_TC) as b:
        info = b.solve(tol=1e-6)
        r, k = b.status()
        assert info["max_k"] == 2 and float(r.max()) <= 1e-6
        rng = np.random.default_rng(4)
        for i, prob in enumerate(probs):
            idx = np.unique(rng.integers(0, prob.ndof, 64))
            sys_ = osolver.ModalSystem(prob, modes=idx)
            ref = osolver.parareal(sys_, tol=0.0, k_max=2)
            assert _rel(b.modal(i, prob.N)[idx], ref.U[-1], sys_.norm_w) <= 1e-6, i


def test_batch_tc_rejections(pe):
    probs = [I.scaled(I.config4_problem(0), (20, 20), N=4, M=24)]
    with pytest.raises(pe.PEError) as ei:
        pe.BatchSolver(probs, precision=pe.PE_MIXED, fine_engine=pe.PE_FINE_TC)
    assert ei.value.status == pe.PE_EINVAL
    probs = [I.scaled(I.config4_problem(0), (20, 20), N=4, M=32)]
    with pytest.raises(pe.PEError) as ei:
        pe.BatchSolver(probs, precision=pe.PE_FP64, fine_engine=pe.PE_FINE_TC)
    assert ei.value.status == pe.PE_EINVAL
