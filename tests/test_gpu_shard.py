"""GPU: the mode-sharded solve (pe_options.mode_begin / mode_end) against the unsharded one.

Two shards of one problem run in turn in one process on one GPU (two contexts, each owning a
block of axis-0 modes); their residual sums are added on the host after every iteration, as
an all-reduce across GPUs would.  Per mode the shards run the same arithmetic as the
unsharded context (the per-axis tables are the rows of the same whole-axis tables), so their
modal iterates are bitwise those of the unsharded solve; the combined residual equals the
unsharded one up to summation order (1e-15), and so does the sum of the shards' nodal
fields (to float32 rounding in the mixed form, whose output transform runs in float32).  A third test drives pe_solve of one shard with the residual_reduce callback
adding the other shard's recorded sums.
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


def _u0(prob):
    rng = np.random.default_rng(3)
    return rng.standard_normal(prob.ndof)


CASES = [("2d_fp64", (37, 45), 0, 0), ("3d_fp64", (11, 9, 13), 0, 0), ("2d_mixed_tc", (37, 45), 1, 1),
         ("2d_mixed_simt", (37, 45), 1, 0)]


@pytest.mark.parametrize("name,n,prec,engine", CASES, ids=[c[0] for c in CASES])
def test_two_shards_in_turn_match_the_unsharded_solve(pe, name, n, prec, engine):
    from paper_2412_01138_gb300 import shard

    prob = I.scaled(I.config2() if len(n) == 2 else I.config3(), n, N=6, M=16)
    u0 = _u0(prob)
    ranges = shard.shard_ranges(n[0], 2)
    with pe.Solver(prob, precision=prec, fine_engine=engine) as full:
        full.set_problem(pe.PE_FIELD_NODAL, nodal=u0)
        ref_r = [full.iterate() for _ in range(3)]
        ref_modal = [full.modal(k) for k in range(prob.N + 1)]
        ref_nodal = full.solution(prob.N)
    shards = [pe.Solver(prob, precision=prec, fine_engine=engine, mode_range=rg) for rg in ranges]
    try:
        for s in shards:
            s.set_problem(pe.PE_FIELD_NODAL, nodal=u0)
        for k in range(3):
            tot = sum(s.iterate_sums() for s in shards)
            r = shard.relative_residual(tot)
            assert r == pytest.approx(ref_r[k], rel=1e-13, abs=1e-300), (k, r, ref_r[k])
        for sl in range(prob.N + 1):
            got = np.concatenate([s.modal(sl) for s in shards])
            assert np.array_equal(got, ref_modal[sl]), sl
        nodal = sum(s.solution(prob.N) for s in shards)
        # the mixed form transforms its output in float32: the shards' sum then agrees with the
        # whole transform to float32 rounding
        bound = 1e-14 if prec == 0 else 1e-6
        assert np.abs(nodal - ref_nodal).max() <= bound * np.abs(ref_nodal).max()
        # the shard's own tables are rows of the whole tables
        lam_full = osolver.ModalSystem(prob).lam
        inner = prob.ndof // n[0]
        for s, (b, e) in zip(shards, ranges):
            np.testing.assert_allclose(s.lam(), lam_full[b * inner:e * inner], rtol=4e-15)
    finally:
        for s in shards:
            s.close()


def test_solve_with_residual_reduce_callback(pe):
    """pe_solve of shard A stops where the unsharded solve stops when its callback adds the
    residual sums that shard B (run before it) recorded for the same iterations."""
    from paper_2412_01138_gb300 import shard

    prob = I.scaled(I.config2(), (40, 33), N=8, M=16)
    u0 = _u0(prob)
    ranges = shard.shard_ranges(prob.n[0], 2)
    with pe.Solver(prob) as full:
        info_full = full.solve(tol=1e-10, u0_kind=pe.PE_FIELD_NODAL, nodal=u0)
        nodal_full = full.solution(prob.N)
    with pe.Solver(prob, mode_range=ranges[1]) as b:
        b.set_problem(pe.PE_FIELD_NODAL, nodal=u0)
        sums_b = [b.iterate_sums() for _ in range(info_full["k"])]
        nodal_b = b.solution(prob.N)
    calls = []

    def reduce(sums):
        tot = sums + sums_b[len(calls)]
        calls.append(sums.copy())
        return tot

    with pe.Solver(prob, mode_range=ranges[0], residual_reduce=reduce) as a:
        info = a.solve(tol=1e-10, u0_kind=pe.PE_FIELD_NODAL, nodal=u0)
        nodal_a = a.solution(prob.N)
    assert info["k"] == info_full["k"] == len(calls)
    assert info["residual"] == pytest.approx(info_full["residual"], rel=1e-12, abs=1e-300)
    nodal = nodal_a + nodal_b
    assert np.abs(nodal - nodal_full).max() <= 1e-14 * np.abs(nodal_full).max()


def test_sharded_context_rejects_what_it_cannot_do(pe):
    prob = I.scaled(I.config2(), (20, 9), N=3, M=4)
    with pe.Solver(prob, mode_range=(5, 12)) as s:
        with pytest.raises(pe.PEError) as ei:
            s.solve(tol=1e-6)  # no residual_reduce: the shard's own residual is not the solve's
        assert ei.value.status == pe.PE_EINVAL
        with pytest.raises(pe.PEError) as ei:
            s.set_problem(pe.PE_FIELD_TERMS_QUADRATURE)
        assert ei.value.status == pe.PE_EINVAL
    for bad in ((5, 5), (-1, 3), (3, 21)):
        with pytest.raises(pe.PEError) as ei:
            pe.Solver(prob, mode_range=bad)
        assert ei.value.status == pe.PE_EINVAL
