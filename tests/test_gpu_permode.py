"""Element-wise (per-mode) parity, the general path at full size in float64, and the failure
statuses that only a GPU run reaches.

The rel-L2 checks elsewhere weight every mode by mu^M_J (the L2 norm of the FE function);
on problems whose initial data sit in one slow mode that weighted norm is dominated by
that mode.  Here the initial data are zero and the source is a set of narrow Gaussian
bumps, which excite the whole spectrum, and every mode of every slice is compared
separately: max_J |c_gpu,J - c_ora,J| / max_J |c_ora,J| at the form's bound (1e-12
float64, 1e-6 mixed).
"""
import dataclasses

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


def _forcing_only(n, N, M, seed=41):
    """u0 = 0, six narrow bumps (widths 0.01..0.03, frequencies up to 40) on the unit box."""
    d = len(n)
    box = ((0.0, 1.0),) * d
    rng = I.SplitMix64(seed)
    bumps = I.gaussian_bumps(rng, d, 6, omega=(1.0, 40.0), width=(0.01, 0.03))
    return I.Problem(d, tuple(n), box, 0.05, 0.0, 1.0, N, M, I.uniform_nodes(4), I.uniform_nodes(2), (), bumps,
                     3, 1e-12, None, "forcing_only")


def _elem(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


FORMS = [("fp64", 0, 0, 1e-12), ("mixed_simt", 1, 0, 1e-6), ("mixed_tc", 1, 1, 1e-6)]


@pytest.mark.parametrize("n", [(95, 70), (13, 11, 17)])
@pytest.mark.parametrize("form,prec,engine,bound", FORMS, ids=[f[0] for f in FORMS])
def test_every_mode_of_every_slice_matches_oracle(pe, n, form, prec, engine, bound):
    prob = _forcing_only(n, N=6, M=16)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    # the whole spectrum is excited: the high half of the modes is far from zero
    hi = np.abs(ref.U[-1]).reshape(n)[tuple(slice(v // 2, None) for v in n)].max()
    assert hi > 1e-6 * np.abs(ref.U[-1]).max()
    with pe.Solver(prob, precision=prec, fine_engine=engine) as s:
        s.set_problem()
        for k in range(0, 3):
            if k > 0:
                s.iterate()
            for slice_ in range(1, prob.N + 1):
                got, want = s.modal(slice_), ref.history[k][slice_]
                err = _elem(got, want)
                assert err <= bound, (form, k, slice_, err)
                if prec == 0:
                    # float64: every mode above 1e-3 of the largest also to 1e-10 of its own size
                    big = np.abs(want) > 1e-3 * np.abs(want).max()
                    rel = np.abs(got[big] - want[big]) / np.abs(want[big])
                    assert rel.max() <= 1e-10, (k, slice_, float(rel.max()))


def test_general_path_full_size_float64_sampled_modes(pe):
    """The 255^2 workload through the general forcing path (a consistent load assembled by
    element quadrature and a DST-I at every one of the 32 x 64 x 4 stage times) in float64,
    against the oracle on 400 sampled modes.  The workload's source is separable, and for a
    separable source the oracle's full element quadrature equals its per-axis route term by
    term (pinned in tests/test_oracle_quadrature.py), so the oracle's mode-subset run (the
    per-axis route) is the reference."""
    prob = I.config2()
    rng = np.random.default_rng(9)
    idx = np.unique(np.concatenate([[0, 1, 254, 255, prob.ndof - 1], rng.integers(0, prob.ndof, 400)]))
    sys_ = osolver.ModalSystem(prob, modes=idx)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    with pe.Solver(prob, precision=pe.PE_FP64, forcing_path=pe.PE_FORCING_GENERAL) as s:
        info = s.solve(tol=1e-6)
        assert info["k"] == 2
        for n in (1, prob.N // 2, prob.N):
            got = s.modal(n)[idx]
            rel = float(np.sqrt(np.sum(sys_.norm_w * (got - ref.U[n]) ** 2)) /
                        np.sqrt(np.sum(sys_.norm_w * ref.U[n] ** 2)))
            assert rel <= 1e-12, (n, rel)
            assert _elem(got, ref.U[n]) <= 1e-12, n


def test_no_convergence_is_reported_with_the_last_residual(pe):
    """max_iter = 1 < N and tol = 1e-14 on the 1D workload: one iteration cannot reach the
    tolerance (the first residual is the coarse-to-fine change), so pe_solve returns
    PE_ENOCONV after filling in k = 1 and that residual, which equals the oracle's r_1."""
    prob = I.config1()
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=1)
    with pe.Solver(prob, max_iter=1) as s:
        with pytest.raises(pe.PEError) as ei:
            s.solve(tol=1e-14)
    assert ei.value.status == pe.PE_ENOCONV
    res = ei.value.result
    assert res is not None and res["k"] == 1 and res["fine_sweeps"] == 1
    assert res["residual"] > 1e-14
    assert res["residual"] == pytest.approx(ref.residuals[0], rel=1e-9)


def test_expired_device_wait_is_reported_as_timeout(pe):
    """The bounded mbarrier wait of the tensor-core kernels, on a barrier nothing arrives at
    (a one-warp kernel, no MMA or copy in flight, about a millisecond of budget): the kernel
    records the expiry and returns, the call reports PE_ETIMEOUT, and the GPU stays usable."""
    import torch

    for _ in range(2):
        with pytest.raises(pe.PEError) as ei:
            pe.probe_wait_timeout(2_000_000)
        assert ei.value.status == pe.PE_ETIMEOUT
    x = torch.arange(64, dtype=torch.float64, device="cuda")
    assert float(x.sum()) == 2016.0


def test_checkpoint_of_a_transposed_grid_is_rejected(pe):
    """A state saved on a 15 x 17 grid must not load into a 17 x 15 context (same Ndof,
    other mode layout), nor into one with another D."""
    base = _forcing_only((15, 17), N=3, M=4)
    with pe.Solver(base) as s:
        s.set_problem()
        s.iterate()
        blob = s.save_state()
    for other in (I.scaled(base, (17, 15)), dataclasses.replace(base, D=0.06)):
        with pe.Solver(other) as s2:
            s2.set_problem()
            with pytest.raises(pe.PEError) as ei:
                s2.load_state(blob)
            assert ei.value.status == pe.PE_EINVAL
    with pe.Solver(base) as s3:  # the same problem still loads
        s3.set_problem()
        s3.load_state(blob)


@pytest.mark.parametrize("dl", [0, 1], ids=["host_loop", "device_loop"])
def test_no_convergence_is_reported_by_the_wait_of_an_asynchronous_solve(pe, dl):
    """The same stop through pe_solve_async / pe_solve_wait, with the loop on the host and on
    the device: the wait returns PE_ENOCONV with k = 1 and the oracle's r_1, and the context
    takes the next solve."""
    prob = I.config1()
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=1)
    with pe.Solver(prob, max_iter=1, device_loop=dl) as s:
        for _ in range(2):
            s.solve_async(tol=1e-14)
            with pytest.raises(pe.PEError) as ei:
                s.wait()
            assert ei.value.status == pe.PE_ENOCONV
            res = ei.value.result
            assert res is not None and res["k"] == 1 and res["history"] == [res["residual"]]
            assert res["residual"] == pytest.approx(ref.residuals[0], rel=1e-9)
