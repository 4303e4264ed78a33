"""GPU: repeated solves of one problem with the set-up and output phases replayed as CUDA graphs
(pe_options.device_loop = 2).

The first solve of a problem runs every phase directly, the second captures the set-up phase
(forward transform of u0, forcing factors, stage weights, coarse sweep) and the output phase
(inverse transform, lifting) into graphs, and later solves replay them around the device-side
loop.  The graphs hold the same kernels with the same arguments, so every solve must be
bitwise the host-driven solve's: k, the residual history, every modal iterate and the nodal
output; nodal u0 held in device memory is read anew by each replay (its values change between
solves here); a pe_set_problem or pe_set_dirichlet call in between drops the graphs.
"""
import numpy as np
import pytest

from oracle import solver as osolver
from paper_2412_01138_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_01138_gb300 import pe as _pe

    _pe.lib()
    return _pe, torch


def _snapshot(s, prob, info):
    return (info["k"], info["history"], info["residual"], [s.modal(n) for n in range(prob.N + 1)],
            s.solution(prob.N))


def _same(a, b):
    assert a[0] == b[0] and a[1] == b[1] and a[2] == b[2]
    for n, (x, y) in enumerate(zip(a[3], b[3])):
        assert np.array_equal(x, y), n
    assert np.array_equal(a[4], b[4])


FORMS = [("fp64", 0, 0), ("mixed_simt", 1, 0), ("mixed_tc", 1, 1)]
# 37 x 45 keeps the set-up on one stream; 71 x 65 (>= 4096 nodes) forks the u0 transform and
# the time tables onto the side stream, so the captured graph has a fork and a join
GRIDS = [(37, 45), (71, 65)]


@pytest.mark.parametrize("n", GRIDS, ids=["one_stream", "forked"])
@pytest.mark.parametrize("name,prec,engine", FORMS, ids=[f[0] for f in FORMS])
def test_replayed_solves_equal_direct_solves(env, name, prec, engine, n):
    pe, _ = env
    prob = I.scaled(I.config2(), n, N=6, M=16)
    runs = {}
    for dl in (0, 1, 2):
        with pe.Solver(prob, precision=prec, fine_engine=engine, device_loop=dl) as s:
            runs[dl] = []
            for _ in range(4):  # direct, capture, replay, replay
                info = s.solve(tol=1e-6)
                runs[dl].append((_snapshot(s, prob, info), info))
    for rep in range(4):
        _same(runs[2][rep][0], runs[0][rep][0])
        i1, i2 = runs[1][rep][1], runs[2][rep][1]
        assert i2["kernel_launches"] == i1["kernel_launches"], rep
        # the timing events inside the captured set-up are graph nodes: replays record them
        assert i2["ms_coarse_kernel"] > 0.0 and i2["ms_tables"] > 0.0, rep
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=1e-6)
    assert runs[2][3][0][0] == ref.k
    bound = 1e-12 if prec == 0 else 1e-6
    assert osolver.rel_l2(runs[2][3][0][3][-1], ref.U[-1], sys_.norm_w) <= bound


@pytest.mark.parametrize("n", GRIDS, ids=["one_stream", "forked"])
def test_device_u0_is_read_anew_by_each_replay(env, n):
    pe, torch = env
    prob = I.scaled(I.config2(), n, N=5, M=16)
    rng = np.random.default_rng(11)
    u0s = [rng.standard_normal(prob.ndof) for _ in range(4)]
    direct = []
    with pe.Solver(prob, device_loop=0) as s:
        for u in u0s:
            info = s.solve(tol=1e-8, u0_kind=pe.PE_FIELD_NODAL, nodal=u)
            direct.append(_snapshot(s, prob, info))
    buf = torch.empty(prob.ndof, dtype=torch.float64, device="cuda")
    with pe.Solver(prob, device_loop=2) as s:
        for rep, u in enumerate(u0s):
            buf.copy_(torch.from_numpy(u))  # same device pointer, new values
            torch.cuda.synchronize()
            info = s.solve(tol=1e-8, u0_kind=pe.PE_FIELD_NODAL, nodal=buf)
            _same(_snapshot(s, prob, info), direct[rep])
        # nodal u0 in host memory is not captured: the phases run directly, same result
        info = s.solve(tol=1e-8, u0_kind=pe.PE_FIELD_NODAL, nodal=u0s[0])
        _same(_snapshot(s, prob, info), direct[0])


def _dirichlet_problem():
    d, box = 2, ((0.0, 1.0), (0.0, 1.5))
    u0, f, _ = I.sin_mode(d, box, 0.15)
    g = I.Term(0.8, tuple(I.Factor(I.S_POLY, (1.0 + 0.3 * a, 0.5 - a, 0.2, 0.0)) for a in range(d)), I.T_EXP,
               (-0.7, 0.0))
    return I.Problem(d, (23, 30), box, 0.15, 0.1, 1.0, 4, 16, I.uniform_nodes(4), I.draw_random_nodes(2, 5),
                     u0, f + I.gaussian_bumps(I.SplitMix64(5), d, 3), 3, 1e-12, None, "dirichlet", (g,))


def test_dirichlet_lifting_and_dropped_graphs(env):
    """Both phases carry the lifting; pe_set_dirichlet and pe_set_problem in between drop the
    graphs, and the solves after them are again the direct ones."""
    pe, _ = env
    prob = _dirichlet_problem()
    out = {}
    for dl in (0, 2):
        with pe.Solver(prob, device_loop=dl) as s:
            seq = [_snapshot(s, prob, s.solve(tol=1e-10)) for _ in range(3)]
            s.set_dirichlet(())  # homogeneous data from here on
            seq += [_snapshot(s, prob, s.solve(tol=1e-10)) for _ in range(3)]
            s.set_problem()
            seq += [_snapshot(s, prob, s.solve(tol=1e-10)) for _ in range(2)]
            out[dl] = seq
    assert not np.array_equal(out[0][0][4], out[0][3][4])  # the data did change the solution
    for a, b in zip(out[2], out[0]):
        _same(a, b)


def test_device_loop_value_is_checked(env):
    pe, _ = env
    prob = I.scaled(I.config2(), (9, 8), N=3, M=4)
    for bad in (-1, 3):
        with pytest.raises(pe.PEError) as ei:
            pe.Solver(prob, device_loop=bad)
        assert ei.value.status == pe.PE_EINVAL


@pytest.mark.parametrize("dl", [0, 2], ids=["host_loop", "replayed"])
def test_solve_out_writes_the_solution(env, dl):
    """pe_solve_out: the nodal solution written by the solve itself (host array or device
    tensor) equals pe_get_solution's, on every solve of a replayed problem as well."""
    pe, torch = env
    prob = I.scaled(I.config2(), (71, 65), N=5, M=16)
    u0 = np.random.default_rng(3).standard_normal(prob.ndof)
    buf = torch.from_numpy(u0).cuda()
    with pe.Solver(prob, precision=pe.PE_MIXED, fine_engine=pe.PE_FINE_TC, device_loop=dl) as s:
        for rep in range(3):
            host = np.full(prob.ndof, np.nan)
            dev = torch.full((prob.ndof,), float("nan"), dtype=torch.float64, device="cuda")
            s.solve(tol=1e-6, u0_kind=pe.PE_FIELD_NODAL, nodal=buf, out=host)
            ref = s.solution(prob.N)
            assert np.array_equal(host, ref), rep
            s.solve(tol=1e-6, u0_kind=pe.PE_FIELD_NODAL, nodal=buf, out=dev)
            assert np.array_equal(dev.cpu().numpy(), ref), rep
        with pytest.raises(ValueError):
            s.solve(tol=1e-6, u0_kind=pe.PE_FIELD_NODAL, nodal=buf, out=np.empty(prob.ndof, dtype=np.float32))
        with pytest.raises(ValueError):
            s.solve(tol=1e-6, u0_kind=pe.PE_FIELD_NODAL, nodal=buf, out=np.empty(prob.ndof - 1))


@pytest.mark.parametrize("dl", [0, 1, 2], ids=["host_loop", "device_loop", "replayed"])
def test_async_solve_equals_solve(env, dl):
    """pe_solve_async + pe_solve_wait report and produce what pe_solve does (k, residual history,
    iterates, the nodal output written into the caller's buffer); one solve may be pending."""
    pe, torch = env
    prob = I.scaled(I.config2(), (71, 65), N=6, M=16)
    buf = torch.from_numpy(np.random.default_rng(5).standard_normal(prob.ndof)).cuda()
    kw = dict(precision=pe.PE_MIXED, fine_engine=pe.PE_FINE_TC, device_loop=dl)
    with pe.Solver(prob, **kw) as s:
        ref = [_snapshot(s, prob, s.solve(tol=1e-6, u0_kind=pe.PE_FIELD_NODAL, nodal=buf)) for _ in range(3)]
    with pe.Solver(prob, **kw) as s:
        for rep in range(3):
            out = torch.full((prob.ndof,), float("nan"), dtype=torch.float64, device="cuda")
            s.solve_async(tol=1e-6, u0_kind=pe.PE_FIELD_NODAL, nodal=buf, out=out)
            if rep == 0:
                for call in (lambda: s.solve_async(tol=1e-6, u0_kind=pe.PE_FIELD_NODAL, nodal=buf),
                             lambda: s.modal(0), lambda: s.solution(prob.N), lambda: s.iterate()):
                    with pytest.raises(pe.PEError) as ei:
                        call()
                    assert ei.value.status == pe.PE_ESTATE
            info = s.wait()
            got = _snapshot(s, prob, info)
            _same(got, ref[rep])
            assert np.array_equal(out.cpu().numpy(), ref[rep][4]), rep
        with pytest.raises(pe.PEError) as ei:
            s.wait()
        assert ei.value.status == pe.PE_ESTATE
