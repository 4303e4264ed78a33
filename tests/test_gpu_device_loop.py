"""GPU: pe_solve with the Parareal loop on the device (pe_options.device_loop = 1).

One CUDA graph whose conditional (while) node repeats the fine sweep and the correction; the
correction kernel's last CTA appends the residual, advances k and decides whether to go on.
The kernels are those of the host-driven loop, so every iterate, k and the residual history
must be bitwise the host loop's, in float64, in the mixed form on both engines, for a solve
that stops by tolerance and one that stops at max_iter; a non-finite source stops the loop and
is reported as PE_ENONFINITE.
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


FORMS = [("fp64", 0, 0), ("mixed_simt", 1, 0), ("mixed_tc", 1, 1)]


@pytest.mark.parametrize("name,prec,engine", FORMS, ids=[f[0] for f in FORMS])
@pytest.mark.parametrize("tol,max_iter", [(1e-6, 0), (0.0, 3)])
def test_device_loop_equals_host_loop(pe, name, prec, engine, tol, max_iter):
    prob = I.scaled(I.config2(), (37, 45), N=6, M=16)
    out = {}
    for dl in (0, 1):
        with pe.Solver(prob, precision=prec, fine_engine=engine, max_iter=max_iter, device_loop=dl) as s:
            for rep in range(2):  # the second solve reuses the graph
                try:
                    info = s.solve(tol=tol)
                except pe.PEError as e:  # tol = 0 stops at max_iter < N: PE_ENOCONV with the result
                    assert e.status == pe.PE_ENOCONV
                    info = e.result
                modal = [s.modal(n) for n in range(prob.N + 1)]
                nodal = s.solution(prob.N)
            out[dl] = (info, modal, nodal)
    (ih, mh, nh), (id_, md, nd) = out[0], out[1]
    assert id_["k"] == ih["k"] and id_["fine_sweeps"] == ih["fine_sweeps"]
    assert id_["history"] == ih["history"] and id_["residual"] == ih["residual"]
    for n in range(prob.N + 1):
        assert np.array_equal(md[n], mh[n]), n
    assert np.array_equal(nd, nh)
    if tol > 0:
        sys_ = osolver.ModalSystem(prob)
        ref = osolver.parareal(sys_, tol=tol)
        assert id_["k"] == ref.k
        bound = 1e-12 if prec == 0 else 1e-6
        assert osolver.rel_l2(md[-1], ref.U[-1], sys_.norm_w) <= bound


def test_device_loop_reports_nonfinite(pe):
    prob = I.scaled(I.config2(), (16, 9), N=3, M=16)
    bad = I.Term(float("nan"), prob.forcing[1].factors, prob.forcing[1].tkind, prob.forcing[1].tp)
    prob = I.Problem(prob.d, prob.n, prob.box, prob.D, prob.t0, prob.T, prob.N, prob.M, prob.fine_nodes,
                     prob.coarse_nodes, prob.u0, prob.forcing[:1] + (bad,), 3, 1e-6)
    with pe.Solver(prob, device_loop=1) as s:
        with pytest.raises(pe.PEError) as ei:
            s.solve(tol=1e-6)
        assert ei.value.status == pe.PE_ENONFINITE
