"""The oracle reproduces the L2 errors the paper prints (Tables 3-1, 4-1 and the 3D table).

These pins fix, all at once, the reading of the paper's "uniformly selected"
nodes (c_i = (i-1)/s), of P_h as the true L2 projection with consistent
loads, of the error as the continuous L2 norm, and the phi/b weights, the
EIFE step Eq. (1-7), the DST-I eigenpairs and Algorithm 1: a dropped term,
a wrong sign or index anywhere in that chain moves these numbers by far more
than the tolerances used.
"""
import math
import os

import numpy as np
import pytest

from oracle import fem, quadrature, solver
from paper_2412_01138_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def _solve_modal(sys, prob, method):
    """EIFE rows: sequential with N steps; PEIFE rows: Algorithm 1, k = 4."""
    if method.startswith("PEIFE"):
        return solver.parareal(sys, tol=0.0, k_max=4, keep_history=False).U[-1]
    return solver.sequential_eife(sys, prob.N * prob.M, prob.fine_nodes)


def _single_mode_error(prob, method):
    """Error of a problem whose data are the first DST-I mode on every axis.

    The solution then stays in mode J* = (1,...,1), and u_h = c * prod_a v_a
    with v_a the hat function with nodal values S_a[:, 0]; the exact solution
    is a rank-one product too, so ||u - u_h||^2 factorises into 1D element
    quadratures (5 Gauss points per element, as for the 1D rows).
    """
    J = np.ravel_multi_index(tuple([0] * prob.d), prob.n)
    sys = solver.ModalSystem(prob, modes=np.array([J]))
    c = float(_solve_modal(sys, prob, method)[0])
    ex = prob.exact[0]
    amp = ex.amp * quadrature.eval_time(ex, prob.t0 + prob.T)
    A = B = C = 1.0
    for a in range(prob.d):
        n = prob.n[a]
        k = np.arange(1, n + 1)
        col = math.sqrt(2.0 / (n + 1)) * np.sin(k * math.pi / (n + 1))
        fac = ex.factors[a]
        aa, bb, cc = quadrature.l2_inner_1d(lambda x, f=fac: quadrature.eval_factor(f, x), col,
                                            prob.box[a][0], prob.box[a][1], 5)
        A, B, C = A * aa, B * bb, C * cc
    return math.sqrt(max(amp * amp * A - 2.0 * amp * c * B + c * c * C, 0.0))


@pytest.mark.parametrize("row", _rows("table_3_1.txt"), ids=lambda r: "-".join(r[:6]))
def test_table_3_1(row):
    method, q, p, N, M, Nx, err = row
    q, p, N, M, Nx, err = int(q), int(p), int(N), int(M), int(Nx), float(err)
    prob = I.example1(Nx, N, M, q, max(p, 1))
    sys = solver.ModalSystem(prob)
    c = _solve_modal(sys, prob, method)
    got = quadrature.l2_error_full(sys.to_nodal(c), prob.exact, prob.t0 + prob.T, prob.n, prob.box, 5)
    if err in (7.3e-3, 1.8e-3):
        # these two rows are printed rounded to 2 significant digits
        assert float(f"{got:.1e}") == err
    else:
        assert got == pytest.approx(err, rel=1.5e-4)


@pytest.mark.parametrize("row", _rows("table_4_1.txt"), ids=lambda r: "-".join(r[:7]))
def test_table_4_1(row):
    method, q, p, N, M, Nx, Ny, err, rtol = row
    prob = I.example2(int(Nx), int(Ny), int(N), int(M), int(q), max(int(p), 1))
    got = _single_mode_error(prob, method)
    assert got == pytest.approx(float(err), rel=float(rtol))


@pytest.mark.parametrize("row", _rows("table_3d.txt"), ids=lambda r: "-".join(r[:6]))
def test_table_3d(row):
    method, q, p, N, M, Nx, err, rtol = row
    prob = I.example3(int(Nx), int(N), int(M), int(q), max(int(p), 1))
    got = _single_mode_error(prob, method)
    assert got == pytest.approx(float(err), rel=float(rtol))


@pytest.mark.parametrize("which", ["ex2", "ex3"])
def test_single_mode_reduction_matches_full_oracle(which):
    """On a small grid the all-mode oracle with element-quadrature error equals the reduction."""
    if which == "ex2":
        prob = I.example2(16, 8, 4, 8, 3, 3)
    else:
        prob = I.example3(8, 4, 8, 3, 3)
    sys = solver.ModalSystem(prob)
    c = solver.sequential_eife(sys, prob.N * prob.M, prob.fine_nodes)
    # every mode but J* stays at roundoff
    cs = np.abs(c.reshape(prob.n))
    top = cs.flat[0]
    cs.flat[0] = 0.0
    assert cs.max() <= 1e-13 * top
    full = quadrature.l2_error_full(sys.to_nodal(c), prob.exact, prob.t0 + prob.T, prob.n, prob.box, 5)
    red = _single_mode_error(prob, "EIFE")
    assert red == pytest.approx(full, rel=1e-6)
