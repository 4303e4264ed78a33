"""GPU parity: every hot-path step of libpe against the CPU oracle, through the C-ABI.

Tolerance: relative L2 (in the L2 norm of the FE function, i.e. weighted by
mu^M_J in mode space) <= 1e-12 on the float64 path; the mixed-precision path
is checked in test_gpu_mixed.py.  Sizes span several 256-mode tiles with a
ragged tail; full-size workloads are checked on sampled modes, which the
oracle computes exactly because modes are independent.
"""
import math

import numpy as np
import pytest

from oracle import fem, quadrature
from oracle import solver as osolver
from paper_2412_01138_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def _bump_problem(n, N, M, seed=11, q=4, p=2, random_coarse=True, R=6, D=0.07, box=None):
    d = len(n)
    box = box or ((0.0, 1.0),) * d
    rng = I.SplitMix64(seed)
    u0, f, _ = I.sin_mode(d, box, D)
    bumps = I.gaussian_bumps(rng, d, R - 1)
    coarse = I.draw_random_nodes(p, seed) if random_coarse else I.uniform_nodes(p)
    return I.Problem(d, tuple(n), box, D, 0.0, 1.0, N, M, I.uniform_nodes(q), coarse, u0, f + bumps, 3, 1e-12)


# ---------------------------------------------------------------------------
# a7: tensor DST-I
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [(1,), (63,), (300,), (1023,), (17, 29), (64, 65), (255, 255), (511, 3), (5, 7, 9),
                               (31, 1, 33), (127, 15, 31)])
def test_dst_matches_oracle(pe, n):
    import torch

    rng = np.random.default_rng(sum(n))
    x = rng.standard_normal(n)
    ref = x
    for a in range(len(n)):
        ref = fem.apply_axis(fem.dst1_matrix(n[a]), ref, a)
    xd = torch.tensor(x.reshape(-1), device="cuda", dtype=torch.float64)
    out = torch.empty_like(xd)
    pe.dst(len(n), n, xd, out)
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy(), ref.reshape(-1)) <= 1e-14 * max(n)
    # in place, and the involution S^2 = I
    pe.dst(len(n), n, out, out)
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy(), x.reshape(-1)) <= 1e-14 * max(n)
    # float32 transform
    xf = xd.float()
    of = torch.empty_like(xf)
    pe.dst(len(n), n, xf, of, f32=True)
    torch.cuda.synchronize()
    assert _rel(of.double().cpu().numpy(), ref.reshape(-1)) <= 2e-6


# ---------------------------------------------------------------------------
# a1, a2: spectra and phi/b tables
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [(63,), (40, 33), (9, 8, 7)])
def test_lambda_and_coefficient_tables(pe, n):
    prob = _bump_problem(n, N=5, M=7, q=4, p=3)
    basis = fem.ClosedFormBasis(prob.n, prob.box, prob.D)
    with pe.Solver(prob) as s:
        lam = s.lam()
        cf = s.coefficients(0)
        cg = s.coefficients(1)
    # sinpi/cospi on the device vs sin/cos of a rounded angle in the oracle: a few ulp
    np.testing.assert_allclose(lam, basis.lam.reshape(-1), rtol=4e-15, atol=0)
    dT = prob.T / prob.N
    for tab, tau, nodes in ((cf, dT / prob.M, prob.fine_nodes), (cg, dT, prob.coarse_nodes)):
        st = osolver.Stepper(basis.lam.reshape(-1), tau, nodes)
        z = basis.lam.reshape(-1) * tau
        # an ulp of lam moves e^{-lam tau} by about z ulp
        np.testing.assert_array_less(np.abs(tab[0] - st.E), 4e-15 * (1 + z) * st.E + 1e-300)
        for i in range(len(nodes)):
            np.testing.assert_allclose(tab[1 + i], tau * st.b[i], rtol=1e-13, atol=1e-15 * tau)


def test_random_coarse_nodes_drawn_on_device_match_generator(pe):
    prob = _bump_problem((15,), N=4, M=4, p=3)
    with pe.Solver(prob, random_coarse_seed=1234) as s:
        assert s.nodes(1) == I.draw_random_nodes(3, 1234)
        assert s.nodes(0) == prob.fine_nodes


# ---------------------------------------------------------------------------
# a3: P_h f in mode space
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [(70,), (33, 40), (11, 6, 13)])
def test_forcing_modal(pe, n):
    prob = _bump_problem(n, N=3, M=2, R=9)
    sys_ = osolver.ModalSystem(prob)
    with pe.Solver(prob) as s:
        s.set_problem()
        for t in (0.0, 0.3141, 0.999):
            assert _rel(s.forcing_modal(t), sys_.ghat(t), sys_.norm_w) <= 1e-13


# ---------------------------------------------------------------------------
# u0 projection routes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["separable", "quadrature", "nodal"])
def test_initial_projection_routes(pe, kind):
    n = (19, 26)
    prob = _bump_problem(n, N=2, M=2)
    rng = I.SplitMix64(5)
    extra = I.gaussian_bumps(rng, 2, 2, width=(0.1, 0.2))
    prob = I.Problem(prob.d, prob.n, prob.box, prob.D, prob.t0, prob.T, prob.N, prob.M, prob.fine_nodes,
                     prob.coarse_nodes, prob.u0 + extra, prob.forcing, 3, prob.tol)
    full = osolver.ModalSystem(prob, basis="closed_form", forcing_route="full")
    with pe.Solver(prob) as s:
        if kind == "nodal":
            nodal = np.random.default_rng(1).standard_normal(n).reshape(-1)
            s.set_problem(pe.PE_FIELD_NODAL, nodal=nodal)
            ref = full.basis.to_modal_from_nodal(nodal.reshape(n)).reshape(-1)
        else:
            s.set_problem(pe.PE_FIELD_TERMS_SEPARABLE if kind == "separable" else pe.PE_FIELD_TERMS_QUADRATURE)
            ref = full.c0
        got = s.modal(0)
    assert _rel(got, ref, full.norm_w) <= 1e-13


# ---------------------------------------------------------------------------
# a4, a5, a6: coarse sweep, fine sweeps, correction and residual
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["1d", "2d", "3d", "2d_R1_q2"])
def test_parareal_iterates_match_oracle(pe, case):
    if case == "1d":
        prob = _bump_problem((300,), N=6, M=9, R=5)
    elif case == "2d":
        prob = _bump_problem((37, 45), N=5, M=8, R=9)
    elif case == "3d":
        prob = _bump_problem((9, 12, 11), N=4, M=6, R=17)
    else:
        box = ((0.0, 1.0), (0.0, 2.0))
        u0, f, _ = I.sin_mode(2, box, 0.3)
        prob = I.Problem(2, (20, 31), box, 0.3, 0.25, 0.75, 7, 5, I.uniform_nodes(2), I.uniform_nodes(2),
                         u0, f, 3, 1e-12)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=3)
    w = sys_.norm_w
    with pe.Solver(prob) as s:
        s.set_problem()
        for n in range(prob.N + 1):
            assert _rel(s.modal(n), ref.history[0][n], w) <= TOL, ("k=0", n)
        for k in range(1, 4):
            r = s.iterate()
            for n in range(1, prob.N + 1):
                assert _rel(s.modal(n), ref.history[k][n], w) <= TOL, (k, n)
            if k == 1:
                assert r == pytest.approx(ref.residuals[0], rel=1e-9)
            else:
                assert r < 1e-13 and ref.residuals[k - 1] < 1e-13
        nodal = s.solution(prob.N)
    ref_nodal = sys_.to_nodal(ref.U[-1]).reshape(-1)
    assert _rel(nodal, ref_nodal) <= TOL


def _term_mix(kinds, seed):
    """Separable terms with the given time kinds ('e' exponential, 's' sinusoid); rates, frequencies
    (up to 200, several turns per substep) and phases from a SplitMix64 stream."""
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


@pytest.mark.parametrize("kinds", ["e", "s", "es", "e" * 32, "s" * 32, "esse" * 4 + "s", "ses" * 10])
def test_stage_contraction_all_column_counts(pe, kinds):
    """The fine step regroups the q-stage forcing sum into K columns (one per exponential, two per
    sinusoid): K from 1 to the maximum 64, odd and even, against the oracle's stage-by-stage sum."""
    box = ((0.0, 1.0), (0.0, 1.0))
    u0, _, _ = I.sin_mode(2, box, 0.05)
    fine = I.draw_random_nodes(5, 77)
    prob = I.Problem(2, (19, 23), box, 0.05, 0.1, 0.6, 3, 7, fine, I.uniform_nodes(2), u0,
                     _term_mix(kinds, len(kinds)), 3, 1e-12)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    w = sys_.norm_w
    with pe.Solver(prob) as s:
        s.set_problem()
        for k in range(1, 3):
            s.iterate()
            for n in range(1, prob.N + 1):
                assert _rel(s.modal(n), ref.history[k][n], w) <= TOL, (k, n)


def test_config1_solve_to_tolerance(pe):
    """Config 1: 1D, 63 nodes, 8 x 16 RK2/RK2, FP64, residual 1e-12."""
    prob = I.config1()
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=prob.tol)
    with pe.Solver(prob) as s:
        info = s.solve()
        assert info["k"] == ref.k == 2
        assert info["residual"] <= prob.tol
        for n in range(prob.N + 1):
            assert _rel(s.modal(n), ref.U[n], sys_.norm_w) <= TOL
        nodal = s.solution(prob.N)
    err_gpu = quadrature.l2_error_full(nodal.reshape(prob.n), prob.exact, prob.t0 + prob.T, prob.n, prob.box, 5)
    err_ora = quadrature.l2_error_full(sys_.to_nodal(ref.U[-1]), prob.exact, prob.t0 + prob.T, prob.n, prob.box, 5)
    assert err_gpu == pytest.approx(err_ora, rel=1e-9)


def test_config2_full_size_sampled_modes(pe):
    """Config 2 at full size (255^2, 32 x 64, RK4 fine, random-node RK2 coarse), sampled modes."""
    prob = I.config2()
    rng = np.random.default_rng(2)
    idx = np.unique(np.concatenate([[0, 1, 255, prob.ndof - 1], rng.integers(0, prob.ndof, 400)]))
    sys_ = osolver.ModalSystem(prob, modes=idx)
    ref = osolver.parareal(sys_, tol=0.0, k_max=2)
    with pe.Solver(prob) as s:
        info = s.solve(tol=prob.tol)
        assert info["k"] == 2 and info["residual"] <= prob.tol
        for n in (1, prob.N // 2, prob.N):
            got = s.modal(n)[idx]
            assert _rel(got, ref.U[n], sys_.norm_w) <= TOL, n


@pytest.mark.parametrize("tag", ["N1_M1", "n1", "R0"])
def test_degenerate_cases(pe, tag):
    if tag == "N1_M1":
        prob = _bump_problem((23, 9), N=1, M=1)
    elif tag == "n1":
        prob = _bump_problem((1, 1, 5), N=3, M=4)
    else:
        box = ((0.0, 1.0),)
        prob = I.Problem(1, (31,), box, 0.5, 0.0, 1.0, 4, 3, I.uniform_nodes(3), I.uniform_nodes(2),
                         I.sin_mode(1, box, 0.5)[0], (), 3, 1e-12)
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=prob.N)
    with pe.Solver(prob) as s:
        s.set_problem()
        for _ in range(prob.N):
            s.iterate()
        for n in range(prob.N + 1):
            assert _rel(s.modal(n), ref.U[n], sys_.norm_w) <= TOL


def test_state_save_and_resume(pe):
    prob = _bump_problem((21, 34), N=6, M=5)
    with pe.Solver(prob) as s:
        s.set_problem()
        s.iterate()
        blob = s.save_state()
        r2 = s.iterate()
        a = np.stack([s.modal(n) for n in range(prob.N + 1)])
    with pe.Solver(prob) as s2:
        s2.set_problem()
        s2.load_state(blob)
        r2b = s2.iterate()
        b = np.stack([s2.modal(n) for n in range(prob.N + 1)])
    assert r2 == r2b
    assert np.array_equal(a, b)


def test_nonfinite_source_is_reported(pe):
    prob = _bump_problem((16,), N=3, M=2)
    bad = I.Term(float("nan"), prob.forcing[0].factors, prob.forcing[0].tkind, prob.forcing[0].tp)
    prob = I.Problem(prob.d, prob.n, prob.box, prob.D, prob.t0, prob.T, prob.N, prob.M, prob.fine_nodes,
                     prob.coarse_nodes, prob.u0, (bad,) + prob.forcing[1:], 3, 1e-12)
    with pe.Solver(prob) as s:
        s.set_problem()
        with pytest.raises(pe.PEError) as ei:
            s.iterate()
        assert ei.value.status == pe.PE_ENONFINITE


def test_state_errors(pe):
    prob = _bump_problem((16,), N=3, M=2)
    with pe.Solver(prob) as s:
        with pytest.raises(pe.PEError) as ei:
            s.iterate()
        assert ei.value.status == pe.PE_ESTATE
