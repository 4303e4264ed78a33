"""Pins of the Q1 assembly and of both diagonalisation routes (Sec. 2.1, Sec. 2.3)."""
import numpy as np
import pytest
import scipy.linalg

from oracle import fem, quadrature, solver
from paper_2412_01138_gb300 import inputs as I


@pytest.mark.parametrize("n,lo,hi", [(1, 0, 1), (5, 0, 1), (31, 0.25, 1.25), (63, 0.125, 0.375)])
def test_axis_eigenpairs_closed_form_vs_dense(n, lo, hi):
    h, _ = fem.axis_grid(lo, hi, n)
    M, K = fem.mass_1d(n, h), fem.stiffness_1d(n, h)
    muM, muK = fem.axis_eigenvalues(n, h)
    lam_dense = scipy.linalg.eigh(K, M, eigvals_only=True)
    # a backward-stable dense eigensolver is accurate to eps * ||lam||_max
    np.testing.assert_allclose(np.sort(muK / muM), lam_dense, rtol=0, atol=1e-13 * lam_dense.max())
    S = fem.dst1_matrix(n)
    np.testing.assert_allclose(S, S.T, atol=0)
    np.testing.assert_allclose(S @ S, np.eye(n), atol=1e-14)
    np.testing.assert_allclose(S @ M @ S, np.diag(muM), atol=1e-13 * np.abs(M).max())
    np.testing.assert_allclose(S @ K @ S, np.diag(muK), atol=1e-13 * np.abs(K).max())


@pytest.mark.parametrize("n", [(3, 4), (4, 3, 5), (7,)])
def test_kron_simultaneous_diagonalisation(n):
    box = tuple((0.0, 1.0 + 0.3 * a) for a in range(len(n)))
    D = 0.37
    M, K = fem.assemble(n, box, D)
    M, K = M.toarray(), K.toarray()
    V = fem.dst1_matrix(n[0])
    for na in n[1:]:
        V = np.kron(V, fem.dst1_matrix(na))
    basis = fem.ClosedFormBasis(n, box, D)
    VMV = V.T @ M @ V
    VKV = V.T @ K @ V
    np.testing.assert_allclose(VMV, np.diag(basis.muM.reshape(-1)), atol=1e-13 * np.abs(M).max())
    np.testing.assert_allclose(VKV, np.diag((basis.muM * basis.lam).reshape(-1)), atol=1e-13 * np.abs(K).max())
    lam_dense = scipy.linalg.eigh(K, M, eigvals_only=True)
    np.testing.assert_allclose(np.sort(basis.lam.reshape(-1)), lam_dense, rtol=0, atol=1e-13 * lam_dense.max())


def test_assembly_against_quadrature():
    """M_ij = int phi_i phi_j and K_ij = D int grad phi_i . grad phi_j on a small 2D grid."""
    n, box, D = (3, 4), ((0.0, 1.0), (0.5, 1.3)), 0.7
    M, K = fem.assemble(n, box, D)
    M, K = M.toarray(), K.toarray()
    hs = [fem.axis_grid(*box[a], n[a])[0] for a in range(2)]
    s, w = quadrature.gauss_legendre(4)
    # integrate hat products element by element, hats written from scratch
    N = n[0] * n[1]
    Mq = np.zeros((N, N))
    Kq = np.zeros((N, N))

    def hat(k, h, y):  # 1D hat of node k (1-based) at local coordinate y in units of h
        return np.maximum(0.0, 1.0 - np.abs(y - k))

    def dhat(k, h, y):
        return np.where(np.abs(y - k) < 1.0, -np.sign(y - k) / h, 0.0)

    for ex in range(n[0] + 1):
        for ey in range(n[1] + 1):
            yx = ex + s
            yy = ey + s
            for i in range(N):
                ix, iy = divmod(i, n[1])
                bi = np.multiply.outer(hat(ix + 1, hs[0], yx), hat(iy + 1, hs[1], yy))
                gxi = np.multiply.outer(dhat(ix + 1, hs[0], yx), hat(iy + 1, hs[1], yy))
                gyi = np.multiply.outer(hat(ix + 1, hs[0], yx), dhat(iy + 1, hs[1], yy))
                for j in range(N):
                    jx, jy = divmod(j, n[1])
                    bj = np.multiply.outer(hat(jx + 1, hs[0], yx), hat(jy + 1, hs[1], yy))
                    gxj = np.multiply.outer(dhat(jx + 1, hs[0], yx), hat(jy + 1, hs[1], yy))
                    gyj = np.multiply.outer(hat(jx + 1, hs[0], yx), dhat(jy + 1, hs[1], yy))
                    W = np.multiply.outer(w, w) * hs[0] * hs[1]
                    Mq[i, j] += np.sum(W * bi * bj)
                    Kq[i, j] += D * np.sum(W * (gxi * gxj + gyi * gyj))
    np.testing.assert_allclose(M, Mq, atol=1e-15)
    np.testing.assert_allclose(K, Kq, atol=1e-13)


@pytest.mark.parametrize("case", ["1d", "2d", "3d"])
def test_dense_full_route_equals_closed_form_separable_route(case):
    """Dense generalized eigensolve + full d-D quadrature load vs DST-I + separable loads.

    Compares nodal solutions after a short Parareal run with bump forcing,
    so the DST, the eigenvalues, the separable projection and the stepping
    are all checked against an independent route.
    """
    rng = I.SplitMix64(99)
    if case == "1d":
        n, box = (9,), ((0.0, 1.0),)
    elif case == "2d":
        n, box = (6, 5), ((0.0, 1.0), (0.0, 0.7))
    else:
        n, box = (4, 3, 5), ((0.0, 1.0),) * 3
    d = len(n)
    u0, f, _ = I.sin_mode(d, box, 0.3)
    bumps = I.gaussian_bumps(rng, d, 3, width=(0.15, 0.3))
    prob = I.Problem(d, n, box, 0.3, 0.1, 0.8, 3, 4, I.uniform_nodes(3), I.draw_random_nodes(2, 5),
                     u0 + bumps[:1], f + bumps, 3)
    a = solver.ModalSystem(prob, basis="closed_form", forcing_route="separable")
    b = solver.ModalSystem(prob, basis="dense", forcing_route="full")
    ra = solver.parareal(a, tol=0.0, k_max=2)
    rb = solver.parareal(b, tol=0.0, k_max=2)
    for n_ in range(prob.N + 1):
        ua = a.to_nodal(ra.U[n_])
        ub = b.to_nodal(rb.U[n_])
        np.testing.assert_allclose(ua, ub, rtol=0, atol=1e-12 * np.abs(ub).max())
    # the M-norm in both bases agrees with u^T M u
    M, _ = fem.assemble(n, box, 0.3)
    u = a.to_nodal(ra.U[-1]).reshape(-1)
    assert a.norm(ra.U[-1]) == pytest.approx(np.sqrt(u @ (M @ u)), rel=1e-13)
    assert b.norm(rb.U[-1]) == pytest.approx(np.sqrt(u @ (M @ u)), rel=1e-12)
