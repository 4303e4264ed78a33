"""Pins of the CPU references behind the learned coarse correction."""
import numpy as np

from oracle import learned, solver
from paper_2412_01138_gb300 import inputs as I


def test_unit_response_reproduces_propagator_difference():
    """F^M(0) - G(0) on every slice equals sum_r P amp Im(e^{i(w T_n + phi)} K): linearity + time shift."""
    rng = I.SplitMix64(5)
    box = ((0.0, 1.0), (0.0, 1.0))
    bumps = I.gaussian_bumps(rng, 2, 3, omega=(1.0, 50.0))
    prob = I.Problem(2, (9, 7), box, 0.02, 0.3, 2.0, 16, 8, I.uniform_nodes(4), I.uniform_nodes(2),
                     I.sin_mode(2, box, 0.02)[0], bumps, 3)
    sys_ = solver.ModalSystem(prob)
    prop = solver.Propagators(sys_)
    zero = np.zeros_like(sys_.lam)
    dT = prob.T / prob.N
    for n in (0, 5, 15):
        direct = prop.FM(zero, n) - prop.G(zero, n)
        via_K = np.zeros_like(sys_.lam)
        for term, P in zip(prob.forcing, sys_._P):
            w, ph = term.tp
            K = learned.unit_response(sys_.lam, w, dT, prob.M, prob.fine_nodes, prob.coarse_nodes)
            via_K += P * term.amp * np.imag(np.exp(1j * (w * prop.T(n) + ph)) * K)
        np.testing.assert_allclose(via_K, direct, rtol=0, atol=1e-13 * np.abs(direct).max())


def test_mlp_gradient_against_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(2 * 64 + 64 + 64 * 64 + 64 + 2 * 64 + 2) * 0.3
    x = rng.standard_normal((17, 2))
    t = rng.standard_normal((17, 2))
    loss, g = learned.mlp_loss_grad(p, x, t)
    for k in rng.choice(p.size, 40, replace=False).tolist() + [0, 200, p.size - 1]:
        e = np.zeros_like(p)
        e[k] = 1e-6
        fd = (learned.mlp_loss_grad(p + e, x, t)[0] - learned.mlp_loss_grad(p - e, x, t)[0]) / 2e-6
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), k
    assert loss == np.sum((learned.mlp_forward(p, x) - t) ** 2) / (2 * 17)
