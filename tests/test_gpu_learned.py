"""GPU tests of the learned coarse correction: label generation, gradients, training, and its gain.

* labels: the library's method-generated K(lam, w) against the CPU reference;
* gradients of the hand-written backward kernels against the float64 CPU
  reference (the float32 kernels accumulate in float32: relative 1e-4);
* the trained network (weights from held-apart seeds 100000+) cuts the Parareal
  iterations on the learned workload's family from 2 to 1 while the answer stays
  the fine solution (<= 1e-12 float64, <= 1e-6 mixed).
"""
import numpy as np
import pytest

from oracle import learned as olearned
from oracle import solver as osolver
from paper_2412_01138_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_01138_gb300 import pe

    pe.lib()
    return pe, torch


def _prob(seed=1, n=63):
    return I.scaled(I.config5(seed=seed), (n, n))


def training_set(pe, torch, solver, prob, seeds, n_lam, rng_seed=123):
    """Method-generated (features, targets) from the frequencies of held-apart seeds."""
    lam = solver.lam()
    lo, hi = np.log(lam.min()), np.log(lam.max())
    rng = np.random.default_rng(rng_seed)
    L, W = [], []
    for s in seeds:
        ws = [t.tp[0] for t in I.config5(seed=s, n=prob.n[0]).forcing]
        ls = np.exp(rng.uniform(lo, hi, n_lam))
        L.append(np.repeat(ls, len(ws)))
        W.append(np.tile(ws, n_lam))
    L, W = np.concatenate(L), np.concatenate(W)
    perm = rng.permutation(L.size)
    L, W = L[perm], W[perm]
    dev = torch.device("cuda")
    lam_d = torch.tensor(L, device=dev)
    om_d = torch.tensor(W, device=dev)
    x = torch.empty((L.size, 2), device=dev, dtype=torch.float32)
    t = torch.empty((L.size, 2), device=dev, dtype=torch.float32)
    K = torch.empty((L.size, 2), device=dev, dtype=torch.float64)
    solver.learned_samples(lam_d, om_d, x, t, K)
    return L, W, x, t, K


def test_labels_match_cpu_reference(env):
    pe, torch = env
    prob = _prob()
    with pe.Solver(prob) as s:
        L, W, x, t, K = training_set(pe, torch, s, prob, range(100000, 100004), 16)
    dT = prob.T / prob.N
    ref = olearned.unit_response(L, W, dT, prob.M, prob.fine_nodes, prob.coarse_nodes)
    got = K.cpu().numpy()
    np.testing.assert_allclose(got[:, 0] + 1j * got[:, 1], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    xr, tr = olearned.features_targets(L, W, dT, ref)
    np.testing.assert_allclose(x.cpu().numpy(), xr, rtol=2e-7, atol=2e-7)
    np.testing.assert_allclose(t.cpu().numpy(), tr, rtol=1e-6, atol=1e-6 * np.abs(tr).max())


def test_gradient_and_forward_match_cpu_reference(env):
    pe, torch = env
    rng = np.random.default_rng(1)
    net = pe.MLP(seed=7)
    p = (rng.standard_normal(net.n_params) * 0.2).astype(np.float32)
    net.set_params(p)
    x = rng.standard_normal((333, 2)).astype(np.float32)
    t = rng.standard_normal((333, 2)).astype(np.float32)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    g, loss = net.gradient(xd, td)
    loss_ref, g_ref = olearned.mlp_loss_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    # inference uses the float16 copy of the weights, float32 accumulation
    y = torch.empty_like(xd)
    net.forward(xd, y)
    y_ref = olearned.mlp_forward(p.astype(np.float16).astype(np.float64), x.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), y_ref, rtol=0, atol=1e-4 * np.abs(y_ref).max())
    net.close()


@pytest.fixture(scope="module")
def trained(env):
    pe, torch = env
    prob = _prob()
    net = pe.MLP(seed=3)
    with pe.Solver(prob) as s:
        L, W, x, t, K = training_set(pe, torch, s, prob, range(100000, 100400), 32)
        loss0 = net.gradient(x[:4096], t[:4096])[1]
        loss = net.train(x, t, epochs=800, batch=2048, lr=3e-3)  # about 60000 Adam steps
        # held-out seeds
        Lh, Wh, xh, th, Kh = training_set(pe, torch, s, prob, range(200000, 200020), 32, rng_seed=9)
    return net, loss0, loss, xh, th


def test_training_fits_held_out_pairs(env, trained):
    pe, torch = env
    net, loss0, loss, xh, th = trained
    assert loss < 1e-4 * loss0
    y = torch.empty_like(xh)
    net.forward(xh, y)
    err = (y - th).norm() / th.norm()
    assert float(err) < 3e-3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_learned_coarse_correction_saves_a_sweep(env, trained, precision):
    pe, torch = env
    net = trained[0]
    prob = _prob(seed=1)
    prec = pe.PE_FP64 if precision == "fp64" else pe.PE_MIXED
    sys_ = osolver.ModalSystem(prob)
    fine = osolver.sequential_fine(sys_)
    tol = 1e-6
    with pe.Solver(prob, precision=prec) as s:
        plain = s.solve(tol=tol)
        s.set_learned(net)
        s.set_problem()
        # the k = 0 iterate's distance to the fine solution, in the residual's norm
        num = sum(sys_.norm(s.modal(n) - fine[n]) ** 2 for n in range(1, prob.N + 1))
        den = sum(sys_.norm(fine[n]) ** 2 for n in range(1, prob.N + 1))
        k0_err = (num / den) ** 0.5
        lrn = s.solve(tol=tol)
        got = [s.modal(n) for n in range(prob.N + 1)]
    assert plain["k"] == 2
    assert k0_err < tol
    assert lrn["k"] == 1 and lrn["residual"] <= tol
    bound = 1e-12 if precision == "fp64" else 1e-6
    for n in range(1, prob.N + 1):
        assert osolver.rel_l2(got[n], fine[n], sys_.norm_w) <= bound, n


@pytest.mark.parametrize("engine", ["tc", "simt"])
def test_batched_learned_correction_saves_a_sweep(env, trained, engine):
    """The mixed, batched form with the learned coarse correction (and the tensor-core fine
    engine): three problems of the learned workload's family in one batch stop after one fine
    sweep each, at the fine solution (<= 1e-6)."""
    pe, torch = env
    net = trained[0]
    probs = [_prob(seed=s) for s in (1, 2, 3)]
    eng = pe.PE_FINE_TC if engine == "tc" else pe.PE_FINE_SIMT
    with pe.BatchSolver(probs, precision=pe.PE_MIXED, fine_engine=eng) as b:
        plain = b.solve(tol=1e-6)
        _, k_plain = b.status()
        b.set_learned(net)
        info = b.solve(tol=1e-6)
        r, k = b.status()
        got = [b.modal(i, p.N) for i, p in enumerate(probs)]
    assert list(k_plain) == [2, 2, 2] and plain["graph_replays"] == 2
    assert list(k) == [1, 1, 1] and info["graph_replays"] == 1 and float(r.max()) <= 1e-6
    for prob, g in zip(probs, got):
        sys_ = osolver.ModalSystem(prob)
        fine = osolver.sequential_fine(sys_)
        assert osolver.rel_l2(g, fine[-1], sys_.norm_w) <= 1e-6
