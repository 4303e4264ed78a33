"""Host side of the mode-sharded solve, on CPU with the gloo backend (world size 2).

Each rank takes its block of axis-0 modes (shard_ranges), runs the CPU oracle's Parareal on
those modes alone (modes are independent, Sec. 2.3), forms its two residual sums per
iteration and its nodal field, and combines them with the other rank through
allreduce_sum.  The combined residuals must equal the unsharded oracle's r_k (Algorithm 1's
stopping rule over every mode) and the combined nodal field its nodal solution; a rank
that stopped early must not be needed for either.  No GPU is involved.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import solver as osolver  # noqa: E402
from paper_2412_01138_gb300 import inputs as I  # noqa: E402
from paper_2412_01138_gb300 import shard  # noqa: E402


def _problem():
    return I.scaled(I.config2(), (21, 13), N=5, M=6)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _shard_sums(sys_, hist_prev, hist_new, N):
    num = sum(float(np.sum(sys_.norm_w * (hist_new[n] - hist_prev[n]) ** 2)) for n in range(1, N + 1))
    den = sum(float(np.sum(sys_.norm_w * hist_new[n] ** 2)) for n in range(1, N + 1))
    return np.array([num, den])


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _problem()
        b, e = shard.shard_ranges(prob.n[0], world)[rank]
        inner = prob.ndof // prob.n[0]
        idx = np.arange(b * inner, e * inner)
        sys_ = osolver.ModalSystem(prob, modes=idx)
        ref = osolver.parareal(sys_, tol=0.0, k_max=3)
        rs = []
        for k in range(1, 4):
            tot = shard.allreduce_sum(_shard_sums(sys_, ref.history[k - 1], ref.history[k], prob.N), dist)
            rs.append(shard.relative_residual(tot))
        # nodal field of this rank's modes alone (the others zero), summed over ranks
        full = osolver.ModalSystem(prob)
        c = np.zeros(prob.ndof)
        c[idx] = ref.U[-1]
        nodal = shard.allreduce_sum(full.to_nodal(c).reshape(-1), dist)
        q.put((rank, (b, e), rs, nodal))
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_every_mode_once():
    for n0, world in ((255, 2), (255, 8), (7, 7), (10, 3), (127, 4)):
        rs = shard.shard_ranges(n0, world)
        assert rs[0][0] == 0 and rs[-1][1] == n0
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        sizes = [e - b for b, e in rs]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_ranges(3, 4)


def test_two_ranks_combine_residuals_and_nodal_fields_like_the_unsharded_solve():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    prob = _problem()
    sys_ = osolver.ModalSystem(prob)
    ref = osolver.parareal(sys_, tol=0.0, k_max=3)
    nodal_ref = sys_.to_nodal(ref.U[-1]).reshape(-1)
    assert out[0][1] == (0, 11) and out[1][1] == (11, 21)
    for rank, _, rs, nodal in out:
        # both ranks see the same combined residual, the unsharded one (up to summation order)
        for k in range(3):
            assert rs[k] == pytest.approx(ref.residuals[k], rel=1e-12, abs=1e-300)
        assert np.abs(nodal - nodal_ref).max() <= 1e-14 * np.abs(nodal_ref).max()


def test_single_process_combination_is_the_identity():
    v = np.array([2.0, 8.0])
    assert np.array_equal(shard.allreduce_sum(v), v)
    assert shard.relative_residual(v) == pytest.approx(0.5)
    assert shard.relative_residual([4.0, 0.0]) == pytest.approx(2.0)
