"""Tensor-core (tcgen05, split-bfloat16) DST-I against the float64 oracle transform.

Bounds: nsplit 2 (three bf16 products) 3e-5; nsplit 3 (six products) 5e-6.  With
six products the operand split carries about 24 bits; what remains is the tensor
core's own float32 accumulation over K = 6 * roundup(n, 64) products (2.9e-6
measured at n = 255), so the bound is set by the accumulator, not by the split.
"""
import numpy as np
import pytest

from oracle import fem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_01138_gb300 import pe

    pe.lib()
    return pe, torch


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [(63,), (255,), (1, 7), (255, 255), (100, 37), (31, 17, 9), (127, 15, 33)])
@pytest.mark.parametrize("nsplit", [2, 3])
def test_dst_tc_matches_oracle(env, n, nsplit):
    pe, torch = env
    rng = np.random.default_rng(sum(n) + nsplit)
    x = rng.standard_normal(n).astype(np.float32)
    ref = x.astype(np.float64)
    for a in range(len(n)):
        ref = fem.apply_axis(fem.dst1_matrix(n[a]), ref, a)
    xd = torch.tensor(x.reshape(-1), device="cuda")
    out = torch.empty_like(xd)
    pe.dst_tc(len(n), n, xd, out, nsplit=nsplit)
    torch.cuda.synchronize()
    err = _rel(out.cpu().numpy().astype(np.float64), ref.reshape(-1))
    assert err <= (3e-5 if nsplit == 2 else 5e-6), err
    # in place
    pe.dst_tc(len(n), n, xd, xd, nsplit=nsplit)
    torch.cuda.synchronize()
    assert _rel(xd.cpu().numpy().astype(np.float64), ref.reshape(-1)) == pytest.approx(err, rel=1e-6, abs=1e-12)
