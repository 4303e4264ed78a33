"""GPU parity of every dispatch class of the tensor DST-I (Sec. 2.3) against the oracle.

The library picks a kernel per axis pass from the transform length n + 1, the
number of pencils of the pass (more than 304: one warp per pencil pair; at
most 304: one pencil pair per CTA) and whether the pencils are contiguous (the
last axis) or strided (the others).  Each shape below drives one pass through
a class that the smaller shapes of test_gpu_parity.py never reach, in float64
and float32, and compares with the oracle's dense DST-I matrices applied axis
by axis, both in the weighted rel-L2 sense and element by element
(max |got - ref| / max |ref|).  The (511, 511, 255) grid of the standalone DST
measurement is compared on full slabs of sampled first-axis indices.
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


def _oracle_dst(x):
    ref = x
    for a in range(x.ndim):
        ref = fem.apply_axis(fem.dst1_matrix(x.shape[a]), ref, a)
    return ref


def _errors(got, ref):
    got, ref = got.reshape(-1), ref.reshape(-1)
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    elem = float(np.abs(got - ref).max() / np.abs(ref).max())
    return rel, elem


# (shape, the classes its passes reach: n + 1 and contiguous / strided pencils, > 304 pencils)
SHAPES = [
    ((400, 15), "L=32 contiguous"),
    ((15, 400), "L=32 strided"),
    ((400, 31), "L=64 contiguous"),
    ((31, 400), "L=64 strided"),
    ((400, 63), "L=128 contiguous"),
    ((63, 400), "L=128 strided"),
    ((400, 127), "n+1=128 contiguous (float64 half-length form)"),
    ((127, 400), "n+1=128 strided"),
    ((400, 255), "n+1=256 contiguous"),
    ((255, 400), "n+1=256 strided"),
    ((320, 511), "n+1=512 contiguous"),
    ((511, 320), "n+1=512 strided"),
    ((310, 1023), "n+1=1024 contiguous"),
    ((1023, 310), "n+1=1024 strided"),
    ((400, 7), "n+1=8 block radix-2 kernel with many pencils"),
    ((15, 31, 63), "three warp classes in one 3D transform"),
    ((300, 65), "matrix form, 64x64 tiles"),
    ((9, 100), "matrix form, 32x32 tiles"),
]


@pytest.mark.parametrize("n,label", SHAPES, ids=[s[1] for s in SHAPES])
def test_dst_dispatch_class_matches_oracle(env, n, label):
    pe, torch = env
    rng = np.random.default_rng(int(np.prod(n)) % 100003)
    x = rng.standard_normal(n)
    ref = _oracle_dst(x)
    xd = torch.tensor(x.reshape(-1), device="cuda", dtype=torch.float64)
    out = torch.empty_like(xd)
    pe.dst(len(n), n, xd, out)
    torch.cuda.synchronize()
    rel, elem = _errors(out.cpu().numpy(), ref)
    assert rel <= 1e-14 * max(n) and elem <= 1e-14 * max(n), (label, rel, elem)
    # the involution S^2 = I through the same kernels, in place
    pe.dst(len(n), n, out, out)
    torch.cuda.synchronize()
    rel, elem = _errors(out.cpu().numpy(), x)
    assert rel <= 1e-14 * max(n) and elem <= 1e-14 * max(n), (label, rel, elem)
    # float32: rounding of the input and float32 butterflies, about 1e-7 per pass
    xf = xd.float()
    of = torch.empty_like(xf)
    pe.dst(len(n), n, xf, of, f32=True)
    torch.cuda.synchronize()
    rel, elem = _errors(of.double().cpu().numpy(), ref)
    assert rel <= 2e-6 and elem <= 1e-5, (label, rel, elem)


def test_dst_bench_grid_on_sampled_slabs(env):
    """The (511, 511, 255) grid (n + 1 = 512, 512, 256: every pass in the warp classes),
    float64 and float32, compared on the full output slabs of 6 sampled first-axis indices
    (each slab computed by the oracle's dense matrices: S_0 rows, then S_1, then S_2)."""
    pe, torch = env
    n = (511, 511, 255)
    gen = torch.Generator(device="cpu").manual_seed(31)
    x = torch.randn(n, dtype=torch.float64, generator=gen).numpy()
    rows = np.array([0, 1, 97, 255, 400, 510])
    S0, S1, S2 = fem.dst1_matrix(n[0]), fem.dst1_matrix(n[1]), fem.dst1_matrix(n[2])
    part = (S0[rows] @ x.reshape(n[0], -1)).reshape(len(rows), n[1], n[2])
    part = np.einsum("jk,skl->sjl", S1, part)
    ref = part @ S2.T
    xd = torch.from_numpy(x.reshape(-1)).cuda()
    for dtype, bound_rel, bound_elem in ((torch.float64, 1e-12, 1e-12), (torch.float32, 2e-6, 1e-5)):
        src = xd.to(dtype)
        out = torch.empty_like(src)
        pe.dst(3, n, src, out, f32=dtype == torch.float32)
        torch.cuda.synchronize()
        got = out.view(n)[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        rel, elem = _errors(got, ref)
        assert rel <= bound_rel and elem <= bound_elem, (dtype, rel, elem)
        del src, out


# The two-pass float32 kernels at n = 255 choose one-warp CTAs for passes of fewer than
# 4 x 8 x (SMs) pencils and eight-warp CTAs above; (255, 17) and (255, 5000) put the strided
# pass in each class, (17, 255) and (5000, 255) the contiguous one.
TWO_PASS = [((255, 17), "strided, one-warp CTAs"), ((255, 5000), "strided, eight-warp CTAs"),
            ((17, 255), "contiguous, one-warp CTAs"), ((5000, 255), "contiguous, eight-warp CTAs"),
            ((255,), "one pencil")]


@pytest.mark.parametrize("n,label", TWO_PASS, ids=[s[1] for s in TWO_PASS])
def test_two_pass_float32_classes(env, n, label):
    pe, torch = env
    rng = np.random.default_rng(int(np.prod(n)) % 9973)
    x = rng.standard_normal(n)
    ref = _oracle_dst(x)
    xf = torch.tensor(x.reshape(-1), device="cuda", dtype=torch.float32)
    of = torch.empty_like(xf)
    pe.dst(len(n), n, xf, of, f32=True)
    torch.cuda.synchronize()
    rel, elem = _errors(of.double().cpu().numpy(), ref)
    assert rel <= 2e-6 and elem <= 1e-5, (label, rel, elem)
