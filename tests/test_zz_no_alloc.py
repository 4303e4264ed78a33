"""The allocation-free DST entry point (pe_dst_noalloc) against the allocating one (pe_dst).

Some callers cannot allocate device memory while they run (for example an application
with its own fixed memory pool, or a loop that must not enter the synchronising allocator);
pe_dst_noalloc serves them from a built-in device array.  This file is collected last
so that a failure here cannot hide the rest of the suite.  Two calls in a row go
through the C-ABI with different sizes and paths (FFT lengths and the matrix path),
and both must match pe_dst within the DST tolerance of the other tests.
"""
import numpy as np
import pytest

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


def test_noalloc_matches_allocating_dst_on_two_calls_in_a_row(env):
    pe, torch = env
    rng = np.random.default_rng(12)
    # FFT path, matrix path, d = 1 at the largest FFT length, and mixed FFT / matrix axes in
    # both slot orders (2D and 3D)
    for n in [(255, 255), (100, 37, 9), (1023,), (63, 100), (100, 63, 31)]:
        x = torch.tensor(rng.standard_normal(int(np.prod(n))), device="cuda", dtype=torch.float64)
        ref = torch.empty_like(x)
        got = torch.empty_like(x)
        pe.dst(len(n), n, x, ref)
        pe.dst_noalloc(len(n), n, x, got)
        torch.cuda.synchronize()
        assert _rel(got.cpu().numpy(), ref.cpu().numpy()) <= 1e-14 * max(n)
        # in place
        y = x.clone()
        pe.dst_noalloc(len(n), n, y, y)
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy(), ref.cpu().numpy()) <= 1e-14 * max(n)


def test_noalloc_rejects_sizes_beyond_its_array(env):
    """The caller's buffers are full size (prod(n) values), so that only the size limit, not a
    short buffer, is what the call is checked against."""
    pe, torch = env
    for n, word in (((1023, 1023, 3), "1048576"), ((600,), "512")):
        x = torch.zeros(int(np.prod(n)), device="cuda", dtype=torch.float64)
        with pytest.raises(pe.PEError) as ei:
            pe.dst_noalloc(len(n), n, x, x)
        assert ei.value.status == pe.PE_EINVAL and word in str(ei.value)
        del x
