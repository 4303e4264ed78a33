"""GPU: the integer float32 -> float64 widening that the mixed form's coarse sweeps use in
place of the conversion instruction equals the conversion bit for bit (pe_probe_widen_f32):
every float32 exponent with random and extreme fractions, both signs, zeros, subnormals,
infinities and NaN (NaN compared as NaN)."""
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


def _patterns():
    rng = np.random.default_rng(7)
    exps = np.repeat(np.arange(256, dtype=np.uint32), 64)
    frac = rng.integers(0, 1 << 23, exps.size, dtype=np.uint32)
    frac[::64] = 0                   # powers of two, +-0 and +-inf at the ends of the range
    frac[1::64] = (1 << 23) - 1      # all-ones fractions (largest subnormal, NaN)
    frac[2::64] = 1                  # smallest fraction (smallest subnormal, signalling NaN)
    sign = (rng.integers(0, 2, exps.size, dtype=np.uint32) << 31)
    bits = sign | (exps << 23) | frac
    extra = np.array([0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0x00800000,
                      0x7F7FFFFF, 0x00000001, 0x807FFFFF], dtype=np.uint32)
    return np.concatenate([bits, extra, rng.integers(0, 1 << 32, 1 << 20, dtype=np.uint64).astype(np.uint32)])


def test_integer_widening_equals_the_conversion(env):
    pe, torch = env
    bits = _patterns()
    x = torch.from_numpy(bits.view(np.float32)).cuda()
    y = torch.empty(x.numel(), dtype=torch.float64, device="cuda")
    pe.probe_widen_f32(x, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    ref = x.double().cpu().numpy()  # the conversion instruction (torch's cast kernel)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), ref[~nan].view(np.uint64))
    assert np.array_equal(np.signbit(got[~nan]), np.signbit(ref[~nan]))
