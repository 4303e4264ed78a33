"""GPU: the mixed form's transforms between nodal values and modal coefficients.

The mixed form rounds float64 nodal u0 to float32, applies the tensor DST-I in float32 and
widens the coefficients back to float64 (and the reverse for the nodal output); on grids whose
axes all have n = 255 the two-pass kernels read the float64 input in their first pass and write
the float64 output in their last.  U^0 of a solve with nodal u0 must equal the float64
transform of u0 to float32 accuracy (the oracle's dense matrices), element by element against
the largest coefficient, and the nodal output must be the transform of the final modal
iterate, on a 255 x 255 grid (the two-pass kernels), a 63 x 255 grid (not every axis at
n = 255: float32 transform between separate conversions) and a 255-node line (below 4096
nodes the mixed form keeps float64 transforms).
"""
import numpy as np
import pytest

from oracle import fem
from paper_2412_01138_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_01138_gb300 import pe as _pe

    _pe.lib()
    return _pe


def _dst(x):
    out = x
    for a in range(x.ndim):
        out = fem.apply_axis(fem.dst1_matrix(x.shape[a]), out, a)
    return out


@pytest.mark.parametrize("n", [(255, 255), (255,), (63, 255)], ids=["255x255", "255", "63x255"])
def test_mixed_form_transforms_u0_and_output(pe, n):
    base = I.config2() if len(n) == 2 else I.config1()
    prob = I.scaled(base, n, N=4, M=16)
    rng = np.random.default_rng(17)
    u0 = rng.standard_normal(n)
    with pe.Solver(prob, precision=pe.PE_MIXED) as s:
        s.solve(tol=1e-6, u0_kind=pe.PE_FIELD_NODAL, nodal=u0.reshape(-1).copy())
        c0 = s.modal(0).reshape(n)
        cN = s.modal(prob.N).reshape(n)
        nodal = s.solution(prob.N).reshape(n)
    ref0 = _dst(u0)
    assert np.abs(c0 - ref0).max() <= 2e-6 * np.abs(ref0).max()
    refN = _dst(cN)
    assert np.abs(nodal - refN).max() <= 2e-6 * np.abs(refN).max()
