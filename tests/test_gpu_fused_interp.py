"""The inverse z transform fused with the interpolation (type-2 step of
Sec. 3.3, Appendix A) against the grid path it replaces (``-m gpu``).

The default pruned pipeline sums each node's long-range velocity from the
z-lines of the column blocks its support reaches, in shared memory, without
writing the real grid.  The deterministic mode and the cuFFT form write the
grid and gather from it.  Both compute the same sum of the same grid values,
so they agree to rounding: 1e-12 of the scale in float64, 2e-6 in the mixed
form (float32 partial sums in a different order).
"""
import math

import numpy as np
import pytest

from paper_2406_07366_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _long_part(f, p):
    import paper_2406_07366_gb300 as B
    bs = B.BiotSavart(p, f.offsets, f.closing)
    nodes = torch.from_numpy(f.nodes).cuda()
    out = bs.parts(nodes)
    bs.status()
    torch.cuda.synchronize()
    bs.close()
    return out.cpu().numpy()[2]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("M,w", [(48, 8), (64, 6), (40, 4)])
def test_fused_interp_equals_grid_gather(prec, M, w):
    import paper_2406_07366_gb300 as B
    f = W.fourier_tangle(150, 40, seed=21, amp=2 * math.pi / 40)
    pr = B.BS_FP64 if prec == "fp64" else B.BS_MIXED
    fused = _long_part(f, B.make_params(f.L, M=M, Q=2, w=w, precision=pr))
    grid = _long_part(f, B.make_params(f.L, M=M, Q=2, w=w, precision=pr, flags=B.BS_DETERMINISTIC))
    tol = 1e-12 if prec == "fp64" else 2e-6
    scale = np.abs(grid).max()
    assert scale > 0
    assert np.abs(fused - grid).max() < tol * scale


def test_small_grid_falls_back_to_the_grid_path():
    """A grid too narrow for the fused kernel's block neighbourhood takes the
    grid path: M = 9, sigma = 1.5 give a 16^3 grid of 4 x 4 column blocks,
    and a w = 10 support reaches 5 blocks per axis.  The result still equals
    the full cuFFT form."""
    import paper_2406_07366_gb300 as B
    f = W.ring(N=32)
    outs = [_long_part(f, B.make_params(f.L, M=9, Q=2, w=10, precision=B.BS_FP64, beta=2.0, flags=extra))
            for extra in (0, B.BS_FFT_CUFFT)]
    assert np.abs(outs[0] - outs[1]).max() < 1e-12 * np.abs(outs[1]).max()
