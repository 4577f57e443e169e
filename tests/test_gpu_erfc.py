"""The float32 erfc of the short-range kernels on the device (``-m gpu``).

Sec. 3.1 (Eq. ewald_green_functions) needs erfc(alpha r) in g^(n) and
f^(n).  The float32 form takes it as exp(-x^2) times a fitted erfcx; this
test measures that device function against CUDA's own erfcf (float32) and
erfc (float64, the reference) over the range the kernels use, [0, 8].
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_device_erfc_fit_against_cuda_erfc():
    import paper_2406_07366_gb300 as B
    x = torch.linspace(0.0, 8.0, 200001, dtype=torch.float32, device="cuda")
    ours = torch.empty_like(x)
    B.bs_erfc_f32(x, ours)
    cuda_f32 = torch.special.erfc(x)                # CUDA's erfcf
    exact = torch.special.erfc(x.double())          # CUDA's erfc, float64
    torch.cuda.synchronize()
    ours, cuda_f32, exact = ours.double().cpu().numpy(), cuda_f32.double().cpu().numpy(), exact.cpu().numpy()
    tiny = exact > 1e-37                            # float32 normal range
    rel_ours = np.abs(ours - exact)[tiny] / exact[tiny]
    rel_cuda = np.abs(cuda_f32 - exact)[tiny] / exact[tiny]
    # the fit's 3.4e-7 plus the rounding of expf(-x^2) in float32, which
    # grows like x^2 ulp (x^2 <= 64 carries about 6 bits of its own)
    xs = x.double().cpu().numpy()[tiny]
    bound = 4e-7 + 2 * (xs * xs + 1) * 2.0 ** -24
    assert np.all(rel_ours < bound), float(np.max(rel_ours / bound))
    # and no worse than a few times CUDA's own float32 erfcf where that is accurate
    assert np.median(rel_ours) < 10 * max(np.median(rel_cuda), 6e-8)
