"""Host-side tests of the C ABI (no GPU needed).

The library loads, exports every function include/bsewald.h declares, and
its host helpers (parameters from beta, error estimates, NUFFT grid and
deconvolution tables, argument validation) agree with independent
computations.  No compute call is made without a GPU.
"""
import json
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))


@pytest.fixture(scope="module")
def B():
    import paper_2406_07366_gb300 as B
    if not os.path.exists(B.LIB_PATH):
        from paper_2406_07366_gb300.build import build_library
        build_library()
    B.lib()
    return B


def _declared():
    src = open(os.path.join(ROOT, "include", "bsewald.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bs_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(B):
    import ctypes
    lib = ctypes.CDLL(B.LIB_PATH)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.EXPORTS) == names


def test_params_from_beta_with_modes(B):
    """Sec. 4: k_max = (2 pi / L) floor((M-1)/2), alpha = k_max/(2 beta), r_c = beta/alpha."""
    L = 2 * math.pi
    for beta, M in [(3.5, 32), (3.5, 64), (3.5, 256), (2.0, 48), (5.5, 128)]:
        p = B.bs_params_from_beta(beta, [L] * 3, M=M)
        K = (M - 1) // 2
        assert p.alpha == pytest.approx(K / (2 * beta), rel=1e-15)
        assert p.rc == pytest.approx(beta / p.alpha, rel=1e-15)
        assert list(p.M) == [M] * 3


def test_params_from_beta_table_and_optimal_alpha(B):
    """Table tab:performance: w per beta; Eq. alpha_optimal_performance for M = 0."""
    L = 2 * math.pi
    for row in GOLD["performance_table"]["rows"]:
        tol, beta, Cb, sigma, w = row[:5]
        p = B.bs_params_from_beta(beta, [L] * 3, M=0, N=2 ** 18)
        assert p.nufft_w == w and p.nufft_sigma == sigma
        alpha0 = max(Cb * (2 ** 18) ** (1 / 3) / L, 2 * beta / L)
        K = math.ceil(beta * alpha0 * L / math.pi)
        assert p.M[0] == 2 * K + 1
        assert p.alpha == pytest.approx(K / (2 * beta), rel=1e-14)
        assert p.rc <= L / 2 + 1e-12


def test_error_estimate_formula(B):
    """Sec. 4, Eqs. error_trunc_velocity and error_trunc_streamfunction."""
    L = 2 * math.pi
    V = L ** 3
    p = B.bs_params_from_beta(3.5, [L] * 3, M=32)
    Lt = 6.58
    ev, ep = B.bs_error_estimate(p, Lt)
    beta = p.alpha * p.rc
    g = math.sqrt(Lt / (8 * math.pi * V))
    ev_ref = (Lt / (math.sqrt(math.pi) * p.alpha * V) + g / beta) * math.exp(-beta ** 2)
    ep_ref = 1 / (2 * p.alpha) * (Lt / (p.alpha * V) + g / math.sqrt(beta)) * math.exp(-beta ** 2) / beta ** 1.5
    assert ev == pytest.approx(ev_ref, rel=1e-14)
    assert ep == pytest.approx(ep_ref, rel=1e-14)


def _smooth(n):
    for q in (2, 3, 5, 7):
        while n % q == 0:
            n //= q
    return n == 1


@pytest.mark.parametrize("M,sigma,w", [(32, 1.5, 8), (64, 1.5, 8), (256, 1.5, 6), (512, 1.5, 6), (41, 2.0, 16)])
def test_nufft_grid_and_deconvolution(B, M, sigma, w):
    """Appendix A: grid of at least sigma M points (FFT-friendly, multiple of
    8); F(m) is the Fourier transform of the normalised backwards
    Kaiser-Bessel kernel over the w-point support, checked by adaptive
    quadrature."""
    from scipy.integrate import quad
    p = B.make_params([2 * math.pi] * 3, M=M, sigma=sigma, w=w)
    ng, tab = B.bs_nufft_setup(p)
    for n in ng:
        assert n >= sigma * M and n % 8 == 0 and _smooth(n)
    zeta = GOLD["nufft_error"]["gamma"] * w * math.pi * (1 - 1 / (2 * ng[0] / M))
    sh = math.sinh(zeta)

    def kern(z):
        s = math.sqrt(max(1 - z * z, 0.0))
        return math.sinh(zeta * s) / (s * sh) if s > 0 else zeta / sh

    K = (M - 1) // 2
    for m in sorted({0, 1, K // 2, K}):
        kap = math.pi * m * w / ng[0]
        ref = 0.5 * w * quad(lambda z: kern(z) * math.cos(kap * z), -1, 1, limit=200, epsabs=0, epsrel=1e-13)[0]
        assert tab[0][m] == pytest.approx(ref, rel=1e-11)
        # the closed-form pair of Eq. kaiser_bessel_bw is the transform of
        # the kernel's analytic form; the truncated kernel differs from it
        # by a relative remainder below 2e-4 at these zeta
        from scipy.special import i0
        closed = 0.5 * w * math.pi * i0(math.sqrt(zeta ** 2 - kap ** 2)) / sh
        assert tab[0][m] == pytest.approx(closed, rel=2e-4)


def test_validation_errors(B):
    L = [2 * math.pi] * 3

    def code(p):
        with pytest.raises(B.BSError) as e:
            B.bs_nufft_setup(p)
        return e.value.code

    p = B.make_params(L, M=32)
    p.rc = 0.51 * L[0]
    assert code(p) == B.BS_ERR_RC_GT_HALF_L
    p = B.make_params(L, M=32, w=7)
    assert code(p) == B.BS_ERR_ARG
    p = B.make_params(L, M=32, order=5)
    assert code(p) == B.BS_ERR_ARG
    assert "spline_order" in B.bs_last_error()
    p = B.make_params(L, M=32, sigma=1.0)
    assert code(p) == B.BS_ERR_ARG
    p = B.make_params(L, M=32)
    p.M[1] = 2
    assert code(p) == B.BS_ERR_ARG
    p = B.make_params(L, M=1024, sigma=1.5)
    assert code(p) == B.BS_ERR_ARG  # grid above 1024 points
    p = B.make_params(L, M=32)
    p.a = 0.0
    assert code(p) == B.BS_ERR_ARG


def test_create_fails_cleanly_without_a_device(B):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    p = B.make_params([2 * math.pi] * 3, M=32)
    with pytest.raises(B.BSError) as e:
        B.bs_create(p)
    assert e.value.code == B.BS_ERR_CUDA


def test_tangle_params_clamp_modes(B):
    """Batch members: alpha from C_beta N^(1/3) (Eq. alpha_optimal_performance),
    M clamped to [32, 128], alpha re-derived so that r_c alpha = beta."""
    L = [2 * math.pi] * 3
    small = B.tangle_params(200, L)
    big = B.tangle_params(100000, L)
    assert small.M[0] == 32 and big.M[0] == 128
    assert B.bs_params_from_beta(3.5, L, M=0, N=200).M[0] < 32
    mid = B.tangle_params(10000, L)
    free = B.bs_params_from_beta(3.5, L, M=0, N=10000)
    assert 32 <= mid.M[0] <= 128 and mid.M[0] == free.M[0]
    for p in (small, mid, big):
        assert p.alpha * p.rc == pytest.approx(3.5, rel=1e-14)
        assert p.alpha == pytest.approx(((p.M[0] - 1) // 2) / (2 * 3.5), rel=1e-14)


def test_library_has_no_unresolved_internal_symbols(B):
    """Every template the translation units use across files is instantiated:
    no symbol of the library's own namespace is left undefined (the dynamic
    loader would refuse the library on the GPU host)."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--undefined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    internal = [ln for ln in out.splitlines() if "_ZN3bsw" in ln]
    assert not internal, internal


def test_fma_peak_rejects_a_null_output(B):
    assert B.lib().bs_fma_peak(B.BS_MIXED, None) == B.BS_ERR_ARG
