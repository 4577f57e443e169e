"""Accuracy sweeps after Figs. 3 and A (``-m gpu``) on the paper's three test
geometries (Sec. 5.1): the trefoil knot (Eq. def_trefoil_knot), three pairs
of straight periodic lines (case 2) and random ellipses (case 3, radii
U[L/16, L/4]).

Fig. 3: the total error against the converged oracle as the accuracy
coefficient beta varies at alpha = 24/L (truncation, Sec. 4).
Fig. A: the error of the long-range part alone as the NUFFT width w varies
at sigma = 1.5, beta = 8, alpha = 24/L, against a sigma = 2, w = 16 run
(Appendix A).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_07366_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA, A_CORE, DELTA = 1.0, 1e-6, 0.25
L = 2 * math.pi
ALPHA = 24.0 / L


def _geometry(name):
    if name == "trefoil":
        return W.trefoil(N=128)
    if name == "lines":
        return W.three_line_pairs(N_l=16)
    return W.ellipses(nfil=8, N_l=32, seed=7, semi=(L / 16, L / 4))


def _rms(v, vr):
    return math.sqrt(np.mean(np.sum((v - vr) ** 2, 1)) / np.mean(np.sum(vr ** 2, 1)))


@pytest.mark.parametrize("case", ["trefoil", "lines", "ellipses"])
def test_error_falls_with_beta_within_the_estimate(case):
    """Fig. 3: at alpha = 24/L (r_c = beta/alpha, k_max = 2 beta alpha) the rms
    error of the total velocity against the converged sum falls like
    e^{-beta^2} and stays within a small factor of the Sec. 4 estimate
    (Eq. error_trunc_velocity).  NUFFT at w = 16, sigma = 2 (its error below
    rounding)."""
    import paper_2406_07366_gb300 as B
    f = _geometry(case)
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    vr, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    vrms = math.sqrt(np.mean(np.sum(vr ** 2, 1)))
    nodes = torch.from_numpy(f.nodes).cuda()
    errs, ests = [], []
    for beta in (2.0, 3.0, 4.0, 5.0):
        K = int(math.ceil(beta * ALPHA * L / math.pi))  # k_max = 2 beta alpha
        p = B.make_params(f.L, kappa=KAPPA, a=A_CORE, delta=DELTA, beta=beta, M=2 * K + 1, Q=2, w=16, sigma=2.0,
                          precision=B.BS_FP64, alpha=ALPHA)
        bs = B.BiotSavart(p, f.offsets, f.closing)
        v = bs.velocity(nodes).cpu().numpy()
        bs.status()
        bs.close()
        e = _rms(v, vr)
        ev, _ = B.bs_error_estimate(p, float(g.lp.sum()))
        errs.append(e)
        ests.append(ev / vrms)
        assert e < 3 * ev / vrms, (case, beta, e, ev / vrms)
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    # e^{-beta^2}: from beta = 2 to 5 the factor is e^{-21} ~ 8e-10; the
    # prefactor's 1/beta and the finite sample leave at least 1e-7
    assert errs[-1] / errs[0] < 1e-7, errs


def _long_range(B, f, nodes, w, sigma):
    """The long-range part v^(f) alone (bs_compute_parts, float64 form) at
    alpha = 24/L, beta = 8, M = 128 modes (n_g = 192 at sigma = 1.5)."""
    p = B.make_params(f.L, kappa=KAPPA, a=A_CORE, delta=DELTA, beta=8.0, M=128, Q=2, w=w, sigma=sigma,
                      precision=B.BS_FP64, alpha=ALPHA)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    parts = bs.parts(nodes)
    bs.status()
    out = parts[2].cpu().numpy()
    bs.close()
    return out


# Prefactor C of the measured error C 10^{-0.9 w} at sigma = 1.5.  Appendix A
# reports the slope 10^{-0.9 w}; the level follows from the kernel: a plain
# one-dimensional type-1 transform with the same truncated backwards
# Kaiser-Bessel kernel and the same deconvolution gives 8e-7 rms over all
# modes at w = 8 (3e-6 with every point on a grid node).  The three line
# pairs lie exactly on grid planes, where the aliasing of the kernel's edge
# jump adds up coherently.
PREFACTOR_MAX = {"trefoil": 20.0, "lines": 80.0, "ellipses": 20.0}


@pytest.mark.parametrize("case", ["trefoil", "lines", "ellipses"])
def test_long_range_error_falls_like_ten_to_minus_0_9_w(case):
    """Fig. A: the long-range velocity error at sigma = 1.5, w = 4..14 against
    the sigma = 2, w = 16 run follows C 10^{-0.9 w}: a least-squares slope in
    [0.8, 1.0] decades per unit of w, every point within 3x of the line, C
    bounded.  The reference run itself equals the oracle's direct Fourier sum
    (no NUFFT) to rounding, and sigma = 2 falls like ~10^{-w}."""
    import paper_2406_07366_gb300 as B
    f = _geometry(case)
    nodes = torch.from_numpy(f.nodes).cuda()
    ref = _long_range(B, f, nodes, 16, 2.0)
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    direct, _ = oracle.long_range(g, f.L, KAPPA, ALPHA, 63)
    assert _rms(ref, direct) < 1e-12
    ws = np.array([4, 6, 8, 10, 12, 14])
    errs = np.array([_rms(_long_range(B, f, nodes, int(w), 1.5), ref) for w in ws])
    assert np.all(np.diff(errs) < 0), errs
    slope = -np.polyfit(ws, np.log10(errs), 1)[0]
    assert 0.8 <= slope <= 1.0, (slope, errs)
    C = errs * 10.0 ** (0.9 * ws)
    Cg = float(np.exp(np.mean(np.log(C))))
    assert np.all(C / Cg < 3.0) and np.all(Cg / C < 3.0), (Cg, C)
    assert Cg < PREFACTOR_MAX[case], (Cg, C)
    ws2 = np.array([4, 6, 8, 10, 12])
    errs2 = np.array([_rms(_long_range(B, f, nodes, int(w), 2.0), ref) for w in ws2])
    slope2 = -np.polyfit(ws2, np.log10(errs2), 1)[0]
    assert 0.9 <= slope2 <= 1.15, (slope2, errs2)
