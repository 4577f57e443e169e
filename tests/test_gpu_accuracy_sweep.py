"""Accuracy sweeps after Figs. 3 and A (``-m gpu``): the error of the fast
method against the converged oracle on the trefoil, as the accuracy
coefficient beta (truncation, Sec. 4) and the NUFFT width w (App. A) vary."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_07366_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA, A_CORE, DELTA = 1.0, 1e-6, 0.25


def _setup():
    import paper_2406_07366_gb300 as B
    f = W.trefoil(N=128)
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    vr, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    return B, f, g, vr, torch.from_numpy(f.nodes).cuda()


def _rms(v, vr):
    return math.sqrt(np.mean(np.sum((v - vr) ** 2, 1)) / np.mean(np.sum(vr ** 2, 1)))


def test_error_falls_with_beta_within_the_estimate():
    """Fig. 3: at fixed M = 64 (alpha = k_max / 2 beta) the error falls like
    e^{-beta^2} and stays within a small factor of the Sec. 4 estimate."""
    B, f, g, vr, nodes = _setup()
    vrms = math.sqrt(np.mean(np.sum(vr ** 2, 1)))
    errs = []
    for beta in (2.0, 3.0, 4.0, 5.0):
        p = B.make_params(f.L, beta=beta, M=64, Q=2, w=16, sigma=2.0, precision=B.BS_FP64)
        bs = B.BiotSavart(p, f.offsets, f.closing)
        v = bs.velocity(nodes).cpu().numpy()
        bs.close()
        e = _rms(v, vr)
        ev, _ = B.bs_error_estimate(p, float(g.lp.sum()))
        assert e < 3 * ev / vrms, (beta, e, ev / vrms)
        errs.append(e)
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-8 and errs[0] > 1e-4, errs


def test_error_falls_with_nufft_width():
    """App. A (Fig. A): with the truncation negligible (beta = 8), the NUFFT
    error at sigma = 1.5 falls roughly like 10^{-0.9 w}."""
    B, f, g, vr, nodes = _setup()
    errs = []
    for w in (4, 6, 8, 10):
        p = B.make_params(f.L, beta=8.0, M=96, Q=2, w=w, sigma=1.5, precision=B.BS_FP64)
        bs = B.BiotSavart(p, f.offsets, f.closing)
        v = bs.velocity(nodes).cpu().numpy()
        bs.close()
        e = _rms(v, vr)
        assert e < 10 * 10 ** (-0.9 * w), (w, e)
        errs.append(e)
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
