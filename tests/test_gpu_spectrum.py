"""Energy spectrum on the grid (``-m gpu``), Eq. def_energy_spectrum."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_07366_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA = 1.0


def _B():
    import paper_2406_07366_gb300 as B
    return B


@pytest.mark.parametrize("prec,w,sigma,tol", [("fp64", 16, 2.0, 1e-9), ("mixed", 8, 1.5, 2e-5)])
@pytest.mark.parametrize("smoothed", [False, True])
def test_spectrum_matches_direct_fourier_sum(prec, w, sigma, tol, smoothed):
    """The spectrum from the spread and the pruned forward transforms equals
    the oracle's direct Fourier sum over the same mode cube, shell by shell
    (relative to the largest shell), for the full and the smoothed field."""
    B = _B()
    f = W.ellipses(nfil=8, N_l=32, seed=11)
    P = B.BS_FP64 if prec == "fp64" else B.BS_MIXED
    p = B.make_params(f.L, M=32, Q=2, w=w, sigma=sigma, precision=P)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    nb = 30
    k, E = bs.energy_spectrum(torch.from_numpy(f.nodes).cuda(), nb, smoothed=smoothed)
    bs.close()
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    ko, Eo = oracle.energy_spectrum(g, f.L, KAPPA, (p.M[0] - 1) // 2, nb, alpha=p.alpha if smoothed else None)
    assert np.allclose(k, ko, rtol=1e-15)
    assert Eo.max() > 0
    err = np.abs(E - Eo).max() / Eo.max()
    assert err < tol, err


def test_spectrum_of_lines_and_argument_errors():
    B = _B()
    f = W.antiparallel_lines(N_l=32)
    p = B.make_params(f.L, M=49, Q=2, w=8, precision=B.BS_FP64)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    nodes = torch.from_numpy(f.nodes).cuda()
    k, E = bs.energy_spectrum(nodes, 40)
    # the corner of the 24-mode cube is shell 42: shells past it stay empty
    assert E[0] == 0.0 and E[6:21].min() > 0
    V = float(np.prod(f.L))
    ratio = E[6:21] * k[6:21] / (KAPPA ** 2 * 2 * f.L[0] / (4 * math.pi * V))
    assert abs(ratio.mean() - 1.0) < 0.05
    with pytest.raises(B.BSError) as e:
        B.bs_energy_spectrum(bs.ctx, nodes, 0)
    assert e.value.code == B.BS_ERR_ARG
    bs.close()
    pc = B.make_params(f.L, M=32, Q=2, w=8, precision=B.BS_FP64, flags=B.BS_FFT_CUFFT)
    bc = B.BiotSavart(pc, f.offsets, f.closing)
    with pytest.raises(B.BSError) as e:
        bc.energy_spectrum(nodes, 10)
    assert e.value.code == B.BS_ERR_STATE
    bc.close()


@pytest.mark.parametrize("prec,w,sigma,tol", [("fp64", 16, 2.0, 1e-10), ("mixed", 8, 1.5, 1e-5)])
def test_coarse_velocity_on_the_grid_matches_fourier_sum(prec, w, sigma, tol):
    """The coarse-grained (long-range) velocity written on the spread grid
    equals the oracle's direct Fourier sum of v^(f) evaluated at those grid
    points (sampled), relative to the field's largest value."""
    import dataclasses
    B = _B()
    f = W.ellipses(nfil=6, N_l=24, seed=17)
    P = B.BS_FP64 if prec == "fp64" else B.BS_MIXED
    p = B.make_params(f.L, M=32, Q=2, w=w, sigma=sigma, precision=P)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    grid = bs.coarse_velocity(torch.from_numpy(f.nodes).cuda()).cpu().numpy()
    bs.close()
    n0, n1, n2 = grid.shape[1:]
    rng = np.random.default_rng(5)
    pts = np.stack([rng.integers(0, n, 40) for n in (n0, n1, n2)], axis=1)
    X = pts * (f.L / np.array([n0, n1, n2]))[None, :]
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    K = (p.M[0] - 1) // 2
    om = oracle.fourier_coefs(g, f.L, KAPPA, np.array([K] * 3, np.int32))
    ge = dataclasses.replace(g, nodes=np.ascontiguousarray(X))
    vr, _ = oracle.fourier_eval(ge, f.L, p.alpha, np.array([K] * 3, np.int32), om, targets=np.arange(len(X)))
    got = grid[:, pts[:, 0], pts[:, 1], pts[:, 2]].T
    err = np.abs(got - vr).max() / np.abs(grid).max()
    assert err < tol, err
