"""Quintic splines with three quadrature points (``-m gpu``): the paper's
production setting (Sec. 5.2, order 6, Q = 3), against the oracle's
periodic quintic B-spline (Appendix B)."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_07366_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA, A_CORE, DELTA = 1.0, 1e-6, 0.25


def _B():
    import paper_2406_07366_gb300 as B
    return B


def _rms(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1)) / np.mean(np.sum(b ** 2, axis=1))))


def _params(B, f, **kw):
    return B.make_params(f.L, kappa=KAPPA, a=A_CORE, delta=DELTA, order=6, Q=3, **kw)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["trefoil", "ellipses", "lines"])
def test_quintic_quadrature_points_and_charges(case, prec):
    """Quadrature points s(tau_j + h_i dtau_j) and charges w_i dtau_j s'(tau)
    of the GPU's Hermite-form quintic equal the oracle's B-spline ones (the
    periodic C4 quintic through the nodes is unique), closed and unclosed."""
    B = _B()
    f = {"trefoil": lambda: W.trefoil(N=48), "ellipses": lambda: W.ellipses(nfil=5, N_l=20, seed=13),
         "lines": lambda: W.three_line_pairs(N_l=12)}[case]()
    p = _params(B, f, M=32, precision=B.BS_FP64 if prec == "fp64" else B.BS_MIXED)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    qX, qq = bs.quadrature(torch.from_numpy(f.nodes).cuda())
    qX, qq = qX.cpu().numpy(), qq.cpu().numpy()
    bs.close()
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 6, 3)
    tol = 1e-12 if prec == "fp64" else 2e-6
    dX = qX - g.qX
    dX -= f.L[None, :] * np.round(dX / f.L[None, :])
    assert np.abs(dX).max() < tol * max(1.0, np.abs(f.nodes).max())
    assert np.abs(qq - g.qq).max() < 10 * tol * np.abs(g.qq).max()


def test_quintic_total_is_implementation_parity():
    """beta = 8, w = 16, sigma = 2: the GPU total with the quintic curve
    equals the converged oracle on the same quintic curve."""
    B = _B()
    f = W.ellipses(nfil=4, N_l=24, seed=5)
    L = f.L[0]
    beta = 8.0
    alpha = 2 * beta / L
    K = int(math.ceil(beta * alpha * L / math.pi))
    p = _params(B, f, M=2 * K + 1, w=16, sigma=2.0, precision=B.BS_FP64, beta=beta, alpha=alpha,
                flags=B.BS_WANT_PSI)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    v, psi = bs.velocity(torch.from_numpy(f.nodes).cuda(), want_psi=True)
    v, psi = v.cpu().numpy(), psi.cpu().numpy()
    bs.close()
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 6, 3)
    vr, pr = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    assert _rms(v, vr) < 1e-10
    assert _rms(psi, pr) < 1e-10


def test_quintic_trefoil_mixed_and_energy():
    """The mixed form with quintic curves stays in the float32 budget on the
    trefoil.  The energy of a quintic curve (Eq. kinetic_energy_streamfunction;
    the line integral interpolates psi . sdot by the periodic quintic on the
    curve's knots) equals the oracle's at the same split: to 1e-10 at w = 16,
    sigma = 2, to 1e-6 at w = 8 and to 1e-5 in the mixed form."""
    B = _B()
    f = W.trefoil(N=96)
    p = _params(B, f, M=48, w=8, precision=B.BS_MIXED)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    nodes = torch.from_numpy(f.nodes).cuda()
    v = bs.velocity(nodes).cpu().numpy()
    bs.close()
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 6, 3)
    vr, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    assert _rms(v, vr) < 1e-5
    for prec, w, sigma, tol in ((B.BS_FP64, 16, 2.0, 1e-10), (B.BS_FP64, 8, 1.5, 1e-6), (B.BS_MIXED, 8, 1.5, 1e-5)):
        pe = _params(B, f, M=48, w=w, sigma=sigma, precision=prec, flags=B.BS_WANT_PSI)
        be = B.BiotSavart(pe, f.offsets, f.closing)
        E = be.energy(nodes)
        be.close()
        Em = oracle.energy(g, f.L, KAPPA, A_CORE, DELTA, pe.alpha, pe.rc, (pe.M[0] - 1) // 2, order=6)
        assert abs(E - Em) < tol * abs(Em), (prec, w, E, Em)


def _spline_impulse(bs, nodes, L, Q):
    """p = (kappa/2) oint s x ds (Sec. 5.2) on the spline curve: the sum over
    the quadrature points of s_q x q_q (q = w_i dtau s'), every point taken
    at the image nearest its node (the points come back wrapped into the box)."""
    qX, qq = bs.quadrature(nodes)
    x = nodes.cpu().numpy()
    qX, qq = qX.cpu().numpy(), qq.cpu().numpy()
    xn = np.repeat(x, Q, axis=0)
    qX = qX - L[None, :] * np.round((qX - xn) / L[None, :])
    return 0.5 * KAPPA * np.cross(qX, qq).sum(axis=0)


def test_leapfrogging_rings_conserve_energy_and_impulse():
    """Sec. 5.2's conservation run in the paper's production setting: two
    leapfrogging elliptical rings of 32 nodes, quintic curves, Q = 3,
    subdivided local segments (f = 0.1), beta = 3.5 with alpha = 7/L, float64,
    RK4 with the Kelvin-wave step.  The energy and impulse are invariants of
    the motion; over 400 steps they move by a few 1e-6 of their size (the paper
    reports variations within 1e-6 over its run), while the rings travel."""
    B = _B()
    f = W.leapfrog_ellipses(N_l=32)
    L = f.L[0]
    alpha = 7.0 / L
    K = int(math.ceil(3.5 * alpha * L / math.pi))
    p = _params(B, f, M=2 * K + 1, w=8, precision=B.BS_FP64, alpha=alpha, flags=B.BS_WANT_PSI, local_frac=0.1)
    nodes = torch.from_numpy(f.nodes.copy()).cuda()
    dmin = min(np.linalg.norm(np.roll(f.nodes[f.offsets[l]:f.offsets[l + 1]], -1, axis=0)
                              - f.nodes[f.offsets[l]:f.offsets[l + 1]], axis=1).min() for l in range(f.nfil))
    dt = B.kelvin_wave_period(dmin, KAPPA, A_CORE, DELTA)
    stream = torch.cuda.Stream()
    bs = B.BiotSavart(p, f.offsets, f.closing, stream=stream)
    with torch.cuda.stream(stream):
        E0 = bs.energy(nodes)
        P0 = _spline_impulse(bs, nodes, f.L, 3)
        Es = [E0]
        for _ in range(4):
            bs.rk4_capture(nodes, dt)
            bs.rk4_launch(100)
            bs.status()
            Es.append(bs.energy(nodes))
        x1 = nodes.cpu().numpy()
        P1 = _spline_impulse(bs, nodes, f.L, 3)
    bs.close()
    dE = max(abs(e - E0) for e in Es) / abs(E0)
    dP = float(np.linalg.norm(P1 - P0) / np.linalg.norm(P0))
    assert np.abs(x1 - f.nodes).max() > 0.05 * L / 32, "the rings must move"
    assert dE < 1e-5, dE
    assert dP < 1e-5, dP


@pytest.mark.parametrize("order", [4, 6])
def test_subdivided_local_segments_match_oracle(order):
    """Sec. 5.2's subdivided local segments (f = 0.1, Q = 3): float64 at
    beta = 8, w = 16, sigma = 2 equals the converged oracle with the same
    subdivision (velocity and streamfunction); the mixed form stays in its
    budget."""
    B = _B()
    f = W.leapfrog_ellipses(N_l=32)
    L = f.L[0]
    beta = 8.0
    alpha = 2 * beta / L
    K = int(math.ceil(beta * alpha * L / math.pi))
    p = B.make_params(f.L, kappa=KAPPA, a=A_CORE, delta=DELTA, order=order, Q=3, M=2 * K + 1, w=16, sigma=2.0,
                      precision=B.BS_FP64, beta=beta, alpha=alpha, flags=B.BS_WANT_PSI, local_frac=0.1)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    nodes = torch.from_numpy(f.nodes).cuda()
    v, psi = bs.velocity(nodes, want_psi=True)
    v, psi = v.cpu().numpy(), psi.cpu().numpy()
    bs.close()
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, order, 3)
    vr, pr = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA, local_frac=0.1, order=order)
    assert _rms(v, vr) < 1e-10
    assert _rms(psi, pr) < 1e-10
    pm = B.make_params(f.L, kappa=KAPPA, a=A_CORE, delta=DELTA, order=order, Q=3, M=32, w=8,
                       precision=B.BS_MIXED, local_frac=0.1)
    bm = B.BiotSavart(pm, f.offsets, f.closing)
    vm = bm.velocity(nodes).cpu().numpy()
    bm.close()
    vr2, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA, local_frac=0.1, order=order)
    assert _rms(vm, vr2) < 1e-5
