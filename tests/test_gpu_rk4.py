"""RK4 time stepping through the library (``-m gpu``), Sec. 5.2."""
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


def _dmin(f):
    d = []
    for l in range(f.nfil):
        s = f.nodes[f.offsets[l]:f.offsets[l + 1]]
        d.append(np.linalg.norm(np.roll(s, -1, axis=0) - s, axis=1).min())
    return min(d)


def test_rk4_graph_replay_equals_direct_steps():
    B = _B()
    f = W.fourier_tangle(nfil=20, N_l=32, seed=61, amp=2 * math.pi / 48)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = B.make_params(f.L, M=32, Q=2, w=8, precision=B.BS_FP64)
        bs = B.BiotSavart(p, f.offsets, f.closing, stream=s)
        dt = B.kelvin_wave_period(_dmin(f), KAPPA, A_CORE, DELTA)
        xa = torch.from_numpy(f.nodes).cuda()
        xb = xa.clone()
        for _ in range(3):
            bs.rk4_step(xa, dt)
        bs.rk4_capture(xb, dt)
        bs.rk4_launch(3)
        bs.status()
        assert not torch.equal(xa, torch.from_numpy(f.nodes).cuda())
        scale = (xa - torch.from_numpy(f.nodes).cuda()).abs().max().item()
        assert (xa - xb).abs().max().item() < 1e-12 * scale
        bs.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rk4_trajectory_matches_oracle(prec):
    """Leapfrogging ellipses, 20 Kelvin-wave steps: the GPU trajectory follows
    the oracle's (converged velocities, same RK4 steps) to the method's beta =
    3.5 accuracy times the distance travelled."""
    B = _B()
    f = W.leapfrog_ellipses(N_l=64)
    dt = B.kelvin_wave_period(_dmin(f), KAPPA, A_CORE, DELTA)
    n = 20
    ref = oracle.rk4_converged(f.nodes, f.offsets, f.closing, f.L, KAPPA, A_CORE, DELTA, dt, n)
    P = B.BS_FP64 if prec == "fp64" else B.BS_MIXED
    p = B.make_params(f.L, M=32, Q=2, w=8, precision=P)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bs = B.BiotSavart(p, f.offsets, f.closing, stream=s)
        x = torch.from_numpy(f.nodes).cuda()
        bs.rk4_capture(x, dt)
        bs.rk4_launch(n)
        bs.status()
        got = x.cpu().numpy()
        bs.close()
    travel = np.linalg.norm(ref - f.nodes, axis=1).max()
    assert travel > 1e-2
    err = np.linalg.norm(got - ref, axis=1).max() / travel
    assert err < (2e-5 if prec == "fp64" else 1e-4), err


def test_rk4_ring_translates_rigidly():
    """Config-1 ring: it travels along its axis at about the Kelvin speed
    (Eq. vortex_ring_velocity).  The periodic images form a cubic lattice, so
    the ring keeps only a four-fold symmetry and its node speeds differ by
    ~3e-5 (in the oracle as on the GPU): the motion is a translation up to
    that slow deformation.  The mean displacement over n steps matches n dt
    times the oracle's mean velocity to the method's beta = 3.5 accuracy;
    per node, and for the radius and the energy, the departures stay at the
    size of that deformation."""
    B = _B()
    f = W.ring(N=64)
    p = B.make_params(f.L, M=32, Q=2, w=8, precision=B.BS_FP64, flags=B.BS_WANT_PSI)
    s = torch.cuda.Stream()
    dt = B.kelvin_wave_period(_dmin(f), KAPPA, A_CORE, DELTA)
    n = 25
    with torch.cuda.stream(s):
        bs = B.BiotSavart(p, f.offsets, f.closing, stream=s)
        x = torch.from_numpy(f.nodes).cuda()
        v0 = bs.velocity(x).cpu().numpy()
        e0 = bs.energy(x)
        bs.rk4_capture(x, dt)
        bs.rk4_launch(n)
        bs.status()
        e1 = bs.energy(x)
        got = x.cpu().numpy()
        bs.close()
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    vo, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    vz = vo[:, 2].mean()
    # the oracle keeps the four-fold symmetry of the ring in the cubic lattice
    assert np.abs(vo[:, 2] - np.roll(vo[:, 2], 16)).max() < 1e-12 * abs(vz)
    dist = n * dt * abs(vz)
    assert dist > 0.05  # about 40% of a grid cell
    disp = got - f.nodes
    assert abs(disp[:, 2].mean() - n * dt * vz) < 1e-5 * dist
    assert np.abs(disp[:, 2] - n * dt * v0[:, 2]).max() < 5e-5 * dist
    r0 = np.linalg.norm(f.nodes[:, :2] - f.L[:2] / 2, axis=1)
    r1 = np.linalg.norm(got[:, :2] - f.L[:2] / 2, axis=1)
    assert np.abs(r1 - r0).max() < 5e-5 * dist
    assert abs(e1 - e0) < 1e-5 * abs(e0)


def test_rk4_quintic_leapfrog_matches_oracle():
    """The paper's setting for the leapfrogging test (Sec. 5.2): quintic
    curves, Q = 3.  The GPU trajectory follows the oracle's on the same
    quintic curves, and the impulse is kept to the discretisation level."""
    B = _B()
    f = W.leapfrog_ellipses(N_l=48)
    dt = B.kelvin_wave_period(_dmin(f), KAPPA, A_CORE, DELTA)
    n = 10
    ref = oracle.rk4_converged(f.nodes, f.offsets, f.closing, f.L, KAPPA, A_CORE, DELTA, dt, n, order=6, Q=3)
    p = B.make_params(f.L, M=32, Q=3, order=6, w=8, precision=B.BS_FP64)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bs = B.BiotSavart(p, f.offsets, f.closing, stream=s)
        x = torch.from_numpy(f.nodes).cuda()
        bs.rk4_capture(x, dt)
        bs.rk4_launch(n)
        bs.status()
        got = x.cpu().numpy()
        bs.close()
    travel = np.linalg.norm(ref - f.nodes, axis=1).max()
    assert travel > 1e-3
    assert np.linalg.norm(got - ref, axis=1).max() / travel < 2e-5
    P0 = oracle.polygon_impulse(f.nodes, f.offsets, KAPPA)
    P1 = oracle.polygon_impulse(got, f.offsets, KAPPA)
    assert np.linalg.norm(P1 - P0) / np.linalg.norm(P0) < 1e-5
