"""Seeded synthetic filament sets.

This module only draws node positions; it holds none of the method's
arithmetic and is the one module that both the CUDA path's callers and the
oracle-based tests import.  Every generator returns a ``Filaments`` record:

    nodes    (N, 3) float64   unwrapped node positions, filament after filament
    offsets  (nfil+1,) int64  filament l owns nodes offsets[l]:offsets[l+1]
    closing  (nfil, 3) int32  n_l with s(tau + T) = s(tau) + n_l * L
                              (zero for closed curves, Sec. 2.1)
    L        (3,) float64     box periods

Shapes follow the paper's workloads: a circular ring (Eq.
vortex_ring_velocity), random ellipses (Sec. 5.1 case 3), straight periodic
lines (Sec. 5.1 case 2), the trefoil knot (Eq. def_trefoil_knot), and
random-phase Fourier tangles standing in for a turbulent tangle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Filaments:
    nodes: np.ndarray
    offsets: np.ndarray
    closing: np.ndarray
    L: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def nfil(self) -> int:
        return int(self.offsets.size - 1)


def _pack(curves, L, closing=None, name="", meta=None) -> Filaments:
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)).copy()
    counts = [c.shape[0] for c in curves]
    offsets = np.zeros(len(curves) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    nodes = np.ascontiguousarray(np.concatenate(curves, axis=0) if curves else np.zeros((0, 3)), dtype=np.float64)
    if closing is None:
        closing = np.zeros((len(curves), 3), dtype=np.int32)
    closing = np.ascontiguousarray(np.asarray(closing, dtype=np.int32).reshape(len(curves), 3))
    return Filaments(nodes, offsets, closing, L, name, meta or {})


def ring(R=math.pi / 3, N=64, L=2 * math.pi, center=None, axis=2, phase=0.0) -> Filaments:
    """Circle of radius R in the plane normal to ``axis``, N equispaced nodes,
    counter-clockwise about +axis.  Default: centred in the box."""
    L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    c = L3 / 2 if center is None else np.asarray(center, dtype=np.float64)
    th = 2 * math.pi * np.arange(N) / N + phase
    a, b = [(axis + 1) % 3, (axis + 2) % 3]
    X = np.zeros((N, 3))
    X[:, a] = R * np.cos(th)
    X[:, b] = R * np.sin(th)
    X += c[None, :]
    return _pack([X], L3, name=f"ring(R={R:.4g},N={N})")


def _random_rotation(rng):
    """Uniform rotation on SO(3) from a normalised 4-D Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def ellipses(nfil=40, N_l=64, L=2 * math.pi, seed=2, semi=(0.5, 1.5)) -> Filaments:
    """Closed ellipses: centres U[0,L)^3, orientations uniform on SO(3),
    semi-axes U[semi], N_l nodes equispaced in angle."""
    rng = np.random.default_rng(seed)
    L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    curves = []
    th = 2 * math.pi * np.arange(N_l) / N_l
    for _ in range(nfil):
        c = rng.uniform(0, 1, 3) * L3
        Rm = _random_rotation(rng)
        a, b = rng.uniform(semi[0], semi[1], 2)
        loc = np.stack([a * np.cos(th), b * np.sin(th), np.zeros_like(th)], axis=1)
        curves.append(c[None, :] + loc @ Rm.T)
    return _pack(curves, L3, name=f"ellipses({nfil}x{N_l})")


def fourier_tangle(nfil=1000, N_l=100, L=2 * math.pi, seed=3, modes=8, amp=None) -> Filaments:
    """Random-phase Fourier closed curves,
    s(theta) = c + sum_{m=1}^{modes} (A/m)(u_m cos m theta + v_m sin m theta),
    u_m, v_m ~ N(0, I_3), c ~ U[0,L)^3, A = L/128 by default."""
    rng = np.random.default_rng(seed)
    L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    A = L3.min() / 128 if amp is None else amp
    th = 2 * math.pi * np.arange(N_l) / N_l
    m = np.arange(1, modes + 1)
    cos_t = np.cos(np.outer(th, m))  # N_l x modes
    sin_t = np.sin(np.outer(th, m))
    c = rng.uniform(0, 1, (nfil, 3)) * L3[None, :]
    u = rng.standard_normal((nfil, modes, 3)) * (A / m)[None, :, None]
    v = rng.standard_normal((nfil, modes, 3)) * (A / m)[None, :, None]
    X = c[:, None, :] + np.einsum("tm,fmc->ftc", cos_t, u) + np.einsum("tm,fmc->ftc", sin_t, v)
    return _pack(list(X), L3, name=f"tangle({nfil}x{N_l})")


def antiparallel_lines(N_l=16, L=2 * math.pi, offset=(0.0, 0.0)) -> Filaments:
    """Two straight lines along z through (x0, y0) (+z) and (x0+L/2, y0+L/2)
    (-z).  Every lattice site is a centre of point symmetry."""
    L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    z = L3[2] * np.arange(N_l) / N_l
    x0, y0 = offset
    a = np.stack([np.full(N_l, x0), np.full(N_l, y0), z], axis=1)
    b = np.stack([np.full(N_l, x0 + L3[0] / 2), np.full(N_l, y0 + L3[1] / 2), L3[2] - z], axis=1)
    return _pack([a, b], L3, closing=[[0, 0, 1], [0, 0, -1]], name="antiparallel_lines")


def three_line_pairs(N_l=16, L=2 * math.pi) -> Filaments:
    """Three pairs of straight periodic lines, one pair per axis, each pair
    antiparallel, placed so that every line carries a velocity along itself
    (after Sec. 5.1 case 2)."""
    L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    t = np.arange(N_l) / N_l
    q = 0.25
    curves, closing = [], []
    for ax in range(3):
        a1, a2 = (ax + 1) % 3, (ax + 2) % 3
        for sgn, (p1, p2) in ((+1, (q, 3 * q)), (-1, (3 * q, q))):
            X = np.zeros((N_l, 3))
            X[:, ax] = L3[ax] * (t if sgn > 0 else 1 - t)
            X[:, a1] = p1 * L3[a1]
            X[:, a2] = p2 * L3[a2]
            curves.append(X)
            n = [0, 0, 0]
            n[ax] = sgn
            closing.append(n)
    return _pack(curves, L3, closing=closing, name="three_line_pairs")


def trefoil(R=None, N=512, L=2 * math.pi, center=None) -> Filaments:
    """Trefoil knot X(theta) = R [sin t + 2 sin 2t, cos t - 2 cos 2t, -sin 3t],
    N equispaced values of theta (Eq. def_trefoil_knot)."""
    L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    R = L3.min() / 6 if R is None else R
    c = L3 / 2 if center is None else np.asarray(center, dtype=np.float64)
    th = 2 * math.pi * np.arange(N) / N
    X = R * np.stack([np.sin(th) + 2 * np.sin(2 * th), np.cos(th) - 2 * np.cos(2 * th), -np.sin(3 * th)], axis=1)
    return _pack([X + c[None, :]], L3, name=f"trefoil(N={N})")


def leapfrog_ellipses(N_l=32, L=2 * math.pi) -> Filaments:
    """Two coaxial elliptical rings normal to x at distance L/4, radii
    R_a = L/4 and R_b = sqrt(2) R_a, major axes along y and z (Sec. 5.2)."""
    L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    Ra = L3[0] / 4
    Rb = Ra * math.sqrt(2)
    th = 2 * math.pi * np.arange(N_l) / N_l
    c = L3 / 2
    e1 = np.stack([np.full(N_l, c[0] - L3[0] / 8), c[1] + Rb * np.cos(th), c[2] + Ra * np.sin(th)], axis=1)
    e2 = np.stack([np.full(N_l, c[0] + L3[0] / 8), c[1] + Ra * np.cos(th), c[2] + Rb * np.sin(th)], axis=1)
    return _pack([e1, e2], L3, name="leapfrog_ellipses")


def tangle_batch(nconf=64, seed=5, lo=3.0, hi=5.0, N_l=100, L=2 * math.pi):
    """Independent Fourier tangles with node counts log-uniform in
    [10^lo, 10^hi], N_l nodes per filament (one child seed per member)."""
    ss = np.random.SeedSequence(seed)
    kids = ss.spawn(nconf)
    out = []
    for k in kids:
        rng = np.random.default_rng(k)
        n = int(round(10 ** rng.uniform(lo, hi)))
        nfil = max(2, int(round(n / N_l)))
        out.append(fourier_tangle(nfil=nfil, N_l=N_l, L=L, seed=int(rng.integers(0, 2**31))))
    return out


# Fixed problem settings of the five workloads (the paper's notation):
# L box period, kappa circulation, a core radius, delta core parameter,
# beta accuracy coefficient, M resolved modes per axis, Q quadrature points
# per segment, order spline order (4 = cubic), sigma / w NUFFT oversampling
# and kernel width.
WORKLOADS = {
    "ring64": dict(gen=lambda: ring(), kappa=1.0, a=1e-6, delta=0.25, beta=3.5, M=32, Q=2, order=4,
                   sigma=1.5, w=8),
    "ellipses40": dict(gen=lambda: ellipses(), kappa=1.0, a=1e-6, delta=0.25, beta=3.5, M=64, Q=3, order=4,
                       sigma=1.5, w=8),
    "tangle1e5": dict(gen=lambda: fourier_tangle(1000, 100, seed=3), kappa=1.0, a=1e-6, delta=0.25, beta=3.5,
                      M=256, Q=2, order=4, sigma=1.5, w=8),
    "tangle4e6": dict(gen=lambda: fourier_tangle(20000, 200, seed=4), kappa=1.0, a=1e-6, delta=0.25, beta=3.5,
                      M=512, Q=2, order=4, sigma=1.5, w=8),
}
