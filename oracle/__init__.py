"""FP64 CPU oracle for the Ewald-split periodic Biot-Savart velocity.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library in ``paper_2406_07366_gb300``.

The arithmetic lives in ``bs_oracle.c`` (plain C, OpenMP over targets);
this module only compiles it, marshals numpy arrays through ctypes and adds
the four parts of the Ewald split (Sec. 3, Eq. ewald_velocity_splitting):

    v = v_local + v^(n) + v^(f) - v^(f)_self

Two modes:
  * ``velocity_converged``: the quadrature-discretised periodic sum itself,
    evaluated with the oracle's own split (beta_o = 6, alpha_o = beta_o/L,
    all 27 images in real space, direct Fourier sum with K_o per axis); the
    result does not depend on any parameter of the fast method.
  * ``components_matched``: each part at the fast method's own alpha, r_c and
    mode cube, for part-by-part parity.

Parity unpinned: nothing here.  Every function has a pin in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile bs_oracle.c into liboracle.so (gcc, OpenMP, strict IEEE)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.or_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
        lib.or_gauss_legendre.restype = ctypes.c_int
        lib.or_spline_eval.argtypes = [ctypes.c_long, _dp, _dp, ctypes.c_int, ctypes.c_long, _dp, ctypes.c_int,
                                       _dp, _dp, _dp]
        lib.or_spline_eval.restype = ctypes.c_int
        lib.or_geometry.argtypes = [ctypes.c_long, _i64p, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                    _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.or_geometry.restype = ctypes.c_int
        lib.or_local.argtypes = [ctypes.c_long, _dp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, _dp, _dp]
        lib.or_local.restype = None
        lib.or_local_sub.argtypes = [ctypes.c_long, _i64p, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
        lib.or_local_sub.restype = ctypes.c_int
        lib.or_short_range.argtypes = [ctypes.c_long, _i64p, _dp, _i64p, _i64p, _dp, ctypes.c_long, ctypes.c_int,
                                       _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, _dp, _dp]
        lib.or_short_range.restype = None
        lib.or_long_range.argtypes = [ctypes.c_long, _i64p, _dp, ctypes.c_long, _dp, _dp, _dp, ctypes.c_double,
                                      ctypes.c_double, _ip, _dp, _dp, _dp]
        lib.or_long_range.restype = None
        lib.or_fourier_coefs.argtypes = [ctypes.c_long, _dp, _dp, _dp, ctypes.c_double, _ip, _dp]
        lib.or_fourier_coefs.restype = None
        lib.or_fourier_eval.argtypes = [ctypes.c_long, _i64p, _dp, _dp, ctypes.c_double, _ip, _dp, _dp, _dp]
        lib.or_fourier_eval.restype = None
        lib.or_energy_fourier.argtypes = [_dp, _ip, _dp, ctypes.c_double]
        lib.or_energy_fourier.restype = ctypes.c_double
        lib.or_energy_line.argtypes = [ctypes.c_long, _i64p, _dp, _dp, ctypes.c_int, _dp]
        lib.or_energy_line.restype = ctypes.c_double
        lib.or_self.argtypes = [ctypes.c_long, _i64p, _dp, _i64p, _i64p, _dp, ctypes.c_int, _dp, _dp,
                                ctypes.c_double, ctypes.c_double, _dp, _dp]
        lib.or_self.restype = None
        lib.or_open_space.argtypes = [ctypes.c_long, _i64p, _dp, _i64p, _i64p, ctypes.c_long, ctypes.c_int,
                                      _dp, _dp, ctypes.c_double, _dp, _dp]
        lib.or_open_space.restype = None
        lib.or_g_far.argtypes = [ctypes.c_double]
        lib.or_g_far.restype = ctypes.c_double
        lib.or_g_near.argtypes = [ctypes.c_double]
        lib.or_g_near.restype = ctypes.c_double
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_get_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def get_threads() -> int:
    return int(_load().or_get_threads())


def gauss_legendre(Q: int):
    """Gauss-Legendre nodes h_i and weights w_i on [0, 1] (Sec. 2.6)."""
    h = np.zeros(Q)
    w = np.zeros(Q)
    if _load().or_gauss_legendre(int(Q), _p(h), _p(w)) != 0:
        raise ValueError("Q out of range")
    return h, w


def g_far(x: float) -> float:
    """g^(f)(x) = erf(x) - 2x/sqrt(pi) exp(-x^2) (Eq. ewald_derivative_weight_functions)."""
    return float(_load().or_g_far(float(x)))


def g_near(x: float) -> float:
    """g^(n)(x) = erfc(x) + 2x/sqrt(pi) exp(-x^2) (Eq. ewald_derivative_weight_functions)."""
    return float(_load().or_g_near(float(x)))


def spline_eval(nodes, shift, order, taus, der=0):
    """Evaluate the oracle's chord-length periodic spline of one filament.

    Returns (values (m x 3), tau_nodes (n), T)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    shift = np.ascontiguousarray(shift, dtype=np.float64)
    taus = np.ascontiguousarray(taus, dtype=np.float64)
    n = nodes.shape[0]
    out = np.zeros((taus.size, 3))
    tau = np.zeros(n)
    T = np.zeros(1)
    rc = _load().or_spline_eval(n, _p(nodes), _p(shift), int(order), taus.size, _p(taus), int(der),
                                _p(out), _p(tau), _p(T))
    if rc != 0:
        raise RuntimeError(f"or_spline_eval failed ({rc})")
    return out, tau, float(T[0])


@dataclass
class Geometry:
    nodes: np.ndarray     # N x 3 unwrapped node positions
    offsets: np.ndarray   # nfil+1
    shift: np.ndarray     # nfil x 3, n_l * L
    fil_of: np.ndarray    # N
    Q: int
    qX: np.ndarray        # N*Q x 3
    qq: np.ndarray        # N*Q x 3
    sp: np.ndarray        # N x 3
    sxs: np.ndarray       # N x 3
    lm: np.ndarray        # N
    lp: np.ndarray        # N
    tau: np.ndarray       # N
    T: np.ndarray         # nfil


def geometry(nodes, offsets, closing, L, order=4, Q=2) -> Geometry:
    """Spline fit, quadrature points/charges and node geometry (Sec. 2.6, App. B)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    L = np.asarray(L, dtype=np.float64)
    nfil = offsets.size - 1
    shift = np.ascontiguousarray(np.asarray(closing, dtype=np.float64).reshape(nfil, 3) * L[None, :])
    N = nodes.shape[0]
    qX = np.zeros((N * Q, 3))
    qq = np.zeros((N * Q, 3))
    sp = np.zeros((N, 3))
    sxs = np.zeros((N, 3))
    lm = np.zeros(N)
    lp = np.zeros(N)
    tau = np.zeros(N)
    T = np.zeros(max(nfil, 1))
    rc = _load().or_geometry(nfil, _p(offsets, _i64p), _p(nodes), _p(shift), int(order), int(Q),
                             _p(qX), _p(qq), _p(sp), _p(sxs), _p(lm), _p(lp), _p(tau), _p(T))
    if rc != 0:
        raise RuntimeError(f"or_geometry failed ({rc})")
    fil_of = np.repeat(np.arange(nfil, dtype=np.int64), np.diff(offsets))
    return Geometry(nodes, offsets, shift, fil_of, Q, qX, qq, sp, sxs, lm, lp, tau, T[:nfil])


def _targets(g: Geometry, targets):
    if targets is None:
        return np.arange(g.nodes.shape[0], dtype=np.int64)
    return np.ascontiguousarray(targets, dtype=np.int64)


def local(g: Geometry, kappa, a, delta, targets=None):
    """v_local and psi_local (Eqs. BS_local, streamfunction_local)."""
    t = _targets(g, targets)
    N = g.nodes.shape[0]
    v = np.zeros((N, 3))
    psi = np.zeros((N, 3))
    _load().or_local(N, _p(g.sp), _p(g.sxs), _p(g.lm), _p(g.lp), kappa, a, delta, _p(v), _p(psi))
    return v[t], psi[t]


def local_subdivided(g: Geometry, kappa, a, delta, frac, order=4):
    """Local terms with the local segments subdivided (Sec. 5.2): Taylor
    expansions on the fraction frac of each local segment next to the node,
    plain Biot-Savart Gauss-Legendre (g.Q points) on the rest.  (N x 3) v, psi."""
    v = np.zeros((g.nodes.shape[0], 3))
    psi = np.zeros((g.nodes.shape[0], 3))
    rc = _load().or_local_sub(g.offsets.size - 1, _p(g.offsets, _i64p), _p(g.nodes), _p(g.shift), int(order),
                              int(g.Q), float(frac), kappa, a, delta, _p(v), _p(psi))
    if rc != 0:
        raise RuntimeError(f"or_local_sub failed ({rc})")
    return v, psi


def short_range(g: Geometry, L, kappa, alpha, rc, all_images=False, targets=None):
    """v^(n), psi^(n) (Eqs. velocity_shortrange, streamfunction_shortrange)."""
    t = _targets(g, targets)
    L = np.asarray(L, dtype=np.float64)
    v = np.zeros((t.size, 3))
    psi = np.zeros((t.size, 3))
    _load().or_short_range(t.size, _p(t, _i64p), _p(g.nodes), _p(g.offsets, _i64p), _p(g.fil_of, _i64p),
                           _p(g.shift), g.qX.shape[0], g.Q, _p(g.qX), _p(g.qq), _p(L), kappa, alpha, rc,
                           1 if all_images else 0, _p(v), _p(psi))
    return v, psi


def long_range(g: Geometry, L, kappa, alpha, K, targets=None, want_omega=False):
    """v^(f), psi^(f) by direct Fourier sum over |m_d| <= K_d (Eq. velocity_longrange_physical)."""
    t = _targets(g, targets)
    L = np.asarray(L, dtype=np.float64)
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.int32), (3,)))
    v = np.zeros((t.size, 3))
    psi = np.zeros((t.size, 3))
    om = np.zeros(((2 * K[0] + 1) * (2 * K[1] + 1) * (2 * K[2] + 1), 3, 2)) if want_omega else None
    _load().or_long_range(t.size, _p(t, _i64p), _p(g.nodes), g.qX.shape[0], _p(g.qX), _p(g.qq), _p(L),
                          kappa, alpha, _p(K, _ip), _p(v), _p(psi), _p(om))
    if want_omega:
        om = om[..., 0] + 1j * om[..., 1]
        return v, psi, om.reshape(2 * K[0] + 1, 2 * K[1] + 1, 2 * K[2] + 1, 3)
    return v, psi


def fourier_coefs(g: Geometry, L, kappa, K):
    """omega_k over the cube |m_d| <= K_d (Eq. vorticity_fourier_coefs), shape (2K+1)^3 x 3 complex."""
    L = np.asarray(L, dtype=np.float64)
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.int32), (3,)))
    om = np.zeros(((2 * K[0] + 1) * (2 * K[1] + 1) * (2 * K[2] + 1), 3, 2))
    _load().or_fourier_coefs(g.qX.shape[0], _p(g.qX), _p(g.qq), _p(L), kappa, _p(K, _ip), _p(om))
    return om


def fourier_eval(g: Geometry, L, alpha, K, om, targets=None):
    """v^(f), psi^(f) at the targets from omega_k of fourier_coefs (Eq. velocity_longrange_physical)."""
    t = _targets(g, targets)
    L = np.asarray(L, dtype=np.float64)
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.int32), (3,)))
    v = np.zeros((t.size, 3))
    psi = np.zeros((t.size, 3))
    _load().or_fourier_eval(t.size, _p(t, _i64p), _p(g.nodes), _p(L), alpha, _p(K, _ip), _p(om), _p(v), _p(psi))
    return v, psi


def self_term(g: Geometry, kappa, alpha, targets=None):
    """v^(f)_self, psi^(f)_self (Eqs. velocity_longrange_self, streamfunction_longrange_self)."""
    t = _targets(g, targets)
    v = np.zeros((t.size, 3))
    psi = np.zeros((t.size, 3))
    _load().or_self(t.size, _p(t, _i64p), _p(g.nodes), _p(g.offsets, _i64p), _p(g.fil_of, _i64p), _p(g.shift),
                    g.Q, _p(g.qX), _p(g.qq), kappa, alpha, _p(v), _p(psi))
    return v, psi


def open_space(g: Geometry, kappa, a, delta, targets=None):
    """Naive open-space sum plus the local term (no periodic images)."""
    t = _targets(g, targets)
    v = np.zeros((t.size, 3))
    psi = np.zeros((t.size, 3))
    _load().or_open_space(t.size, _p(t, _i64p), _p(g.nodes), _p(g.offsets, _i64p), _p(g.fil_of, _i64p),
                          g.qX.shape[0], g.Q, _p(g.qX), _p(g.qq), kappa, _p(v), _p(psi))
    vl, pl = local(g, kappa, a, delta, targets=t)
    return v + vl, psi + pl


def _fsum_rows(parts, signs):
    out = np.zeros_like(parts[0])
    it = np.nditer(out, flags=["multi_index"], op_flags=[["writeonly"]])
    for x in it:
        idx = it.multi_index
        x[...] = math.fsum(s * p[idx] for p, s in zip(parts, signs))
    return out


def energy(g: Geometry, L, kappa, a, delta, alpha, rc, K, all_images=False, order=4):
    """Kinetic energy E = kappa/(2V) oint psi . ds (Eq. kinetic_energy_streamfunction):
    the long-range part as the Fourier reduction (1/2) sum_{k!=0} e^{-k^2/4alpha^2}
    |omega_k|^2/k^2 over the mode cube K, plus kappa/(2V) times the line integral
    of the spline interpolant of (psi_local + psi^(n) - psi^(f)_self) . sdot.
    all_images selects the converged short range (27 images, no cut-off)."""
    L = np.asarray(L, dtype=np.float64)
    Kv = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.int32), (3,)))
    om = fourier_coefs(g, L, kappa, Kv)
    ef = float(_load().or_energy_fourier(_p(om), _p(Kv, _ip), _p(L), alpha))
    _, pl = local(g, kappa, a, delta)
    _, ps = short_range(g, L, kappa, alpha, rc, all_images=all_images)
    _, px = self_term(g, kappa, alpha)
    rest = np.ascontiguousarray(pl + ps - px)
    line = float(_load().or_energy_line(g.offsets.size - 1, _p(g.offsets, _i64p), _p(g.nodes), _p(g.shift),
                                        int(order), _p(rest)))
    V = float(np.prod(L))
    return ef + kappa / (2 * V) * line


def energy_converged(g: Geometry, L, kappa, a, delta, beta_o=6.0, alpha_scale=1.0):
    """The energy with the oracle's own converged split (27 images, mode cube K_o)."""
    alpha, K = converged_params(L, beta_o, alpha_scale)
    return energy(g, L, kappa, a, delta, alpha, 0.0, K, all_images=True)


def converged_params(L, beta_o=6.0, alpha_scale=1.0):
    """alpha_o = beta_o / min(L) (times alpha_scale >= 1), K_o,d = ceil(beta_o alpha_o L_d / pi)."""
    L = np.asarray(L, dtype=np.float64)
    if alpha_scale < 1.0:
        raise ValueError("27 images need alpha >= beta_o / min(L)")
    alpha = alpha_scale * beta_o / L.min()
    K = np.ceil(beta_o * alpha * L / math.pi).astype(np.int32)
    return alpha, K


def velocity_converged(g: Geometry, L, kappa, a, delta, targets=None, beta_o=6.0, alpha_scale=1.0,
                       return_parts=False, local_frac=0.0, order=4):
    """Quadrature-discretised periodic Biot-Savart velocity and streamfunction.

    Evaluated with the oracle's own converged Ewald split (short range over
    all 27 images with no cut-off, long range over the mode cube K_o, self
    and local terms), combined with an exactly rounded sum."""
    alpha, K = converged_params(L, beta_o, alpha_scale)
    if local_frac > 0:
        vl, pl = local_subdivided(g, kappa, a, delta, local_frac, order)
        if targets is not None:
            t = _targets(g, targets)
            vl, pl = vl[t], pl[t]
    else:
        vl, pl = local(g, kappa, a, delta, targets)
    vs, ps = short_range(g, L, kappa, alpha, 0.0, all_images=True, targets=targets)
    vf, pf = long_range(g, L, kappa, alpha, K, targets=targets)
    vx, px = self_term(g, kappa, alpha, targets=targets)
    v = _fsum_rows([vl, vs, vf, vx], [1, 1, 1, -1])
    psi = _fsum_rows([pl, ps, pf, px], [1, 1, 1, -1])
    if return_parts:
        return v, psi, dict(local=vl, short=vs, long=vf, self=vx, psi_local=pl, psi_short=ps, psi_long=pf,
                            psi_self=px, alpha=alpha, K=K)
    return v, psi


def components_matched(g: Geometry, L, kappa, a, delta, alpha, rc, K, targets=None):
    """Each Ewald part at the fast method's own (alpha, r_c, mode cube K)."""
    vl, pl = local(g, kappa, a, delta, targets)
    vs, ps = short_range(g, L, kappa, alpha, rc, all_images=False, targets=targets)
    vf, pf = long_range(g, L, kappa, alpha, K, targets=targets)
    vx, px = self_term(g, kappa, alpha, targets=targets)
    return dict(local=vl, short=vs, long=vf, self=vx, psi_local=pl, psi_short=ps, psi_long=pf, psi_self=px,
                total=_fsum_rows([vl, vs, vf, vx], [1, 1, 1, -1]),
                psi_total=_fsum_rows([pl, ps, pf, px], [1, 1, 1, -1]))


def rk4_converged(nodes, offsets, closing, L, kappa, a, delta, dt, nsteps, order=4, Q=2):
    """Node positions after nsteps classical RK4 steps of ds/dt = v(s)
    (Sec. 5.2), each stage velocity the oracle's converged one (the spline
    refitted at every stage)."""
    x = np.array(nodes, dtype=np.float64, copy=True)

    def v(y):
        g = geometry(y, offsets, closing, L, order, Q)
        return velocity_converged(g, L, kappa, a, delta)[0]

    for _ in range(nsteps):
        k1 = v(x)
        k2 = v(x + 0.5 * dt * k1)
        k3 = v(x + 0.5 * dt * k2)
        k4 = v(x + dt * k3)
        x = x + dt / 6.0 * (k1 + 2.0 * (k2 + k3) + k4)
    return x


def polygon_impulse(nodes, offsets, kappa):
    """Impulse (kappa/2) oint s x ds of the closed polygons through the nodes."""
    P = np.zeros(3)
    for l in range(offsets.size - 1):
        s = nodes[offsets[l]:offsets[l + 1]]
        P += 0.5 * kappa * np.cross(s, np.roll(s, -1, axis=0)).sum(axis=0)
    return P


def energy_spectrum(g: Geometry, L, kappa, K, nbins, alpha=None):
    """Energy spectrum of Eq. def_energy_spectrum: E(k_m) = 1/(2 dk) times the
    sum of |v_k|^2 over the modes with m - 1/2 <= |k| / dk < m + 1/2,
    v_k = i k x omega_k / k^2 over the cube |m_d| <= K_d (k = 0 excluded),
    dk = 2 pi / min L.  With alpha, the long-range field's spectrum
    (|v_k|^2 e^{-k^2 / 2 alpha^2}).  Returns (k_m, E)."""
    L = np.asarray(L, dtype=np.float64)
    Kv = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.int32), (3,)))
    om = fourier_coefs(g, L, kappa, Kv).reshape(2 * Kv[0] + 1, 2 * Kv[1] + 1, 2 * Kv[2] + 1, 3, 2)
    w = om[..., 0] + 1j * om[..., 1]
    k = [2 * math.pi / L[d] * np.arange(-Kv[d], Kv[d] + 1) for d in range(3)]
    kx, ky, kz = np.meshgrid(k[0], k[1], k[2], indexing="ij")
    kv = np.stack([kx, ky, kz], axis=-1)
    ksq = kx ** 2 + ky ** 2 + kz ** 2
    cross = np.cross(kv, w)  # k x omega (complex)
    v2 = np.sum(np.abs(cross) ** 2, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        v2 = np.where(ksq > 0, v2 / ksq ** 2, 0.0)
    if alpha is not None:
        v2 = v2 * np.exp(-ksq / (2 * alpha ** 2))
    dk = 2 * math.pi / L.min()
    m = np.floor(np.sqrt(ksq) / dk + 0.5).astype(np.int64)
    E = np.zeros(int(nbins))
    sel = (ksq > 0) & (m < nbins)
    np.add.at(E, m[sel], v2[sel])
    return dk * np.arange(int(nbins)), E / (2 * dk)
