"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to a library routine, a closed form, an
invariant or brute force, chosen so that a dropped term, a wrong sign or
index, or a transposed operand in ``oracle/bs_oracle.c`` fails at least one.
All CPU-only (``-m "not gpu"``).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2406_07366_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
KAPPA, A_CORE, DELTA = 1.0, 1e-6, 0.25


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("Q", list(range(1, 11)))
def test_gauss_legendre_matches_numpy(Q):
    """Sec. 2.6: rule on [0,1] with sum w = 1 is numpy's leggauss mapped."""
    h, w = oracle.gauss_legendre(Q)
    x, wx = np.polynomial.legendre.leggauss(Q)
    np.testing.assert_allclose(h, (x + 1) / 2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, wx / 2, rtol=0, atol=1e-15)
    assert abs(w.sum() - 1) < 1e-15


# ---------------------------------------------------------------- splines
def _random_closed_curve(n, seed):
    rng = np.random.default_rng(seed)
    th = np.sort(rng.uniform(0, 2 * np.pi, n))
    r = 1 + 0.3 * np.cos(3 * th)
    return np.stack([r * np.cos(th), r * np.sin(th), 0.4 * np.sin(2 * th)], axis=1) + 3.0


def test_cubic_spline_matches_scipy_periodic():
    """App. B: the order-4 periodic B-spline interpolant with knots at the
    chord-length parameters is the periodic C2 cubic that scipy builds."""
    from scipy.interpolate import CubicSpline
    X = _random_closed_curve(23, 1)
    shift = np.zeros(3)
    xs = np.random.default_rng(5).uniform(-1, 30, 200)
    for der in range(3):
        val, tau, T = oracle.spline_eval(X, shift, 4, xs, der)
        cs = CubicSpline(np.append(tau, T), np.vstack([X, X[:1]]), bc_type="periodic")
        ref = cs(np.mod(xs, T), der)
        np.testing.assert_allclose(val, ref, rtol=0, atol=1e-11 * max(1, np.abs(ref).max()))


def test_quintic_spline_matches_scipy_periodic():
    """App. B: order-6 (quintic) periodic interpolant equals scipy's periodic k=5 spline."""
    from scipy.interpolate import make_interp_spline
    X = _random_closed_curve(19, 2)
    shift = np.zeros(3)
    xs = np.random.default_rng(6).uniform(0, 20, 150)
    for der in range(4):
        val, tau, T = oracle.spline_eval(X, shift, 6, xs, der)
        sp = make_interp_spline(np.append(tau, T), np.vstack([X, X[:1]]), k=5, bc_type="periodic")
        ref = sp(np.mod(xs, T), der)
        np.testing.assert_allclose(val, ref, rtol=0, atol=1e-9 * max(1, np.abs(ref).max()))


def test_unclosed_curve_periodic_part():
    """Sec. 2.1 / reading on unclosed curves: a helix s(tau+T) = s(tau) + L e_z
    is interpolated through s - n L tau / T; scipy on that periodic part plus
    the linear drift must agree."""
    from scipy.interpolate import CubicSpline
    L = 2 * np.pi
    n = 17
    th = 2 * np.pi * np.arange(n) / n + 0.1 * np.sin(np.arange(n))
    X = np.stack([1 + 0.5 * np.cos(th), 1 + 0.5 * np.sin(th), L * th / (2 * np.pi)], axis=1)
    shift = np.array([0, 0, L])
    xs = np.linspace(0.01, 10, 77)
    val, tau, T = oracle.spline_eval(X, shift, 4, xs, 0)
    P = X - shift[None, :] * tau[:, None] / T
    cs = CubicSpline(np.append(tau, T), np.vstack([P, P[:1]]), bc_type="periodic")
    xr = np.mod(xs, T)
    ref = cs(xr) + shift[None, :] * (xs / T)[:, None]
    np.testing.assert_allclose(val, ref, atol=1e-11)
    # a straight periodic line is reproduced exactly
    z = L * np.arange(8) / 8
    Xl = np.stack([np.full(8, 1.0), np.full(8, 2.0), z], axis=1)
    v, tau, T = oracle.spline_eval(Xl, shift, 4, np.linspace(0, 2 * L, 31), 0)
    np.testing.assert_allclose(v[:, :2], [[1.0, 2.0]] * 31, atol=1e-13)
    np.testing.assert_allclose(v[:, 2], np.linspace(0, 2 * L, 31), atol=1e-12)


# ---------------------------------------------------------------- quadrature geometry
@pytest.mark.parametrize("order,Q", [(4, 2), (4, 3), (6, 3)])
def test_net_charge_of_closed_curves_vanishes(order, Q):
    """Sec. 2.2: sum of q over a closed curve is the integral of ds = 0; GL
    with 2Q-1 >= order-2 integrates the spline derivative exactly."""
    f = W.ellipses(nfil=5, N_l=20, seed=11)
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, order, Q)
    for l in range(f.nfil):
        sl = slice(f.offsets[l] * Q, f.offsets[l + 1] * Q)
        s = g.qq[sl].sum(0)
        assert np.abs(s).max() < 1e-14 * np.abs(g.qq[sl]).sum()


def test_net_charge_of_unclosed_lines_is_nL():
    f = W.three_line_pairs(N_l=12)
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    for l in range(f.nfil):
        s = g.qq[f.offsets[l] * 2:f.offsets[l + 1] * 2].sum(0)
        np.testing.assert_allclose(s, f.closing[l] * f.L, atol=1e-13)


def test_circle_length_and_curvature_converge():
    """Arc length -> 2 pi R and s' x s'' -> e_z / R (Sec. 2.3) as N grows, at
    the rates of cubic interpolation: O(h^4) for length, O(h^2) for
    the second derivative."""
    R = 1.3
    errs_len, errs_k = [], []
    for N in (16, 32, 64):
        f = W.ring(R=R, N=N)
        g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 3)
        errs_len.append(abs(g.lp.sum() - 2 * np.pi * R))
        errs_k.append(np.abs(g.sxs - np.array([0, 0, 1 / R])).max())
        np.testing.assert_allclose(np.linalg.norm(g.sp, axis=1), 1, atol=1e-14)
    assert errs_len[1] < errs_len[0] / 10 and errs_len[2] < errs_len[1] / 10
    assert errs_k[1] < errs_k[0] / 3 and errs_k[2] < errs_k[1] / 3
    assert errs_k[2] < 1e-3


# ---------------------------------------------------------------- weight functions
def test_weight_functions_against_mpmath():
    """Eq. ewald_derivative_weight_functions at 40 digits, including the small-x
    series branch of g^(f) where erf and the Gaussian term cancel."""
    import mpmath
    mpmath.mp.dps = 40
    for x in [1e-6, 1e-3, 0.05, 0.2, 0.4999, 0.5, 0.7, 1.0, 2.0, 4.0]:
        xm = mpmath.mpf(x)
        gf = mpmath.erf(xm) - 2 * xm / mpmath.sqrt(mpmath.pi) * mpmath.exp(-xm * xm)
        gn = mpmath.erfc(xm) + 2 * xm / mpmath.sqrt(mpmath.pi) * mpmath.exp(-xm * xm)
        assert abs(oracle.g_far(x) - float(gf)) <= 1e-15 * float(gf) + 1e-300
        assert abs(oracle.g_near(x) - float(gn)) <= 1e-15 * float(gn)
    # Sec. 3.1 small-r limit of grad G^(f): g^(f)(x)/x^3 -> 4/(3 sqrt(pi))
    lim = GOLD["kernel_limits"]["gf_over_x3_at_0"]
    assert abs(oracle.g_far(1e-4) / 1e-12 - lim) < 1e-7


# ---------------------------------------------------------------- whole sums
def _geom(f, order=4, Q=2):
    return oracle.geometry(f.nodes, f.offsets, f.closing, f.L, order, Q)


@pytest.mark.parametrize("case", ["ring", "ellipses", "lines", "trefoil"])
def test_total_is_independent_of_alpha(case):
    """Sec. 3.1: the physical fields do not depend on alpha.  Changing alpha
    moves weight between short range, long range and self term; any error in
    one of them (normalisation, Gaussian filter, curl sign, 1/k^2, the C_0
    bookkeeping) breaks the agreement."""
    f = {"ring": lambda: W.ring(N=32),
         "ellipses": lambda: W.ellipses(nfil=3, N_l=24, seed=7),
         "lines": lambda: W.three_line_pairs(N_l=12),
         "trefoil": lambda: W.trefoil(N=48)}[case]()
    g = _geom(f)
    v1, p1 = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA, alpha_scale=1.0)
    v2, p2 = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA, alpha_scale=1.6)
    sv, sp = np.abs(v1).max(), np.abs(p1).max()
    assert np.abs(v1 - v2).max() < 1e-13 * sv
    assert np.abs(p1 - p2).max() < 1e-13 * sp


def test_alpha_zero_short_range_is_plain_biot_savart():
    """Sec. 3.2: alpha = 0 recovers the original integrals.  For a ring far
    smaller than L/2 the minimum-image sum with r_c = L/2 holds every source."""
    f = W.ring(R=0.6, N=40)
    g = _geom(f)
    vs, ps = oracle.short_range(g, f.L, KAPPA, 0.0, f.L[0] / 2)
    vo, po = oracle.open_space(g, KAPPA, A_CORE, DELTA)
    vl, pl = oracle.local(g, KAPPA, A_CORE, DELTA)
    np.testing.assert_allclose(vs, vo - vl, rtol=0, atol=1e-14 * np.abs(vs).max())
    np.testing.assert_allclose(ps, po - pl, rtol=0, atol=1e-14 * np.abs(ps).max())


def test_periodic_sum_tends_to_open_space_as_box_grows():
    """A fixed ring in boxes L = 2 pi, 4 pi, 8 pi: the periodic images and the
    zero-mean condition perturb the open-space velocity by O((R/L)^3)."""
    diffs = []
    for L in (2 * np.pi, 4 * np.pi, 8 * np.pi):
        f = W.ring(R=np.pi / 3, N=32, L=L)
        g = _geom(f)
        v, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
        vo, _ = oracle.open_space(g, KAPPA, A_CORE, DELTA)
        diffs.append(np.abs(v - vo).max())
    r1, r2 = diffs[0] / diffs[1], diffs[1] / diffs[2]
    assert 5 < r1 < 11 and 6 < r2 < 10, diffs


def test_kelvin_ring_speed_convergence():
    """Eq. vortex_ring_velocity: the open-space ring speed approaches
    kappa/(4 pi R)[ln(8R/a) - Delta] as N grows (the paper prints no
    tolerance: convergence only), and all nodes move alike."""
    k = GOLD["kelvin_ring"]
    errs = []
    for N in (16, 32, 64):
        f = W.ring(R=k["R"], N=N, L=64.0)
        g = _geom(f, 4, 3)
        vo, _ = oracle.open_space(g, k["kappa"], k["a"], k["delta"])
        errs.append(np.abs(vo[:, 2] - k["V"]).max() / k["V"])
        # roundoff of near-neighbour terms (~1/l^2) grows like N^2
        assert np.abs(vo[:, :2]).max() < 1e-10
        assert np.ptp(vo[:, 2]) < 1e-10
    # the local term's Taylor error is O(l^2): the error falls ~4x per doubling
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3 and errs[2] < 1e-3, errs


def test_periodic_ring_four_fold_symmetry():
    """A ring centred in a cube about e_z: nodes a quarter turn apart have
    equal axial speed and in-plane velocities rotated by 90 degrees."""
    f = W.ring(N=64)
    g = _geom(f)
    v, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    vr = np.roll(v, -16, axis=0)
    # node positions carry cos/sin rounding (~1e-16 R), amplified by the sums
    np.testing.assert_allclose(vr[:, 2], v[:, 2], rtol=0, atol=5e-12)
    np.testing.assert_allclose(vr[:, 0], -v[:, 1], rtol=0, atol=5e-12)
    np.testing.assert_allclose(vr[:, 1], v[:, 0], rtol=0, atol=5e-12)


def test_antiparallel_lines_have_zero_velocity():
    """Two antiparallel straight lines on a point-symmetric lattice: every
    node is a centre of symmetry of all other vorticity, and a straight line
    induces nothing on itself (Sec. 5.1 case 2), so v = 0 exactly."""
    f = W.antiparallel_lines(N_l=16, offset=(0.3, 0.7))
    g = _geom(f)
    v, psi = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    assert np.abs(v).max() < 2e-13


def test_matched_split_at_high_beta_equals_converged():
    """At beta = 8 the fast method's own truncation (minimum image with
    r_c = beta/alpha, mode cube |m| <= K) is converged: the matched parts
    must add up to the converged total."""
    f = W.ellipses(nfil=2, N_l=16, seed=3)
    g = _geom(f)
    beta = 8.0
    alpha = 2 * beta / f.L[0]         # r_c = L/2
    K = int(math.ceil(2 * beta * alpha * f.L[0] / (2 * np.pi)))
    m = oracle.components_matched(g, f.L, KAPPA, A_CORE, DELTA, alpha, beta / alpha, K)
    v, psi = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    assert np.abs(m["total"] - v).max() < 1e-12 * np.abs(v).max()
    assert np.abs(m["psi_total"] - psi).max() < 1e-12 * np.abs(psi).max()


def test_truncation_error_within_paper_estimate():
    """Sec. 4, Eq. error_trunc_velocity: at beta = 3.5 the rms error of the
    matched sum against the converged one stays below the estimate
    (an upper bound 'in almost all cases')."""
    f = W.ellipses(nfil=6, N_l=24, seed=9)
    g = _geom(f)
    L = f.L[0]
    V = L ** 3
    beta, M = 3.5, 32
    Kc = (M - 1) // 2
    alpha = (2 * np.pi / L) * Kc / (2 * beta)
    m = oracle.components_matched(g, f.L, KAPPA, A_CORE, DELTA, alpha, beta / alpha, Kc)
    v, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    rms = lambda u: np.sqrt(np.mean(np.sum(u ** 2, axis=1)))
    err = rms(m["total"] - v)
    Lt = g.lp.sum()
    eps_v = KAPPA * (Lt / (np.sqrt(np.pi) * alpha * V) + (1 / beta) * np.sqrt(Lt / (8 * np.pi * V))) * np.exp(-beta ** 2)
    assert err < eps_v, (err, eps_v)
    assert err > eps_v / 100  # the estimate is not wildly loose either


def test_ring_energy_converges_to_closed_form():
    """Eq. vortex_ring_energy: E V = kappa^2 R/2 [ln(8R/a) - (Delta + 1)] for an
    isolated ring; the periodic, discretised energy approaches it as N and L
    grow (the paper prints no tolerance: convergence only)."""
    k = GOLD["kelvin_ring"]
    errs = []
    for N, L in ((32, 2 * np.pi), (64, 4 * np.pi), (128, 8 * np.pi)):
        f = W.ring(R=k["R"], N=N, L=L)
        g = _geom(f, 4, 3)
        E = oracle.energy_converged(g, f.L, k["kappa"], k["a"], k["delta"])
        errs.append(abs(E * L ** 3 - k["E_times_V"]) / k["E_times_V"])
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-5, errs


def test_energy_depends_on_alpha_only_through_interpolation():
    """The long-range energy is the exact Fourier reduction while the other
    parts are interpolated from the nodes, so the total moves with alpha only
    by the interpolation error, which vanishes as the nodes get denser."""
    d = []
    for N in (24, 48, 96):
        f = W.ring(R=1.0, N=N)
        g = _geom(f, 4, 2)
        e1 = oracle.energy_converged(g, f.L, KAPPA, A_CORE, DELTA)
        e2 = oracle.energy_converged(g, f.L, KAPPA, A_CORE, DELTA, alpha_scale=1.5)
        d.append(abs(e1 - e2) / abs(e1))
    assert d[0] > d[1] > d[2] and d[2] < 1e-8, d


def test_rk4_energy_and_impulse_drift_shrink_with_resolution():
    """Sec. 5.2: the filament energy and impulse are invariants of the
    continuous motion, so their drift over a fixed time under RK4 with the
    Kelvin-wave step comes only from the discretisation and must shrink as
    the curves are refined (leapfrogging ellipses, N_l = 32 -> 64, same
    physical time).  A wrong sign or a dropped term in any velocity part
    breaks the conservation at every resolution."""
    def kelvin_wave_period(lam):
        # Sec. 5.2: T = (2 lam^2 / kappa) / [ln(lam / (pi a)) + 1/2 - (Delta + gamma_E)]
        gamma_e = 0.57721566490153286061
        return 2.0 * lam * lam / KAPPA / (math.log(lam / (math.pi * A_CORE)) + 0.5 - (DELTA + gamma_e))

    drifts = []
    T = None
    for N_l in (32, 64):
        f = W.leapfrog_ellipses(N_l=N_l)
        dmin = min(np.linalg.norm(np.diff(f.nodes[f.offsets[l]:f.offsets[l + 1]], axis=0, append=f.nodes[
            f.offsets[l]:f.offsets[l] + 1]), axis=1).min() for l in range(f.nfil))
        dt = kelvin_wave_period(dmin)
        if T is None:
            T = 10 * dt
        n = int(round(T / dt))
        dt = T / n
        x1 = oracle.rk4_converged(f.nodes, f.offsets, f.closing, f.L, KAPPA, A_CORE, DELTA, dt, n)
        e0 = oracle.energy_converged(oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2), f.L, KAPPA,
                                     A_CORE, DELTA)
        e1 = oracle.energy_converged(oracle.geometry(x1, f.offsets, f.closing, f.L, 4, 2), f.L, KAPPA,
                                     A_CORE, DELTA)
        p0 = oracle.polygon_impulse(f.nodes, f.offsets, KAPPA)
        p1 = oracle.polygon_impulse(x1, f.offsets, KAPPA)
        drifts.append((abs(e1 - e0) / abs(e0), np.linalg.norm(p1 - p0) / np.linalg.norm(p0)))
        # the pair moves: the time span is not trivially short
        assert np.abs(x1 - f.nodes).max() > 1e-3
    (e32, p32), (e64, p64) = drifts
    assert e32 < 1e-4 and p32 < 2e-5
    assert e64 < e32 / 2.5 and p64 < p32 / 2.5


def test_energy_spectrum_of_straight_lines_follows_inverse_k():
    """Sec. 6: at scales below the vortex spacing the spectrum of straight
    vortices is E(k) = kappa^2 Lv / (4 pi V) k^-1 (Lv the total length).  Two
    antiparallel z-lines (Lv = 2L); averaged over shells 6..20 the
    compensated spectrum E(k) k / (kappa^2 Lv / 4 pi V) is 1 within 5 %, and
    only modes with k_z = 0 carry energy (the field does not vary along z)."""
    f = W.antiparallel_lines(N_l=32)
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    k, E = oracle.energy_spectrum(g, f.L, KAPPA, 24, 30)
    V = float(np.prod(f.L))
    pred = KAPPA ** 2 * 2 * f.L[0] / (4 * math.pi * V)
    ratio = E[6:21] * k[6:21] / pred
    assert abs(ratio.mean() - 1.0) < 0.05, ratio
    # no energy at k = 0 and none in modes with k_z != 0: the k_z = 0 plane alone gives it all
    Kv = 24
    om = oracle.fourier_coefs(g, f.L, KAPPA, np.array([Kv] * 3, np.int32)).reshape(49, 49, 49, 3, 2)
    off_plane = np.abs(np.delete(om, Kv, axis=2)).max()
    assert off_plane < 1e-12 * np.abs(om).max()
    assert E[0] == 0.0


def test_subdivided_local_terms():
    """Sec. 5.2: with the local segments subdivided, the Taylor part covers a
    fraction f of each local segment and the plain Biot-Savart kernel the
    rest (geometric pieces).  f = 1 is the plain local term; the pieces
    resolve the near-singular integrand (3 and 12 Gauss points agree to
    1e-5); on a coarse ring the subdivided speed is already near its
    converged value while the plain one is not."""
    f = W.ring(N=32, L=8 * math.pi)
    g3 = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 6, 3)
    v1, p1 = oracle.local_subdivided(g3, KAPPA, A_CORE, DELTA, 1.0, 6)
    v0, p0 = oracle.local(g3, KAPPA, A_CORE, DELTA)
    assert np.abs(v1 - v0).max() < 1e-14 * np.abs(v0).max()
    assert np.abs(p1 - p0).max() < 1e-14 * np.abs(p0).max()
    g12 = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 6, 12)
    va, _ = oracle.local_subdivided(g3, KAPPA, A_CORE, DELTA, 0.1, 6)
    vb, _ = oracle.local_subdivided(g12, KAPPA, A_CORE, DELTA, 0.1, 6)
    assert np.abs(va - vb).max() < 1e-5 * np.abs(vb).max()
    dev = {}
    for N in (16, 64):
        fr = W.ring(N=N, L=8 * math.pi)
        g = oracle.geometry(fr.nodes, fr.offsets, fr.closing, fr.L, 6, 3)
        plain, _ = oracle.velocity_converged(g, fr.L, KAPPA, A_CORE, DELTA)
        sub, _ = oracle.velocity_converged(g, fr.L, KAPPA, A_CORE, DELTA, local_frac=0.1, order=6)
        dev[N] = (plain[:, 2].mean(), sub[:, 2].mean())
    gap_plain = abs(dev[16][0] - dev[64][0])
    gap_sub = abs(dev[16][1] - dev[64][1])
    assert gap_sub < gap_plain / 2, (gap_sub, gap_plain)
