"""Parity of the CUDA path against the FP64 oracle (``-m gpu``).

Every call goes through the C ABI (ctypes binding).  Tolerances:
  * float64 form, parts at the method's own split: each part to <= 1e-12 of
    its scale (short range, local, self), the long-range part to the NUFFT
    error (<= 1e-10 at w = 16, sigma = 2; <= 1e-6 at w = 8, sigma = 1.5,
    Appendix A: ~10^{-0.9 w});
  * float64 form, total against the converged sum: <= 1e-6 rms relative at
    beta = 3.5 (the method's own truncation, Sec. 4) and <= 1e-10 at
    beta = 8, w = 16, sigma = 2 (implementation parity);
  * mixed form: <= 1e-5 rms relative (the float32 budget).
"""
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


def rms_rel(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1)) / np.mean(np.sum(b ** 2, axis=1))))


def geom(f, order=4, Q=2):
    return oracle.geometry(f.nodes, f.offsets, f.closing, f.L, order, Q)


def gpu_velocity(f, p, want_psi=False):
    B = _B()
    bs = B.BiotSavart(p, f.offsets, f.closing)
    nodes = torch.from_numpy(f.nodes).cuda()
    out = bs.velocity(nodes, want_psi=want_psi)
    bs.status()
    torch.cuda.synchronize()
    bs.close()
    if want_psi:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


def gpu_parts(f, p, want_psi=False):
    B = _B()
    bs = B.BiotSavart(p, f.offsets, f.closing)
    nodes = torch.from_numpy(f.nodes).cuda()
    out = bs.parts(nodes, want_psi=want_psi)
    bs.status()
    torch.cuda.synchronize()
    bs.close()
    if want_psi:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


def params(f, **kw):
    B = _B()
    return B.make_params(f.L, kappa=KAPPA, a=A_CORE, delta=DELTA, **kw)


def _min_image(d, L):
    return d - L[None, :] * np.round(d / L[None, :])


# ------------------------------------------------------------------ geometry
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["ellipses", "lines", "ragged"])
def test_quadrature_points_and_charges(case, prec):
    """Sec. 2.6 / 3.3: quadrature points s(tau_j + h_i dtau_j) and charges
    w_i dtau_j s'(tau) from the GPU spline equal the oracle's B-spline ones."""
    B = _B()
    f = {"ellipses": lambda: W.ellipses(nfil=5, N_l=20, seed=11),
         "lines": lambda: W.three_line_pairs(N_l=12),
         "ragged": lambda: _ragged()}[case]()
    Q = 3
    p = params(f, M=32, Q=Q, precision=B.BS_FP64 if prec == "fp64" else B.BS_MIXED)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    qX, qq = bs.quadrature(torch.from_numpy(f.nodes).cuda())
    torch.cuda.synchronize()
    qX, qq = qX.cpu().numpy(), qq.cpu().numpy()
    bs.close()
    g = geom(f, 4, Q)
    tol = 1e-12 if prec == "fp64" else 2e-6
    dX = _min_image(qX - g.qX, f.L)
    assert np.abs(dX).max() < tol * max(1.0, np.abs(f.nodes).max())
    assert np.abs(qq - g.qq).max() < tol * np.abs(g.qq).max() * 10
    assert np.all(qX >= 0) and np.all(qX < f.L[None, :])


def test_long_filament_spline_fallback():
    """A filament too long for the shared-memory spline fit (1500 nodes in
    float64) takes the global-memory path; its quadrature must match too."""
    B = _B()
    f = W.ring(R=1.1, N=1500)
    p = params(f, M=32, Q=2, precision=B.BS_FP64)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    qX, qq = bs.quadrature(torch.from_numpy(f.nodes).cuda())
    torch.cuda.synchronize()
    qX, qq = qX.cpu().numpy(), qq.cpu().numpy()
    bs.close()
    g = geom(f, 4, 2)
    assert np.abs(_min_image(qX - g.qX, f.L)).max() < 1e-12 * np.abs(f.nodes).max()
    assert np.abs(qq - g.qq).max() < 1e-11 * np.abs(g.qq).max()


def _ragged():
    """Filaments of very different sizes, including the minimum N_l = 4."""
    parts = [W.ring(R=0.9, N=4, center=[1.0, 2.0, 3.0]), W.ring(R=0.5, N=5, center=[4.0, 1.0, 2.0], axis=0),
             W.ellipses(nfil=2, N_l=17, seed=4), W.ring(R=1.2, N=64, center=[3.0, 3.0, 5.0], axis=1)]
    nodes = np.concatenate([q.nodes for q in parts])
    counts = np.concatenate([np.diff(q.offsets) for q in parts])
    off = np.zeros(counts.size + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    return W.Filaments(nodes, off, np.zeros((counts.size, 3), np.int32), parts[0].L, "ragged")


# ------------------------------------------------------------------ parts at the method's own split
@pytest.mark.parametrize("nufft", ["w16s2", "w8s15"])
@pytest.mark.parametrize("case", ["ring", "ellipses", "ragged"])
def test_parts_fp64_match_oracle(case, nufft):
    """Each part of Eq. ewald_velocity_splitting, float64 form, against the
    oracle evaluated at the same alpha, r_c and mode cube."""
    B = _B()
    f = {"ring": lambda: W.ring(N=64), "ellipses": lambda: W.ellipses(nfil=6, N_l=24, seed=9),
         "ragged": _ragged}[case]()
    w, sigma = (16, 2.0) if nufft == "w16s2" else (8, 1.5)
    p = params(f, M=32, Q=2, w=w, sigma=sigma, precision=B.BS_FP64, flags=B.BS_WANT_PSI)
    (vp, pp) = gpu_parts(f, p, want_psi=True)
    g = geom(f, 4, 2)
    K = (p.M[0] - 1) // 2
    m = oracle.components_matched(g, f.L, KAPPA, A_CORE, DELTA, p.alpha, p.rc, K)
    vscale = np.abs(m["total"]).max()
    pscale = np.abs(m["psi_total"]).max()
    for i, name in enumerate(["local", "short", "long", "self"]):
        tol = 1e-12
        if name == "long":
            tol = 1e-10 if nufft == "w16s2" else 1e-6
        err = np.abs(vp[i] - m[name]).max() / vscale
        assert err < tol, (name, err)
        errp = np.abs(pp[i] - m["psi_" + name]).max() / pscale
        assert errp < tol, ("psi_" + name, errp)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["ellipses", "tangle"])
def test_pruned_fft_equals_full_cufft(case, prec):
    """The library's pruned per-axis transforms and the full cuFFT R2C/C2R
    path compute the same long-range part (and psi) up to rounding."""
    B = _B()
    f = W.ellipses(nfil=10, N_l=32, seed=4) if case == "ellipses" else W.fourier_tangle(200, 40, seed=8,
                                                                                          amp=2 * math.pi / 50)
    pr = B.BS_FP64 if prec == "fp64" else B.BS_MIXED
    outs = []
    for extra in (0, B.BS_FFT_CUFFT):
        p = params(f, M=48, Q=2, w=8, precision=pr, flags=B.BS_WANT_PSI | extra)
        outs.append(gpu_parts(f, p, want_psi=True))
    (va, pa), (vb, pb) = outs
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert np.abs(va[2] - vb[2]).max() < tol * np.abs(vb[2]).max()
    assert np.abs(pa[2] - pb[2]).max() < tol * np.abs(pb[2]).max()


def test_parts_mixed_match_oracle():
    B = _B()
    f = W.ellipses(nfil=6, N_l=24, seed=9)
    p = params(f, M=32, Q=2, w=8, precision=B.BS_MIXED)
    vp = gpu_parts(f, p)
    g = geom(f, 4, 2)
    m = oracle.components_matched(g, f.L, KAPPA, A_CORE, DELTA, p.alpha, p.rc, (p.M[0] - 1) // 2)
    vscale = np.abs(m["total"]).max()
    for i, name in enumerate(["local", "short", "long", "self"]):
        err = np.abs(vp[i] - m[name]).max() / vscale
        assert err < 1e-5, (name, err)


# ------------------------------------------------------------------ totals against the converged sum
@pytest.mark.parametrize("case", ["ring", "ellipses"])
def test_total_fp64_beta35(case):
    """Config-1-like ring and a small ellipse set at beta = 3.5: rms error
    within 1e-6; for the ellipses also within twice the Sec. 4 estimate (a
    statistical estimate for disordered sets, which a lone ring need not meet)."""
    B = _B()
    f = W.ring(N=64) if case == "ring" else W.ellipses(nfil=8, N_l=32, seed=5)
    p = params(f, M=32, Q=2, w=8, precision=B.BS_FP64)
    v = gpu_velocity(f, p)
    g = geom(f, 4, 2)
    vr, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    eps_v, _ = B.bs_error_estimate(p, g.lp.sum())
    err = rms_rel(v, vr)
    vrms = np.sqrt(np.mean(np.sum(vr ** 2, axis=1)))
    assert err < 1e-6, err
    if case == "ellipses":
        assert err < 2 * eps_v / vrms, (err, eps_v / vrms)


def test_total_fp64_high_accuracy_is_implementation_parity():
    """beta = 8, w = 16, sigma = 2: truncation and NUFFT errors are below
    rounding, so the GPU total must equal the converged oracle."""
    B = _B()
    f = W.ellipses(nfil=4, N_l=24, seed=3)
    L = f.L[0]
    beta = 8.0
    alpha = 2 * beta / L
    K = int(math.ceil(beta * alpha * L / math.pi))
    p = params(f, M=2 * K + 1, Q=2, w=16, sigma=2.0, precision=B.BS_FP64, beta=beta, alpha=alpha,
               flags=B.BS_WANT_PSI)
    v, psi = gpu_velocity(f, p, want_psi=True)
    g = geom(f, 4, 2)
    vr, pr = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    assert rms_rel(v, vr) < 1e-10
    assert rms_rel(psi, pr) < 1e-10


@pytest.mark.parametrize("case", ["ring64", "ellipses40"])
def test_total_mixed_configs(case):
    """Mixed precision on the ring (64 nodes, M = 32) and the 40-ellipse set
    (2560 nodes, Q = 3, M = 64): rms error <= 1e-5 against the converged sum.
    w = 8 keeps the NUFFT error (~1e-5 of the total at w = 6 on the ring,
    Appendix A) below the float32 budget being checked here."""
    B = _B()
    spec = W.WORKLOADS[case]
    f = spec["gen"]()
    p = params(f, M=spec["M"], Q=spec["Q"], w=8, sigma=1.5, precision=B.BS_MIXED)
    v = gpu_velocity(f, p)
    g = geom(f, 4, spec["Q"])
    vr, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    assert rms_rel(v, vr) < 1e-5


def test_ellipses40_fp64_and_alpha_sweep():
    """40 ellipses, float64, alpha in {0.5, 0.71, 1, 1.41, 2} alpha_0 with M
    re-derived (k_max = 2 beta alpha): every result within the Sec. 4 bound of
    the converged sum, hence of each other (Sec. 3.1 alpha-invariance)."""
    B = _B()
    f = W.ellipses()
    g = geom(f, 4, 3)
    vr, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    L = f.L[0]
    beta = 3.5
    a0 = 31.0 / (2 * beta)
    outs = []
    for s in (0.5, 0.71, 1.0, 1.41, 2.0):
        alpha = s * a0
        K = int(math.ceil(beta * alpha * L / math.pi))
        p = params(f, M=2 * K + 1, Q=3, w=8, precision=B.BS_FP64, beta=beta, alpha=alpha)
        assert p.rc <= L / 2
        v = gpu_velocity(f, p)
        eps_v, _ = B.bs_error_estimate(p, g.lp.sum())
        vrms = np.sqrt(np.mean(np.sum(vr ** 2, axis=1)))
        err = rms_rel(v, vr)
        assert err < max(1e-6, 2 * eps_v / vrms), (s, err, eps_v / vrms)
        outs.append(v)
    for v in outs[1:]:
        assert rms_rel(v, outs[0]) < 2e-6


# ------------------------------------------------------------------ full-size workloads
# The benchmarked workloads (tangle1e5, tangle4e6, the 64-tangle batch) are
# checked against stored converged-oracle samples in
# tests/test_gpu_workload_accuracy.py.


# ------------------------------------------------------------------ edge cases
def test_antiparallel_lines_zero_velocity():
    B = _B()
    f = W.antiparallel_lines(N_l=16, offset=(0.3, 0.7))
    for prec, tol in ((B.BS_FP64, 1e-10), (B.BS_MIXED, 1e-5)):
        v = gpu_velocity(f, params(f, M=32, Q=2, precision=prec))
        assert np.abs(v).max() < tol


def test_three_line_pairs_vs_oracle():
    """Unclosed periodic lines (velocity purely non-local, Sec. 5.1 case 2).
    At w = 16, sigma = 2 the GPU equals the oracle at the same split (NUFFT
    error below rounding); at the workloads' w = 8, sigma = 1.5 it stays
    within the Sec. 4 truncation estimate of the converged sum.  The
    long-range part dominates here, so its NUFFT error (~3e-6 of its size
    at w = 8: the truncated kernel jumps by zeta/sinh(zeta) ~ 2e-6 at the
    support edge) is not masked by a large local term."""
    B = _B()
    f = W.three_line_pairs(N_l=16)
    g = geom(f, 4, 2)
    p16 = params(f, M=32, Q=2, w=16, sigma=2.0, precision=B.BS_FP64)
    v16 = gpu_velocity(f, p16)
    m = oracle.components_matched(g, f.L, KAPPA, A_CORE, DELTA, p16.alpha, p16.rc, (p16.M[0] - 1) // 2)
    assert rms_rel(v16, m["total"]) < 1e-10
    p = params(f, M=32, Q=2, w=8, precision=B.BS_FP64)
    v = gpu_velocity(f, p)
    vr, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    eps_v, _ = B.bs_error_estimate(p, g.lp.sum())
    vrms = np.sqrt(np.mean(np.sum(vr ** 2, axis=1)))
    assert rms_rel(v, vr) < 2 * eps_v / vrms


def test_ragged_and_minimum_filaments():
    B = _B()
    f = _ragged()
    v = gpu_velocity(f, params(f, M=32, Q=2, precision=B.BS_FP64))
    g = geom(f, 4, 2)
    vr, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    assert rms_rel(v, vr) < 1e-6


@pytest.mark.parametrize("cell_div", [1, 2, 3, 4])
def test_cell_size_does_not_change_short_range(cell_div):
    B = _B()
    f = W.ellipses(nfil=6, N_l=24, seed=9)
    p = params(f, M=48, Q=2, precision=B.BS_FP64, cell_div=cell_div)
    vp = gpu_parts(f, p)
    g = geom(f, 4, 2)
    vs, _ = oracle.short_range(g, f.L, KAPPA, p.alpha, p.rc)
    assert np.abs(vp[1] - vs).max() < 1e-12 * np.abs(vs).max()


def test_rc_equal_half_box():
    """alpha = 7/L so that r_c = L/2 exactly (Sec. 5.2): fewer cells than
    2m+1 per axis, every pair seen once through its minimum image."""
    B = _B()
    f = W.leapfrog_ellipses(N_l=32)
    L = f.L[0]
    alpha = 7.0 / L
    K = int(math.ceil(3.5 * alpha * L / math.pi))
    p = params(f, M=2 * K + 1, Q=3, w=8, precision=B.BS_FP64, alpha=alpha)
    assert abs(p.rc - L / 2) < 1e-12
    v = gpu_velocity(f, p)
    g = geom(f, 4, 3)
    vr, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
    assert rms_rel(v, vr) < 1e-6


def test_empty_filament_set():
    B = _B()
    p = B.make_params([2 * math.pi] * 3, M=32)
    ctx = B.bs_create(p)
    B.bs_set_filaments(ctx, np.zeros(1, np.int64))
    vel = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    nodes = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    B.bs_compute(ctx, nodes, vel)
    B.bs_status(ctx)
    B.bs_destroy(ctx)


def test_host_entry_point_equals_device_entry_point():
    B = _B()
    f = W.ellipses(nfil=5, N_l=20, seed=2)
    p = params(f, M=32, Q=2, precision=B.BS_MIXED, flags=B.BS_WANT_PSI)
    ctx = B.bs_create(p)
    B.bs_set_filaments(ctx, f.offsets, f.closing)
    vh = np.zeros_like(f.nodes)
    ph = np.zeros_like(f.nodes)
    B.bs_compute_host(ctx, f.nodes, vh, ph)
    nodes = torch.from_numpy(f.nodes).cuda()
    vd = torch.empty_like(nodes)
    pd = torch.empty_like(nodes)
    B.bs_compute(ctx, nodes, vd, pd)
    B.bs_status(ctx)
    torch.cuda.synchronize()
    B.bs_destroy(ctx)
    np.testing.assert_allclose(vh, vd.cpu().numpy(), rtol=0, atol=1e-6 * np.abs(vh).max())
    np.testing.assert_allclose(ph, pd.cpu().numpy(), rtol=0, atol=1e-6 * np.abs(ph).max())


def test_errors_are_reported_not_raised_on_device():
    B = _B()
    L = [2 * math.pi] * 3
    p = B.make_params(L, M=32)
    ctx = B.bs_create(p)
    with pytest.raises(B.BSError) as e:
        B.bs_compute(ctx, torch.zeros((4, 3), dtype=torch.float64, device="cuda"),
                     torch.zeros((4, 3), dtype=torch.float64, device="cuda"))
    assert e.value.code == B.BS_ERR_STATE
    with pytest.raises(B.BSError) as e:
        B.bs_set_filaments(ctx, np.array([0, 3], np.int64))
    assert e.value.code == B.BS_ERR_SPLINE
    with pytest.raises(B.BSError) as e:
        B.bs_set_filaments(ctx, np.array([0, 8], np.int64), np.array([[0, 0, 1]], np.int32))
    assert e.value.code == B.BS_ERR_NET_VORTICITY
    B.bs_destroy(ctx)
    bad = B.make_params(L, M=32)
    bad.rc = 0.6 * L[0]
    with pytest.raises(B.BSError) as e:
        B.bs_create(bad)
    assert e.value.code == B.BS_ERR_RC_GT_HALF_L


def test_nonfinite_node_sets_status():
    B = _B()
    f = W.ring(N=16)
    nodes = f.nodes.copy()
    nodes[3, 1] = np.nan
    p = params(f, M=32, Q=2, precision=B.BS_MIXED)
    ctx = B.bs_create(p)
    B.bs_set_filaments(ctx, f.offsets, f.closing)
    d = torch.from_numpy(nodes).cuda()
    v = torch.empty_like(d)
    B.bs_compute(ctx, d, v)
    with pytest.raises(B.BSError) as e:
        B.bs_status(ctx)
    assert e.value.code == B.BS_ERR_NONFINITE
    # the context stays usable
    B.bs_compute(ctx, torch.from_numpy(f.nodes).cuda(), v)
    B.bs_status(ctx)
    B.bs_destroy(ctx)


def test_stage_times_are_recorded():
    B = _B()
    f = W.ellipses(nfil=5, N_l=20, seed=2)
    p = params(f, M=32, Q=2, precision=B.BS_MIXED, flags=B.BS_TIMING)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    bs.velocity(torch.from_numpy(f.nodes).cuda())
    t = bs.stage_times()
    bs.close()
    assert set(t) == set(B.STAGES) and all(x >= 0 for x in t.values())


@pytest.mark.parametrize("path", ["pruned", "cufft"])
def test_energy_matches_oracle(path):
    """Energy (Eq. kinetic_energy_streamfunction, float64 Fourier reduction +
    spline line integral): at w = 16, sigma = 2 the GPU equals the oracle's
    energy at the same split to 1e-10; at beta = 3.5, w = 8 it is within 1e-6
    of the oracle's energy at that split, the mixed form within 1e-5.  (The
    split energy itself moves by a few 1e-6 with alpha on this coarse curve:
    the line integral of the interpolated psi and the quadrature sum behind
    the Fourier part discretise the curve differently.)"""
    B = _B()
    f = W.ellipses(nfil=6, N_l=24, seed=9)
    g = geom(f, 4, 2)
    extra = B.BS_FFT_CUFFT if path == "cufft" else 0
    p = params(f, M=32, Q=2, w=16, sigma=2.0, precision=B.BS_FP64, flags=B.BS_WANT_PSI | extra)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    E = bs.energy(torch.from_numpy(f.nodes).cuda())
    bs.close()
    Em = oracle.energy(g, f.L, KAPPA, A_CORE, DELTA, p.alpha, p.rc, (p.M[0] - 1) // 2)
    assert abs(E - Em) < 1e-10 * abs(Em), (E, Em)
    for prec, w, tol in ((B.BS_FP64, 8, 1e-6), (B.BS_MIXED, 8, 1e-5)):
        p = params(f, M=32, Q=2, w=w, precision=prec, flags=B.BS_WANT_PSI | extra)
        bs = B.BiotSavart(p, f.offsets, f.closing)
        E = bs.energy(torch.from_numpy(f.nodes).cuda())
        bs.close()
        Em = oracle.energy(g, f.L, KAPPA, A_CORE, DELTA, p.alpha, p.rc, (p.M[0] - 1) // 2)
        assert abs(E - Em) < tol * abs(Em), (prec, E, Em)


def test_graph_replay_equals_direct_call():
    """The CUDA-graph replay of one evaluation gives the direct call's result,
    and follows new node positions written into the bound buffer."""
    B = _B()
    f = W.ellipses(nfil=8, N_l=32, seed=12)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = params(f, M=32, Q=2, precision=B.BS_FP64)
        bs = B.BiotSavart(p, f.offsets, f.closing, stream=s)
        nodes = torch.from_numpy(f.nodes).cuda()
        ref = bs.velocity(nodes).clone()
        vg = torch.empty_like(ref)
        bs.capture(nodes, vg)
        bs.launch()
        s.synchronize()
        assert (vg - ref).abs().max().item() < 1e-13 * ref.abs().max().item()
        nodes.add_(0.01)
        ref2 = bs.velocity(nodes).clone()
        bs.launch()
        s.synchronize()
        assert (vg - ref2).abs().max().item() < 1e-13 * ref2.abs().max().item()
        bs.status()
        bs.close()


def test_repeated_calls_agree():
    B = _B()
    f = W.ellipses(nfil=8, N_l=32, seed=8)
    p = params(f, M=32, Q=2, precision=B.BS_MIXED)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    nodes = torch.from_numpy(f.nodes).cuda()
    a = bs.velocity(nodes).clone()
    b = bs.velocity(nodes)
    torch.cuda.synchronize()
    bs.close()
    assert (a - b).abs().max().item() < 1e-6 * a.abs().max().item()
