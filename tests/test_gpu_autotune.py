"""Choice of the Ewald parameter by timing (``-m gpu``), Sec. 5.3."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_07366_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA, A_CORE, DELTA = 1.0, 1e-6, 0.25


def test_autotune_keeps_beta_and_picks_the_fastest_candidate():
    import paper_2406_07366_gb300 as B
    f = W.fourier_tangle(nfil=200, N_l=50, seed=71, amp=2 * math.pi / 64)
    base = B.make_params(f.L, beta=3.5, M=64, Q=2, w=8, precision=B.BS_FP64)
    nodes = torch.from_numpy(f.nodes).cuda()
    cands = [1.0, 1.71, 3.0]
    best, ms = B.bs_autotune_alpha(base, f.offsets, f.closing, nodes, cands, reps=2)
    assert all(t > 0 for t in ms)
    i = int(np.argmin(ms))
    # the fastest candidate's parameters, beta kept, rc <= L/2
    N = f.N
    alpha0 = max(cands[i] * N ** (1 / 3) / f.L.min(), 2 * 3.5 / f.L.min())
    K = math.ceil(3.5 * alpha0 * f.L.min() / math.pi)
    assert best.M[0] == 2 * K + 1
    assert best.alpha * best.rc == pytest.approx(3.5, rel=1e-14)
    assert best.rc <= f.L.min() / 2 + 1e-12
    assert (best.quad_Q, best.nufft_w, best.precision) == (base.quad_Q, base.nufft_w, base.precision)
    # the chosen split is as accurate as any other at this beta
    bs = B.BiotSavart(best, f.offsets, f.closing)
    v = bs.velocity(nodes).cpu().numpy()
    bs.status()
    bs.close()
    tg = np.sort(np.random.default_rng(3).choice(f.N, 24, replace=False))
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    vr, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA, targets=tg)
    rms = math.sqrt(np.mean(np.sum((v[tg] - vr) ** 2, 1)) / np.mean(np.sum(vr ** 2, 1)))
    assert rms < 1e-5, rms


def test_autotune_rejects_bad_arguments():
    import paper_2406_07366_gb300 as B
    f = W.ellipses(nfil=3, N_l=16, seed=3)
    base = B.make_params(f.L, M=24, Q=2, precision=B.BS_FP64)
    nodes = torch.from_numpy(f.nodes).cuda()
    with pytest.raises(B.BSError) as e:
        B.bs_autotune_alpha(base, f.offsets, f.closing, nodes, [], reps=1)
    assert e.value.code == B.BS_ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tile_autotune_changes_speed_not_results(prec):
    """bs_autotune_tiles: z-column blocks, threads and cells per cut-off are
    implementation choices; every admissible candidate gives the same
    velocity up to rounding order, inadmissible ones are skipped (-1), and
    the returned parameters are the fastest candidate's."""
    import paper_2406_07366_gb300 as B
    f = W.fourier_tangle(nfil=200, N_l=50, seed=72, amp=2 * math.pi / 64)
    P = B.BS_FP64 if prec == "fp64" else B.BS_MIXED
    base = B.make_params(f.L, beta=3.5, M=96, Q=2, w=6 if prec == "mixed" else 8, precision=P)
    nodes = torch.from_numpy(f.nodes).cuda()
    # (2, 1): a block one column high takes the spread's generic record loop
    cands = [(0, 0, 0, 0), (2, 4, 256, 2), (4, 4, 256, 3), (1, 2, 256, 1), (4, 4, 512, 2), (3, 4, 256, 2),
             (2, 1, 256, 2)]
    best, ms = B.bs_autotune_tiles(base, f.offsets, f.closing, nodes, cands, reps=2)
    assert ms[5] == -1.0  # block_x = 3 is not a tile shape
    if prec == "fp64":
        assert ms[4] == -1.0  # 512 threads are for float32 only
    ok = [i for i, t in enumerate(ms) if t > 0]
    i = min(ok, key=lambda k: ms[k])
    assert (best.block_x, best.block_y, best.block_threads, best.cell_div) == cands[i]
    outs = []
    for k in ok:
        q = B.make_params(f.L, beta=3.5, M=96, Q=2, w=base.nufft_w, precision=P)
        q.block_x, q.block_y, q.block_threads = cands[k][:3]
        q.cell_div = cands[k][3]
        bs = B.BiotSavart(q, f.offsets, f.closing)
        outs.append(bs.velocity(nodes).cpu().numpy())
        bs.status()
        bs.close()
    tol = 1e-12 if prec == "fp64" else 2e-6
    scale = np.abs(outs[0]).max()
    for o in outs[1:]:
        assert np.abs(o - outs[0]).max() < tol * scale
