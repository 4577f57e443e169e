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
