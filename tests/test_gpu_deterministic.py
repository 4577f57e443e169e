"""BS_DETERMINISTIC: bitwise-reproducible evaluations (``-m gpu``)."""
import math

import numpy as np
import pytest

from paper_2406_07366_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _B():
    import paper_2406_07366_gb300 as B
    return B


@pytest.mark.parametrize("prec,M", [("mixed", 64), ("fp64", 64), ("mixed", 192)])
def test_deterministic_mode_repeats_bit_for_bit(prec, M):
    """Two contexts and two calls give identical bits for the velocity, the
    streamfunction and the energy; the result agrees with the default mode
    to the default mode's own run-to-run spread.  M = 192 (a 288^3 grid)
    takes the float32 path with 4 x 4 column blocks and 512-thread CTAs."""
    B = _B()
    f = W.fourier_tangle(nfil=300, N_l=40, seed=81, amp=2 * math.pi / 48)
    P = B.BS_MIXED if prec == "mixed" else B.BS_FP64
    nodes = torch.from_numpy(f.nodes).cuda()
    outs = []
    for _ in range(2):
        p = B.make_params(f.L, M=M, Q=2, w=6 if prec == "mixed" else 8, precision=P,
                          flags=B.BS_DETERMINISTIC | B.BS_WANT_PSI)
        bs = B.BiotSavart(p, f.offsets, f.closing)
        for _ in range(2):
            v, psi = bs.velocity(nodes, want_psi=True)
            e = bs.energy(nodes)
            outs.append((v.clone(), psi.clone(), e))
        bs.status()
        bs.close()
    v0, p0, e0 = outs[0]
    for v, psi, e in outs[1:]:
        assert torch.equal(v, v0) and torch.equal(psi, p0) and e == e0
    p = B.make_params(f.L, M=M, Q=2, w=6 if prec == "mixed" else 8, precision=P)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    vd = bs.velocity(nodes)
    bs.close()
    tol = 1e-5 if prec == "mixed" else 1e-12
    assert (vd - v0).abs().max().item() < tol * v0.abs().max().item()


def test_deterministic_mode_rejects_cufft_path():
    B = _B()
    f = W.ellipses(nfil=3, N_l=16, seed=3)
    p = B.make_params(f.L, M=24, Q=2, precision=B.BS_FP64, flags=B.BS_DETERMINISTIC | B.BS_FFT_CUFFT)
    with pytest.raises(B.BSError) as e:
        B.BiotSavart(p, f.offsets, f.closing)
    assert e.value.code == B.BS_ERR_ARG
