"""The allocation-free short-range entry point (``-m gpu``).

bs_short_range_static serves callers that cannot allocate device memory
(an application that owns all device memory through its own allocator or a
fixed budget, or a latency-critical loop that must avoid the device
synchronisation cudaMalloc/cudaFree can cause): its cell-list scratch is a
fixed array inside the library.  This test checks it against the short-range
part that the regular entry point (bs_compute_parts, float64 form) returns
and against the oracle's brute-force short-range sum (minimum image, cut-off
r_c, Sec. 3.2), at the 1e-12 tolerance the float64 parity tests use, on
several problems called back to back: larger and smaller ones, and cut-offs
small enough that the cells per cut-off drop from 3 to 2 and to 1 to fit the
fixed cell table.  No call may see an earlier call's leftovers in the shared
scratch array.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_07366_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _regular_short_range(B, f, M, rc_over_L=None):
    """Short-range part and quadrature sources from the regular entry points
    (rc_over_L: the cut-off as a fraction of L, alpha = beta / rc)."""
    kw = {}
    if rc_over_L is not None:
        rc = rc_over_L * float(f.L[0])
        kw = dict(alpha=3.5 / rc, rc=rc)
    p = B.make_params(f.L, kappa=1.0, a=1e-6, delta=0.25, M=M, Q=2, w=8, precision=B.BS_FP64, **kw)
    bs = B.BiotSavart(p, f.offsets, f.closing)
    nodes = torch.from_numpy(f.nodes).cuda()
    parts = bs.parts(nodes)
    qX, qq = bs.quadrature(nodes)
    bs.status()
    torch.cuda.synchronize()
    bs.close()
    return p, nodes, parts[1].clone(), qX, qq


def _static_short_range(B, f, p, nodes, qX, qq):
    Q = p.quad_Q
    N = f.N
    seg = torch.arange(N * Q, dtype=torch.int32, device="cuda") // Q
    prev = np.empty(N, dtype=np.int32)
    for l in range(f.nfil):
        a, b = int(f.offsets[l]), int(f.offsets[l + 1])
        prev[a:b] = np.roll(np.arange(a, b), 1)
    omit = torch.from_numpy(np.stack([np.arange(N, dtype=np.int32), prev], axis=1)).cuda()
    vel = torch.full((N, 3), float("nan"), dtype=torch.float64, device="cuda")
    B.bs_short_range_static(f.L, p.kappa, p.alpha, p.rc, qX, qq, seg, nodes, omit, vel,
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return vel


def _cells_per_cutoff(L, rc):
    """The m the entry point settles on: the largest of 3, 2, 1 whose cells
    of edge >= rc / m number at most 65536."""
    for m in (3, 2, 1):
        if np.prod([max(1, math.floor(Ld * m / rc)) for Ld in L]) <= 1 << 16:
            return m
    return 0


def test_static_scratch_short_range_matches_regular_entry_point_and_oracle():
    import paper_2406_07366_gb300 as B
    small = W.ellipses(nfil=12, N_l=32, seed=21)
    tangle = W.fourier_tangle(nfil=60, N_l=40, seed=22, amp=2 * math.pi / 40)
    # calls in a row: small, larger, larger with a cut-off of L/16 (m = 2),
    # the small one again (fewer cells and sources than the call before), and
    # a cut-off of L/30 (m = 1)
    problems = [(small, 48, None, 3), (tangle, 64, None, 3), (tangle, 32, 1 / 16, 2), (small, 48, None, 3),
                (tangle, 32, 1 / 30, 1)]
    for f, M, rcl, m_expected in problems:
        p, nodes, ref, qX, qq = _regular_short_range(B, f, M, rcl)
        assert _cells_per_cutoff(f.L, p.rc) == m_expected
        got = _static_short_range(B, f, p, nodes, qX, qq)
        scale = ref.abs().max().item()
        err = (got - ref).abs().max().item() / scale
        assert err < 1e-12, (M, rcl, err)
        g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
        vo, _ = oracle.short_range(g, f.L, p.kappa, p.alpha, p.rc)
        err_o = np.abs(got.cpu().numpy() - vo).max() / np.abs(vo).max()
        assert err_o < 1e-12, (M, rcl, err_o)


def test_static_scratch_rejects_oversize_input():
    import paper_2406_07366_gb300 as B
    n = (1 << 17) + 1
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    seg = torch.zeros(n, dtype=torch.int32, device="cuda")
    tgt = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    omit = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    vel = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(B.BSError) as e:
        B.bs_short_range_static([2 * math.pi] * 3, 1.0, 2.0, 1.0, pos, pos, seg, tgt, omit, vel)
    assert e.value.code == B.BS_ERR_ARG and "131072" in str(e.value)


def test_static_scratch_rejects_bad_arrays():
    """Wrong dtypes or shapes are refused before anything reaches the GPU."""
    import paper_2406_07366_gb300 as B
    n = 8
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    seg = torch.zeros(n, dtype=torch.int32, device="cuda")
    tgt = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    omit = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    vel = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    L = [2 * math.pi] * 3
    bad = [(pos.float(), pos, seg, tgt, omit, vel), (pos, pos[:4], seg, tgt, omit, vel),
           (pos, pos, seg.long(), tgt, omit, vel), (pos, pos, seg, tgt, omit[:1], vel),
           (pos, pos, seg, tgt, omit, vel[:1]), (pos, pos, seg, tgt, omit, vel.cpu())]
    for args in bad:
        with pytest.raises(B.BSError) as e:
            B.bs_short_range_static(L, 1.0, 2.0, 1.0, *args)
        assert e.value.code == B.BS_ERR_ARG
