"""The allocation-free short-range entry point (``-m gpu``).

bs_short_range_static serves callers that cannot allocate device memory
(an application that owns all device memory through its own allocator or a
fixed budget, or a latency-critical loop that must avoid the device
synchronisation cudaMalloc/cudaFree can cause): its cell-list scratch is a
fixed array inside the library.  This test checks it against the short-range
part that the regular entry point (bs_compute_parts, float64 form) returns,
at the 1e-12 tolerance the float64 parity tests use, on two different
problems called back to back: the second call must not see the first call's
leftovers in the shared scratch array.
"""
import math

import numpy as np
import pytest

from paper_2406_07366_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _regular_short_range(B, f, M):
    """Short-range part and quadrature sources from the regular entry points."""
    p = B.make_params(f.L, kappa=1.0, a=1e-6, delta=0.25, M=M, Q=2, w=8, precision=B.BS_FP64)
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


def test_static_scratch_short_range_matches_regular_entry_point():
    import paper_2406_07366_gb300 as B
    problems = [(W.ellipses(nfil=12, N_l=32, seed=21), 48),
                (W.fourier_tangle(nfil=60, N_l=40, seed=22, amp=2 * math.pi / 40), 64)]
    for f, M in problems:  # two calls in a row, different sizes
        p, nodes, ref, qX, qq = _regular_short_range(B, f, M)
        got = _static_short_range(B, f, p, nodes, qX, qq)
        scale = ref.abs().max().item()
        err = (got - ref).abs().max().item() / scale
        assert err < 1e-12, err


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
