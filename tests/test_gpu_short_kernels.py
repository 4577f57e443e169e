"""The two short-range kernels against the oracle (``-m gpu``, Sec. 3.2).

BS_SHORT_TILED stages the sources near each r_c cube of nodes in shared
memory; BS_SHORT_PER_NODE walks each node's neighbour rows in global memory.
Both must equal the oracle's brute-force short-range sum (minimum image,
cut-off r_c, C_0 omitted) to rounding in float64, over the cell sizes
r_c/m, m = 1..4, the r_c = L/2 case where the staged cells would wrap onto
themselves, and staged sets larger than one shared-memory chunk.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_07366_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA, A_CORE, DELTA = 1.0, 1e-6, 0.25


def _short(B, f, p, kernel):
    p.flags = (p.flags & ~(B.BS_SHORT_TILED | B.BS_SHORT_PER_NODE)) | kernel
    bs = B.BiotSavart(p, f.offsets, f.closing)
    nodes = torch.from_numpy(f.nodes).cuda()
    parts = bs.parts(nodes)
    bs.status()
    torch.cuda.synchronize()
    out = parts[1].cpu().numpy()
    bs.close()
    return out


def _kernels(B):
    return {"tiled": B.BS_SHORT_TILED, "per_node": B.BS_SHORT_PER_NODE}


@pytest.mark.parametrize("kernel", ["tiled", "per_node"])
@pytest.mark.parametrize("cell_div", [1, 2, 3, 4])
def test_short_range_kernels_match_oracle_fp64(kernel, cell_div):
    import paper_2406_07366_gb300 as B
    f = W.ellipses(nfil=6, N_l=24, seed=9)
    p = B.make_params(f.L, kappa=KAPPA, a=A_CORE, delta=DELTA, M=48, Q=2, precision=B.BS_FP64, cell_div=cell_div)
    v = _short(B, f, p, _kernels(B)[kernel])
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    vs, _ = oracle.short_range(g, f.L, KAPPA, p.alpha, p.rc)
    assert np.abs(v - vs).max() < 1e-12 * np.abs(vs).max()


@pytest.mark.parametrize("kernel", ["tiled", "per_node"])
def test_short_range_kernels_half_box_cutoff_and_many_sources(kernel):
    """r_c = L/2 (alpha = 7/L): every axis of the staged region wraps onto
    itself, so all sources are staged once and pairs take the minimum image;
    the 40 ellipses' 7680 sources exceed one staging chunk."""
    import paper_2406_07366_gb300 as B
    f = W.ellipses()
    L = f.L[0]
    alpha = 7.0 / L
    K = int(math.ceil(3.5 * alpha * L / math.pi))
    p = B.make_params(f.L, kappa=KAPPA, a=A_CORE, delta=DELTA, M=2 * K + 1, Q=3, w=8, precision=B.BS_FP64,
                      alpha=alpha)
    assert abs(p.rc - L / 2) < 1e-12
    v = _short(B, f, p, _kernels(B)[kernel])
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 3)
    vs, _ = oracle.short_range(g, f.L, KAPPA, p.alpha, p.rc)
    assert np.abs(v - vs).max() < 1e-12 * np.abs(vs).max()


def test_short_range_kernels_agree_on_a_dense_tangle_mixed():
    """A dense random tangle in float32: the two kernels sum the same pairs
    (only the order differs) and both match the oracle to the float32 budget."""
    import paper_2406_07366_gb300 as B
    f = W.fourier_tangle(nfil=300, N_l=100, seed=31)
    ref = B.make_params(f.L, M=256, beta=3.5)  # the cut-off of the 1e5-node tangle
    p = B.make_params(f.L, kappa=KAPPA, a=A_CORE, delta=DELTA, M=64, Q=2, w=6, precision=B.BS_MIXED,
                      alpha=ref.alpha, rc=ref.rc)
    vt = _short(B, f, p, B.BS_SHORT_TILED)
    vn = _short(B, f, p, B.BS_SHORT_PER_NODE)
    scale = np.abs(vn).max()
    assert np.abs(vt - vn).max() < 1e-5 * scale
    rng = np.random.default_rng(3)
    tg = np.sort(rng.choice(f.N, 256, replace=False))
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, 2)
    vs, _ = oracle.short_range(g, f.L, KAPPA, p.alpha, p.rc, targets=tg)
    assert np.abs(vt[tg] - vs).max() < 1e-5 * scale
