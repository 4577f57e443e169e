"""Batches of independent configurations (``-m gpu``).

Each member of a batch is evaluated by the same stage kernels as a single
context; the batch only changes how the members are issued: the staged group
(small members, or BS_BATCH_STAGED) with one launch per stage for all its
members (each running its own blocks with its own parameters), the other
members (large, or BS_BATCH_PER_MEMBER) by themselves on concurrent streams,
all in one CUDA graph.  So every member must reproduce the result of its own
single context, and, through that, the oracle.
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


def _members(seed=31):
    """Five members of different sizes, shapes and grids."""
    fs = [W.fourier_tangle(nfil=n, N_l=N_l, seed=seed + k, amp=2 * math.pi / 48)
          for k, (n, N_l) in enumerate([(30, 40), (6, 24), (80, 32), (12, 64)])]
    fs.append(W.ellipses(nfil=9, N_l=32, seed=seed + 7))
    return fs


def _run_batch(B, params, fs, stream):
    with torch.cuda.stream(stream):
        bt = B.BiotSavartBatch(params, fs, stream=stream)
        nodes = torch.from_numpy(np.concatenate([f.nodes for f in fs])).cuda()
        vel = bt.velocity(nodes)
        bt.status()
    return bt, nodes, vel


def _single(B, p, f):
    bs = B.BiotSavart(p, f.offsets, f.closing)
    v = bs.velocity(torch.from_numpy(f.nodes).cuda()).clone()
    bs.status()
    bs.close()
    return v


ISSUE = {"staged": (1, 1, 1, 1, 1), "per_member": (0, 0, 0, 0, 0), "hybrid": (1, 0, 1, 0, 1)}


@pytest.mark.parametrize("issue", sorted(ISSUE))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_members_equal_single_contexts(prec, issue):
    B = _B()
    fs = _members()
    P = B.BS_FP64 if prec == "fp64" else B.BS_MIXED
    params = [B.tangle_params(f.N, f.L, M_min=24, M_max=48, Q=2, w=8 if prec == "fp64" else 6, precision=P)
              for f in fs]
    for p, g in zip(params, ISSUE[issue]):
        p.flags |= B.BS_BATCH_STAGED if g else B.BS_BATCH_PER_MEMBER
    assert len({p.M[0] for p in params}) > 1  # the members have different grids
    s = torch.cuda.Stream()
    bt, nodes, vel = _run_batch(B, params, fs, s)
    assert tuple(int(x) for x in bt.staged) == ISSUE[issue]
    off = bt.offsets
    assert list(np.diff(off)) == [f.N for f in fs]
    tol = 1e-12 if prec == "fp64" else 1e-6  # float atomics reorder the mixed sums
    for i, (p, f) in enumerate(zip(params, fs)):
        ref = _single(B, p, f)
        got = vel[off[i]:off[i + 1]]
        err = (got - ref).abs().max().item() / ref.abs().max().item()
        assert err < tol, (i, err)
    bt.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("M", [47, 95])
def test_tensor_copy_passes_equal_per_element_passes(prec, M):
    """With K_z + 1 even (M = 47: 24 z-modes on a 72-point grid; M = 95: 48 on
    144) a single context's y and x passes move their rows with tensor copies,
    while the staged batch kernels move the same rows with per-element copies.
    The transforms, the k-space step and every sum are the same, so one member
    staged by itself reproduces its single context (float64 to 1e-12; float32
    up to the order of its atomic sums)."""
    B = _B()
    f = W.fourier_tangle(nfil=24, N_l=32, seed=91, amp=2 * math.pi / 48)
    P = B.BS_FP64 if prec == "fp64" else B.BS_MIXED
    p = B.make_params(f.L, beta=3.5, M=M, Q=2, w=8 if prec == "fp64" else 6, precision=P)
    p.flags |= B.BS_BATCH_STAGED
    s = torch.cuda.Stream()
    bt, nodes, vel = _run_batch(B, [p], [f], s)
    assert tuple(int(x) for x in bt.staged) == (1,)
    got = vel.clone()
    bt.close()
    ref = _single(B, p, f)
    err = (got - ref).abs().max().item() / ref.abs().max().item()
    assert err < (1e-12 if prec == "fp64" else 1e-6), err


def test_batch_replay_follows_new_positions_and_matches_oracle():
    """The captured batch reads the node buffer at replay time; after
    deforming the curves in place, each member matches the oracle's
    converged velocity at the method's beta = 3.5 accuracy."""
    B = _B()
    fs = _members(seed=41)[:3]
    params = [B.tangle_params(f.N, f.L, M_min=32, M_max=48, Q=2, w=8, precision=B.BS_FP64) for f in fs]
    s = torch.cuda.Stream()
    bt, nodes, vel = _run_batch(B, params, fs, s)
    moved = [f.nodes + 0.02 * np.sin(3.0 * f.nodes[:, [1, 2, 0]]) for f in fs]
    with torch.cuda.stream(s):
        nodes.copy_(torch.from_numpy(np.concatenate(moved)))
        bt.velocity(nodes, vel)
        bt.status()
    off = bt.offsets
    for i, f in enumerate(fs):
        g = oracle.geometry(moved[i], f.offsets, f.closing, f.L, 4, 2)
        vo, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA)
        d = vel[off[i]:off[i + 1]].cpu().numpy() - vo
        rms = math.sqrt(np.mean(np.sum(d ** 2, 1)) / np.mean(np.sum(vo ** 2, 1)))
        assert rms < 1e-5, (i, rms)
    bt.close()


def test_batch_on_legacy_stream_issues_directly():
    """With the legacy default stream there is no graph; the result is the same."""
    B = _B()
    fs = _members(seed=51)[:2]
    params = [B.tangle_params(f.N, f.L, M_min=24, M_max=32, Q=2, w=8, precision=B.BS_FP64) for f in fs]
    bt = B.BiotSavartBatch(params, fs, stream=torch.cuda.default_stream())
    nodes = torch.from_numpy(np.concatenate([f.nodes for f in fs])).cuda()
    vel = bt.velocity(nodes)
    bt.status()
    off = bt.offsets
    for i, (p, f) in enumerate(zip(params, fs)):
        ref = _single(B, p, f)
        assert (vel[off[i]:off[i + 1]] - ref).abs().max().item() < 1e-12 * ref.abs().max().item()
    bt.close()


def test_batch_member_without_filaments_is_an_error():
    B = _B()
    f = W.ellipses(nfil=3, N_l=16, seed=3)
    p = B.make_params(f.L, M=24, Q=2, precision=B.BS_FP64)
    b = B.bs_batch_create([p, p], torch.cuda.current_stream().cuda_stream)
    try:
        B.bs_batch_set(b, 0, f.offsets, f.closing)
        nodes = torch.from_numpy(f.nodes).cuda()
        vel = torch.empty_like(nodes)
        with pytest.raises(B.BSError) as e:
            B.bs_batch_compute(b, nodes, vel)
        assert e.value.code == B.BS_ERR_STATE
    finally:
        B.bs_batch_destroy(b)


def test_staged_batch_with_an_empty_member_and_mixed_widths():
    """An empty member (no filaments) takes no blocks of the staged launches;
    members of different kernel widths cannot share launches, so the member
    whose width differs from the first grouped member's is issued by itself:
    both give each member's single-context result."""
    B = _B()
    fs = _members(seed=61)[:2]
    empty = W.Filaments(np.zeros((0, 3)), np.zeros(1, np.int64), np.zeros((0, 3), np.int32), fs[0].L, "empty")
    for widths in ((8, 8, 8), (8, 8, 6)):
        members = [fs[0], empty, fs[1]]
        params = [B.tangle_params(max(f.N, 1), f.L, M_min=24, M_max=40, Q=2, w=wd, precision=B.BS_FP64)
                  for f, wd in zip(members, widths)]
        s = torch.cuda.Stream()
        bt, nodes, vel = _run_batch(B, params, members, s)
        assert list(bt.staged) == [True, False, widths[2] == 8]
        off = bt.offsets
        assert off[2] - off[1] == 0
        for i in (0, 2):
            ref = _single(B, params[i], members[i])
            got = vel[off[i]:off[i + 1]]
            assert (got - ref).abs().max().item() < 1e-12 * ref.abs().max().item(), (widths, i)
        bt.close()


def test_staged_group_follows_the_size_rule_and_flags():
    """By default members of at most 2048 nodes join the staged group and
    larger ones are issued by themselves; BS_BATCH_STAGED and
    BS_BATCH_PER_MEMBER override the rule; both on one member is an error."""
    B = _B()
    small = W.fourier_tangle(nfil=20, N_l=50, seed=71)   # 1000 nodes
    large = W.fourier_tangle(nfil=30, N_l=100, seed=72)  # 3000 nodes
    fs = [small, large, small, large]
    params = [B.tangle_params(f.N, f.L, M_min=24, M_max=48, Q=2, w=6, precision=B.BS_MIXED) for f in fs]
    params[2].flags |= B.BS_BATCH_PER_MEMBER
    params[3].flags |= B.BS_BATCH_STAGED
    s = torch.cuda.Stream()
    bt, nodes, vel = _run_batch(B, params, fs, s)
    assert list(bt.staged) == [True, False, False, True]
    off = bt.offsets
    for i, (p, f) in enumerate(zip(params, fs)):
        ref = _single(B, p, f)
        got = vel[off[i]:off[i + 1]]
        assert (got - ref).abs().max().item() < 1e-6 * ref.abs().max().item(), i
    bt.close()
    bad = B.tangle_params(small.N, small.L, M_min=24, M_max=32, Q=2, w=6, precision=B.BS_MIXED)
    bad.flags |= B.BS_BATCH_STAGED | B.BS_BATCH_PER_MEMBER
    with pytest.raises(B.BSError) as e:
        B.bs_batch_create([bad], torch.cuda.current_stream().cuda_stream)
    assert e.value.code == B.BS_ERR_ARG
