#!/usr/bin/env python
"""Throughput of the Ewald-split periodic Biot-Savart velocity evaluation.

One step = one full evaluation (bs_compute) of the velocity at every node
of the workload: spline fit, quadrature sources, short range, long range
(spread, FFT, k-space, FFT^-1, interpolation) and local / self terms.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank evaluates its own
replica of the workload (a single configuration does not shard without an
exchange step) and `value` counts the nodes of all ranks
over the slowest rank's time.  `--impl reference` times the FP64 CPU oracle
on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "filament nodes/s per Biot–Savart eval at 1e-6 rel. err; FP32/batched vs FP64"
UNIT = "nodes/s"
L2_FLUSH_BYTES = 512 << 20
# spline, nodes, 3 x (count, 3 scan, scatter: short-range cells, spread blocks, node blocks), short range,
# spread + z FFT, y FFT, x FFT + k-space, inverse y, inverse z + interpolation, final sum
KERNELS_PER_STEP = 24


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="tangle1e5")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-sample", type=int, default=16, help="oracle targets timed for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--no-batched-form", action="store_true")
    ap.add_argument("--no-large-form", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--rk4-steps", type=int, default=100, help="RK4 steps of the large tangle")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            t0 = time.time()  # the sampler is up once its first line is written
            while time.time() - t0 < 5 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ helpers
def workload(name):
    from paper_2406_07366_gb300 import workloads as W
    spec = W.WORKLOADS[name]
    return spec, spec["gen"]()


def make_params(B, spec, f, precision, flags=0):
    w = spec["w"] if precision == B.BS_MIXED else max(spec["w"], 8)
    return B.make_params(f.L, kappa=spec["kappa"], a=spec["a"], delta=spec["delta"], beta=spec["beta"],
                         M=spec["M"], Q=spec["Q"], w=w, sigma=spec["sigma"], precision=precision, flags=flags)


def max_over_ranks(x, dist, device=None):
    """The slowest rank's time: every replica waits for the last one."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_per_rank, world, seconds):
    """Nodes/s of the whole job: every replica evaluates its own n_per_rank
    nodes per step (weak scaling) and the step ends with the slowest."""
    return n_per_rank * world / seconds


def run_batched_form(B, dev, stream, flush, steps):
    """The batched form: 64 independent Fourier tangles with node counts
    log-uniform in [10^3, 10^5] (100 nodes per filament), grids matched to
    k_max (alpha = C_beta N^(1/3)/L, M in [32, 128]), mixed precision, the
    whole batch replayed from one CUDA graph per evaluation."""
    import torch
    from paper_2406_07366_gb300 import workloads as W
    fs = W.tangle_batch(nconf=64, seed=5)
    params = [B.tangle_params(f.N, f.L, beta=3.5, M_min=32, M_max=128, Q=2, w=6, sigma=1.5,
                              precision=B.BS_MIXED) for f in fs]
    bt = B.BiotSavartBatch(params, fs, stream=stream)
    nodes = torch.from_numpy(np.concatenate([f.nodes for f in fs])).to(dev)
    vel = torch.empty_like(nodes)
    for _ in range(3):
        bt.velocity(nodes, vel)
    bt.status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        bt.velocity(nodes, vel)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    bt.status()
    bt.close()
    t = statistics.mean(ms)
    Ms = sorted(p.M[0] for p in params)
    return {"value": bt.N / (t * 1e-3), "ms_per_step": t, "steps": steps, "nconf": len(fs), "N_total": bt.N,
            "N_range": [min(f.N for f in fs), max(f.N for f in fs)], "M_range": [Ms[0], Ms[-1]],
            "issue": "one CUDA graph per evaluation, members on 8 concurrent streams"}


def run_autotuned(B, dev, spec, f, prec):
    """Sec. 5.3's alpha = C_beta N^(1/3) / L re-chosen by timing on this GPU at
    the same beta (accuracy): C_beta candidates around the paper's 1.71."""
    import torch
    base = make_params(B, spec, f, prec)
    nodes = torch.from_numpy(f.nodes).to(dev)
    cands = [1.0, 1.25, 1.5, 1.71, 2.0, 2.5, 3.0]
    best, ms = B.bs_autotune_alpha(base, f.offsets, f.closing, nodes, cands, reps=5)
    i = min(range(len(ms)), key=lambda k: ms[k])
    nxt = np.arange(f.N) + 1
    nxt[f.offsets[1:] - 1] = f.offsets[:-1]  # closed polygons
    length = float(np.linalg.norm(f.nodes[nxt] - f.nodes, axis=1).sum())
    eps_v, _ = B.bs_error_estimate(best, length)
    return {"candidates_C_beta": cands, "ms": ms, "best_C_beta": cands[i], "M": list(best.M), "alpha": best.alpha,
            "rc": best.rc, "value": f.N / (ms[i] * 1e-3), "unit": UNIT, "eps_v": eps_v,
            "note": "beta = 3.5 kept; the headline keeps the workload's M = 256"}


def polygon_impulse(nodes, offsets, kappa=1.0):
    """(kappa/2) sum over the closed polygons of s_j x s_{j+1} (host diagnostic)."""
    x = nodes.reshape(-1, 3)
    nxt = np.arange(x.shape[0]) + 1
    nxt[offsets[1:] - 1] = offsets[:-1]
    return 0.5 * kappa * np.cross(x, x[nxt]).sum(axis=0)


def run_large_form(B, dev, stream, flush, steps, rk_steps):
    """Large tangle: 20000 filaments x 200 nodes (4e6 nodes), M = 512, mixed
    precision; one evaluation replayed from its CUDA graph, then rk_steps RK4
    steps (Sec. 5.2, dt = Kelvin-wave period at the smallest node spacing)
    replayed from the captured step, with the energy and impulse drift."""
    import torch
    spec, f = workload("tangle4e6")
    p = make_params(B, spec, f, B.BS_MIXED, flags=B.BS_WANT_PSI)
    bs = B.BiotSavart(p, f.offsets, f.closing, stream=stream)
    nodes = torch.from_numpy(f.nodes).to(dev)
    vel = torch.empty_like(nodes)
    bs.capture(nodes, vel)
    for _ in range(2):
        bs.launch()
    bs.status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        bs.launch()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.mean(ms)
    out = {"workload": "tangle4e6: 20000 closed filaments x 200 nodes, N=4e6, M=512^3 modes, beta=3.5",
           "value": f.N / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "steps": steps, "n_g": B.bs_nufft_setup(
               p, want_table=False)[0], "mode": "CUDA graph replay"}
    if rk_steps > 0:
        seg = []
        x = f.nodes
        for l in range(f.nfil):
            s = x[f.offsets[l]:f.offsets[l + 1]]
            seg.append(np.linalg.norm(np.roll(s, -1, axis=0) - s, axis=1).min())
        dt = B.kelvin_wave_period(min(seg), spec["kappa"], spec["a"], spec["delta"])
        # the energies come from a float64 evaluation, so that the drift is
        # the motion's and not the float32 evaluation noise
        b64 = B.BiotSavart(make_params(B, spec, f, B.BS_FP64, flags=B.BS_WANT_PSI), f.offsets, f.closing,
                           stream=stream)
        E0 = b64.energy(nodes)
        P0 = polygon_impulse(nodes.cpu().numpy(), f.offsets, spec["kappa"])
        bs.rk4_capture(nodes, dt)
        torch.cuda.synchronize()
        e0.record(stream)
        bs.rk4_launch(rk_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        rk_ms = e0.elapsed_time(e1)
        bs.status()
        E1 = b64.energy(nodes)
        b64.close()
        P1 = polygon_impulse(nodes.cpu().numpy(), f.offsets, spec["kappa"])
        out["rk4"] = {"steps": rk_steps, "dt": dt, "ms": rk_ms, "ms_per_step": rk_ms / rk_steps,
                      "evaluations_per_s": 4 * rk_steps / (rk_ms * 1e-3),
                      "energy_rel_drift": (E1 - E0) / E0, "energy_eval": "float64 form",
                      "impulse_rel_drift": float(np.linalg.norm(P1 - P0) / np.linalg.norm(P0)),
                      "max_node_displacement": float(np.abs(nodes.cpu().numpy() - f.nodes).max())}
    bs.close()
    return out


def spread_zfft_bytes(p, ng, K, NQ, real_bytes):
    """Algorithmic bytes of one fused spread + z-transform launch: read every
    spread record once (32 B float / 64 B double) and write the retained
    z-modes 0..K_z of the three components, complex, for every (x, y) grid
    column."""
    rec = 32 if real_bytes == 4 else 64
    return rec * NQ + 3 * ng[0] * ng[1] * (K[2] + 1) * 2 * real_bytes


def stage_rooflines(ng, K, NQ, N, w, real_bytes, stage_ms, peak_gbs):
    """Algorithmic bytes of each long-range stage of the pruned pipeline and
    the fraction of the HBM peak its live stage time reaches (stages of the
    concurrent evaluation, so shared with the short-range branch).  3 real
    components, complex modes of 2 * real_bytes; retained z-modes K_z + 1,
    y-modes 2 K_y + 1."""
    cb = 2 * real_bytes
    nk, ny2 = K[2] + 1, 2 * K[1] + 1
    full = 3 * ng[0] * ng[1] * nk * cb      # F1: every (x, y) column, retained z-modes
    half = 3 * ng[0] * ny2 * nk * cb        # F2: every x, retained y- and z-modes
    nd = -(-(8 + 3 * w * real_bytes) // 16) * 16  # sorted node record with its weights
    rec = 32 if real_bytes == 4 else 64
    stage_bytes = {
        "spread": rec * NQ + full,
        "fft_fwd": full + half,
        "kspace": 2 * half,
        "fft_inv": half + full,
        # inverse z + interpolation: modes in, node records in, sums added, final float64 sum
        "interp": full + N * (nd + 3 * real_bytes + 3 * real_bytes + 24 + 24 + 24),
    }
    out = {}
    for k, b in stage_bytes.items():
        gbs = b / (stage_ms[k] * 1e-3) / 1e9
        out[k] = {"bytes": int(b), "ms": stage_ms[k], "gbs": gbs, "frac": gbs / peak_gbs}
    return out


def short_range_pairs(rc, L, N, NQ):
    """Useful short-range pairs per evaluation at uniform density: each of
    the N targets sees (4 pi / 3) r_c^3 NQ / V sources inside r_c."""
    V = float(L[0]) * float(L[1]) * float(L[2])
    return N * (4.0 * math.pi / 3.0) * rc ** 3 * NQ / V


def source_digest(path):
    """SHA-1 (12 hex digits) of a CUDA source with its comments removed and
    its whitespace collapsed: the code that ran, whatever its comments say."""
    import hashlib
    import re
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
    txt = re.sub(r"//[^\n]*", " ", txt)
    txt = " ".join(txt.split())
    return hashlib.sha1(txt.encode()).hexdigest()[:12]


def ncu_traffic(kernel, workload, source):
    """Per-launch DRAM traffic from the committed ncu summary of this kernel and
    workload, if the summary was taken from the current code (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    sha = source_digest(os.path.join(ROOT, source))
    tb = [ln.split(":")[1].strip() for ln in txt.splitlines() if ln.startswith("traffic_bytes_per_launch:")]
    src = [ln.split()[1] for ln in txt.splitlines() if ln.startswith("source:")]
    if tb and src and src[0] == sha:
        return int(tb[0])
    return None


def oracle_fixed(f, spec):
    """The oracle's per-evaluation fixed work: spline fit and quadrature of
    all filaments, and the Fourier coefficients of all sources."""
    import oracle
    t0 = time.perf_counter()
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, spec["Q"])
    alpha, K = oracle.converged_params(f.L)
    om = oracle.fourier_coefs(g, f.L, spec["kappa"], K)
    return dict(g=g, alpha=alpha, K=K, om=om, fixed_s=time.perf_counter() - t0, threads=oracle.get_threads())


def oracle_targets(f, spec, fx, tg):
    """The oracle's per-target work on targets tg: short range over all
    sources and 27 images, Fourier synthesis, self and local terms."""
    import oracle
    g, alpha, K = fx["g"], fx["alpha"], fx["K"]
    t0 = time.perf_counter()
    vs, _ = oracle.short_range(g, f.L, spec["kappa"], alpha, 0.0, all_images=True, targets=tg)
    vf, _ = oracle.fourier_eval(g, f.L, alpha, K, fx["om"], targets=tg)
    vx, _ = oracle.self_term(g, spec["kappa"], alpha, targets=tg)
    vl, _ = oracle.local(g, spec["kappa"], spec["a"], spec["delta"], targets=tg)
    return vl + vs + vf - vx, time.perf_counter() - t0


def oracle_sample(f, spec, n_sample, seed=0):
    """Time the oracle on n_sample random targets and extrapolate a full
    evaluation as fixed work + N x per-target work."""
    rng = np.random.default_rng(seed)
    tg = np.sort(rng.choice(f.N, min(n_sample, f.N), replace=False))
    fx = oracle_fixed(f, spec)
    v, tt = oracle_targets(f, spec, fx, tg)
    per_target = tt / tg.size
    return dict(v=v, targets=tg, geom=fx["g"], fixed_s=fx["fixed_s"], per_target_s=per_target,
                full_s=fx["fixed_s"] + per_target * f.N, sample_s=fx["fixed_s"] + tt, threads=fx["threads"])


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, dist):
    import torch
    import paper_2406_07366_gb300 as B

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    spec, f = workload(args.workload)
    prec = B.BS_MIXED if args.precision == "mixed" else B.BS_FP64
    p = make_params(B, spec, f, prec, flags=B.BS_TIMING)
    stream = torch.cuda.Stream(device=dev)  # non-default: the evaluation is replayed as a CUDA graph
    torch.cuda.set_stream(stream)
    bs = B.BiotSavart(p, f.offsets, f.closing, stream=stream)
    nodes = torch.from_numpy(f.nodes).to(dev)
    vel = torch.empty_like(nodes)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    for _ in range(max(args.warmup, 3)):
        bs.velocity(nodes, vel)
    bs.status()
    torch.cuda.synchronize()
    # direct calls (no graph), for reference
    ed0, ed1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    direct = []
    for _ in range(5):
        flush.zero_()
        ed0.record(stream)
        bs.velocity(nodes, vel)
        ed1.record(stream)
        torch.cuda.synchronize()
        direct.append(ed0.elapsed_time(ed1))
    # the same evaluation replayed from a CUDA graph (context without stage events)
    bsg = B.BiotSavart(make_params(B, spec, f, prec), f.offsets, f.closing, stream=stream)
    velg = torch.empty_like(nodes)
    bsg.capture(nodes, velg)
    for _ in range(3):
        bsg.launch()
    torch.cuda.synchronize()
    graph_ms = []
    for _ in range(10):
        flush.zero_()
        ed0.record(stream)
        bsg.launch()
        ed1.record(stream)
        torch.cuda.synchronize()
        graph_ms.append(ed0.elapsed_time(ed1))
    bsg.close()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = Clocks(dev.index if dev.index is not None else 0)
    clocks.start()
    step_ms, stages = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()  # L2 flush between steps, outside the timed events
        ev[k][0].record(stream)
        bs.velocity(nodes, vel)  # one full evaluation (bs_compute)
        ev[k][1].record(stream)
        stages.append(bs.stage_times())  # synchronises the streams
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    bs.status()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(step_ms)
    ms = max_over_ranks(ms, dist, dev)

    stage_mean = {k: statistics.mean(s[k] for s in stages) for k in stages[0]}
    ng, _ = B.bs_nufft_setup(p, want_table=False)
    real_bytes = 4 if prec == B.BS_MIXED else 8
    NQ = f.N * spec["Q"]
    Kd = [(p.M[i] - 1) // 2 for i in range(3)]
    sb = spread_zfft_bytes(p, ng, Kd, NQ, real_bytes)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = sb / (stage_mean["spread"] * 1e-3) / 1e9
    stage_roof = stage_rooflines(ng, Kd, NQ, f.N, p.nufft_w, real_bytes, stage_mean, peak)
    pairs = short_range_pairs(p.rc, f.L, f.N, NQ)
    short = {"pairs_est": pairs, "pairs_per_s": pairs / (stage_mean["short_range"] * 1e-3),
             "note": "uniform-density estimate of the pairs inside r_c; live stage time (concurrent branch)"}
    torch.cuda.synchronize()
    fma_peak = {"fp32_tflops": B.bs_fma_peak(B.BS_MIXED) / 1e12, "fp64_tflops": B.bs_fma_peak(B.BS_FP64) / 1e12,
                "how": "bs_fma_peak: 8 independent FMA chains per thread, 8 x 256-thread CTAs per SM"}

    # end to end through the host-buffer entry point (pinned memory)
    hn = torch.from_numpy(f.nodes).pin_memory()
    hv = torch.empty_like(hn).pin_memory()
    ctx2 = B.BiotSavart(make_params(B, spec, f, prec), f.offsets, f.closing, stream=stream)
    for _ in range(2):
        B.bs_compute_host(ctx2.ctx, hn, hv)
    torch.cuda.synchronize()
    ke = max(5, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(ke):
        B.bs_compute_host(ctx2.ctx, hn, hv)
    e2e_s = (time.perf_counter() - t0) / ke
    ctx2.close()
    e2e_s = max_over_ranks(e2e_s, dist, dev)

    autotuned = None
    if not args.no_autotune and world == 1:
        autotuned = run_autotuned(B, dev, spec, f, prec)

    large = None
    if not args.no_large_form and world == 1:
        large = run_large_form(B, dev, stream, flush, 5, args.rk4_steps)

    batched = None
    if not args.no_batched_form and world == 1:
        batched = run_batched_form(B, dev, stream, flush, min(args.steps, 20))

    # the float64 form on the same workload, for the FP32-vs-FP64 comparison
    fp64 = None
    if not args.no_fp64_form and prec == B.BS_MIXED:
        p64 = make_params(B, spec, f, B.BS_FP64)
        b64 = B.BiotSavart(p64, f.offsets, f.closing, stream=stream)
        v64 = torch.empty_like(nodes)
        for _ in range(2):
            b64.velocity(nodes, v64)
        torch.cuda.synchronize()
        k64 = min(args.steps, 5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(k64):
            flush.zero_()
            e0.record(stream)
            b64.velocity(nodes, v64)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        b64.close()
        ms64 = tot / k64
        fp64 = {"value": whole_job_rate(f.N, world, ms64 * 1e-3), "ms_per_step": ms64, "steps": k64,
                "nufft_w": p64.nufft_w}

    result = None
    if rank == 0:
        cpu = None
        accuracy = None
        if world == 1 and not args.no_cpu_baseline:
            vgpu = vel.cpu().numpy()
            o = oracle_sample(f, spec, args.cpu_sample)
            tg = o["targets"]
            d = vgpu[tg] - o["v"]
            rms = float(np.sqrt(np.mean(np.sum(d ** 2, 1)) / np.mean(np.sum(o["v"] ** 2, 1))))
            mx = float(np.max(np.linalg.norm(d, axis=1) / np.linalg.norm(o["v"], axis=1)))
            eps_v, _ = B.bs_error_estimate(p, float(o["geom"].lp.sum()))
            vrms = float(np.sqrt(np.mean(np.sum(o["v"] ** 2, 1))))
            accuracy = {"rms_rel_err": rms, "max_rel_err": mx, "targets": int(tg.size),
                        "eps_v_over_vrms": eps_v / vrms, "against": "FP64 CPU oracle (converged Ewald sum)"}
            cpu = {"value": f.N / o["full_s"], "unit": UNIT, "cores": o["threads"], "kind": "oracle",
                   "sample": (f"{tg.size} random target nodes of the {f.N}-node workload timed in full "
                              f"({o['sample_s']:.1f} s: spline fit, Fourier coefficients of all sources, "
                              f"27-image short range); full evaluation extrapolated as fixed "
                              f"{o['fixed_s']:.2f} s + N x {o['per_target_s'] * 1e3:.2f} ms")}
        launches = KERNELS_PER_STEP * args.steps
        result = {
            "metric": METRIC, "value": whole_job_rate(f.N, world, ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == B.BS_MIXED else "f64",
            "data": "synthetic (seeded random-phase Fourier tangles, no dataset)",
            "config": {"workload": f"{args.workload}: {f.nfil} closed filaments x {f.N // max(f.nfil, 1)} nodes, "
                                   f"N={f.N}, L=2pi, M={spec['M']}^3 modes, beta={spec['beta']}",
                       "precision": "mixed: f32 kernels, f64 positions/offsets and final sum"
                       if prec == B.BS_MIXED else "f64",
                       "N": f.N, "nfil": f.nfil, "M": spec["M"], "n_g": ng, "Q": spec["Q"], "w": p.nufft_w,
                       "sigma": spec["sigma"], "beta": spec["beta"], "alpha": p.alpha, "rc": p.rc,
                       "l2": "512 MiB L2 flush between timed steps (outside the events)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": "k_spread_zfft", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": ncu_traffic("k_spread_zfft", args.workload, "paper_2406_07366_gb300/csrc/k_fft.cu")
                         if prec == B.BS_MIXED else None,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)",
                         "algorithmic_bytes": sb, "ms": stage_mean["spread"]},
            "cpu_baseline": cpu,
            "e2e": {"value": whole_job_rate(f.N, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(f.N * 24),
                    "d2h_bytes_per_step": int(f.N * 24), "ms_per_step": e2e_s * 1e3,
                    "api": "bs_compute_host (pinned host buffers)"},
            "gpu_launches": launches,
            "ms_per_step_graph_replay": statistics.median(graph_ms),
            "clocks": clk,
            "stages_ms": stage_mean,
            "stage_roofline": stage_roof,
            "short_range": short,
            "fma_peak": fma_peak,
            "fp64_form": fp64,
            "batched_form": batched,
            "large_form": large,
            "autotuned": autotuned,
            "accuracy": accuracy,
        }
    bs.close()
    return result


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args):
    """The oracle as the reference arm: its fixed work (spline fit, Fourier
    coefficients of all sources) is timed once; each step then evaluates a
    fresh random sample of targets in full (all sources, 27 images), and the
    full-evaluation rate is N / (fixed + N x mean per-target time)."""
    spec, f = workload(args.workload)
    n = max(1, min(args.cpu_sample // 2, 8))
    fx = oracle_fixed(f, spec)
    rng = np.random.default_rng(1234)
    for _ in range(args.warmup):
        oracle_targets(f, spec, fx, np.sort(rng.choice(f.N, n, replace=False)))
    per = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, tt = oracle_targets(f, spec, fx, np.sort(rng.choice(f.N, n, replace=False)))
        per.append(tt / n)
    wall = time.perf_counter() - t0
    full = fx["fixed_s"] + statistics.mean(per) * f.N
    v = f.N / full
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": full * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random-phase Fourier tangles)",
            "impl": "reference",
            "config": {"workload": args.workload, "N": f.N, "M": spec["M"]},
            "cpu_baseline": {"kind": "oracle", "cores": fx["threads"], "value": v, "unit": UNIT,
                             "sample": (f"fixed work once ({fx['fixed_s']:.1f} s: spline fit + Fourier coefficients "
                                        f"of all {f.N * spec['Q']} sources); each of {args.steps} steps: {n} random "
                                        f"targets in full ({wall:.1f} s total); ms_per_step = extrapolated full "
                                        f"evaluation")},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)), flush=True)
        return 0
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    res = run_ours(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
