#!/usr/bin/env python
"""Throughput of the Ewald-split periodic Biot-Savart velocity evaluation.

One step = one full evaluation (bs_compute) of the velocity at every node
of the workload: spline fit, quadrature sources, short range, long range
(spread, FFT, k-space, FFT^-1, interpolation) and local / self terms.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl ours|reference]

The headline workload is the largest single-GPU one, tangle4e6 (20000
filaments x 200 nodes, M = 512 modes, 768^3 spread grid, float32 kernels).
The same line carries the float64 form on that workload, the 1e5-node
tangle, the 64-tangle batch and RK4 stepping, each with its accuracy against
stored converged-oracle samples (tests/golden/oracle_<workload>.json).

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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="tangle4e6")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="oracle targets timed for cpu_baseline (0: four per host thread)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--no-batched-form", action="store_true")
    ap.add_argument("--no-large-form", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 1e5-node tangle forms")
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
    return B.workload_params(spec, f.L, precision, flags)


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


def golden(name):
    """Stored converged-oracle velocities at sampled nodes of a workload
    (tests/golden/make_oracle_samples.py), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        return json.load(fh)


def rel_errors(v, vr):
    """rms relative error (Sec. 5.1, Eq. def_relative_errors) and the largest
    per-node relative error."""
    d = v - vr
    rms = float(np.sqrt(np.mean(np.sum(d ** 2, 1)) / np.mean(np.sum(vr ** 2, 1))))
    mx = float(np.max(np.linalg.norm(d, axis=1) / np.linalg.norm(vr, axis=1)))
    return rms, mx


def polygon_length(f):
    nxt = np.arange(f.N) + 1
    nxt[f.offsets[1:] - 1] = f.offsets[:-1]
    return float(np.linalg.norm(f.nodes[nxt] - f.nodes, axis=1).sum())


def accuracy_of(B, name, f, p, vel):
    """Accuracy of one evaluation (vel: host array, N x 3) against the stored
    oracle samples of the workload, next to the Sec. 4 estimate."""
    doc = golden(name)
    if doc is None:
        return None
    tg = np.asarray(doc["targets"], dtype=np.int64)
    vr = np.asarray(doc["velocity"])
    rms, mx = rel_errors(vel[tg], vr)
    eps_v, _ = B.bs_error_estimate(p, polygon_length(f))
    vrms = float(np.sqrt(np.mean(np.sum(vr ** 2, 1))))
    return {"rms_rel_err": rms, "max_rel_err": mx, "targets": int(tg.size), "eps_v_over_vrms": eps_v / vrms,
            "against": "converged FP64 CPU oracle at sampled nodes (tests/golden/oracle_%s.json)" % name}


def time_form(B, stream, flush, spec, f, nodes, prec, steps, graph=False):
    """Mean CUDA-event milliseconds of `steps` evaluations of a workload in one
    precision (after two untimed ones), and the last velocity (host)."""
    import torch
    p = make_params(B, spec, f, prec)
    bs = B.BiotSavart(p, f.offsets, f.closing, stream=stream)
    vel = torch.empty_like(nodes)
    if graph:
        bs.capture(nodes, vel)
        run = bs.launch
    else:
        def run():
            bs.velocity(nodes, vel)
    for _ in range(2):
        run()
    bs.status()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    bs.status()
    out = vel.cpu().numpy()
    bs.close()
    del vel
    return statistics.mean(ms), out, p


def run_batched_form(B, dev, stream, flush, steps, nconf=64, lo=3.0, hi=5.0, N_l=100, gold="tangle_batch"):
    """The batched form: nconf independent Fourier tangles with node counts
    log-uniform in [10^lo, 10^hi] (N_l nodes per filament), grids matched to
    k_max (alpha = C_beta N^(1/3)/L, M in [32, 128]), mixed precision, the
    whole batch replayed from one CUDA graph per evaluation."""
    import torch
    from paper_2406_07366_gb300 import workloads as W
    fs = W.tangle_batch(nconf=nconf, seed=5, lo=lo, hi=hi, N_l=N_l)
    params = B.tangle_batch_params(fs, B.BS_MIXED)
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
    v = vel.cpu().numpy()
    off = bt.offsets
    nst = int(bt.staged.sum())
    bt.close()
    t = statistics.mean(ms)
    Ms = sorted(p.M[0] for p in params)
    out = {"value": bt.N / (t * 1e-3), "ms_per_step": t, "steps": steps, "nconf": len(fs), "N_total": bt.N,
           "N_range": [min(f.N for f in fs), max(f.N for f in fs)], "M_range": [Ms[0], Ms[-1]],
           "staged_members": nst,
           "issue": "one CUDA graph per evaluation: members of <= 2048 nodes share one launch per stage, "
                    "the others on 8 concurrent streams"}
    doc = golden(gold) if gold else None
    if doc is not None:
        errs, mxs = [], []
        for i, m in enumerate(doc["members"]):
            tg = np.asarray(m["targets"], dtype=np.int64)
            r, x = rel_errors(v[off[i]:off[i + 1]][tg], np.asarray(m["velocity"]))
            errs.append(r)
            mxs.append(x)
        out["accuracy"] = {"worst_member_rms_rel_err": max(errs), "median_member_rms_rel_err": statistics.median(errs),
                           "max_rel_err": max(mxs), "targets_per_member": len(doc["members"][0]["targets"]),
                           "against": "converged FP64 CPU oracle at sampled nodes (tests/golden/oracle_tangle_batch.json)"}
    return out


def run_autotuned(B, dev, spec, f, prec, cands=(1.0, 1.25, 1.5, 1.71, 2.0)):
    """Sec. 5.3's alpha = C_beta N^(1/3) / L re-chosen by timing on this GPU at
    the same beta (accuracy): C_beta candidates around the paper's 1.71."""
    import torch
    base = make_params(B, spec, f, prec)
    nodes = torch.from_numpy(f.nodes).to(dev)
    cands = list(cands)
    best, ms = B.bs_autotune_alpha(base, f.offsets, f.closing, nodes, cands, reps=3)
    i = min((k for k in range(len(ms)) if ms[k] > 0), key=lambda k: ms[k])
    eps_v, _ = B.bs_error_estimate(best, polygon_length(f))
    return {"candidates_C_beta": cands, "ms": ms, "best_C_beta": cands[i], "M": list(best.M), "alpha": best.alpha,
            "rc": best.rc, "value": f.N / (ms[i] * 1e-3), "unit": UNIT, "eps_v": eps_v,
            "note": "beta = 3.5 kept; the headline keeps the workload's M"}


def run_tile_autotune(B, dev, spec, f, prec):
    """bs_autotune_tiles on the workload: z-column blocks (block_x x block_y
    columns, threads per CTA) and short-range cells per cut-off (m), timed on
    this GPU; the library default is candidate 0."""
    import torch
    base = make_params(B, spec, f, prec)
    nodes = torch.from_numpy(f.nodes).to(dev)
    cands = [(0, 0, 0, 0), (2, 4, 512, 3), (2, 4, 512, 1), (4, 2, 512, 2), (4, 4, 512, 2), (2, 4, 256, 2),
             (2, 2, 256, 2)]
    best, ms = B.bs_autotune_tiles(base, f.offsets, f.closing, nodes, cands, reps=3)
    i = min((k for k in range(len(ms)) if ms[k] > 0), key=lambda k: ms[k])
    return {"candidates": [list(c) for c in cands], "fields": "block_x, block_y, block_threads, cell_div (0 = default)",
            "ms": ms, "best": list(cands[i]), "default_ms": ms[0], "best_ms": ms[i],
            "note": "the method and its accuracy are unchanged; the headline uses the library default"}


def polygon_impulse(nodes, offsets, kappa=1.0):
    """(kappa/2) sum over the closed polygons of s_j x s_{j+1} (host diagnostic)."""
    x = nodes.reshape(-1, 3)
    nxt = np.arange(x.shape[0]) + 1
    nxt[offsets[1:] - 1] = offsets[:-1]
    return 0.5 * kappa * np.cross(x, x[nxt]).sum(axis=0)


def run_rk4(B, dev, stream, spec, f, rk_steps):
    """rk_steps RK4 steps of the workload (Sec. 5.2, dt = Kelvin-wave period at
    the smallest node spacing) replayed from the captured step, mixed
    precision, with the energy (float64 evaluation) and impulse drift."""
    import torch
    p = make_params(B, spec, f, B.BS_MIXED)
    bs = B.BiotSavart(p, f.offsets, f.closing, stream=stream)
    nodes = torch.from_numpy(f.nodes).to(dev)
    seg = []
    for l in range(f.nfil):
        s = f.nodes[f.offsets[l]:f.offsets[l + 1]]
        seg.append(np.linalg.norm(np.roll(s, -1, axis=0) - s, axis=1).min())
    dt = B.kelvin_wave_period(min(seg), spec["kappa"], spec["a"], spec["delta"])
    # the energies come from a float64 evaluation, so that the drift is the
    # motion's and not the float32 evaluation noise
    b64 = B.BiotSavart(make_params(B, spec, f, B.BS_FP64, flags=B.BS_WANT_PSI), f.offsets, f.closing, stream=stream)
    E0 = b64.energy(nodes)
    P0 = polygon_impulse(f.nodes, f.offsets, spec["kappa"])
    bs.rk4_capture(nodes, dt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bs.rk4_launch(rk_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    rk_ms = e0.elapsed_time(e1)
    bs.status()
    E1 = b64.energy(nodes)
    b64.close()
    x1 = nodes.cpu().numpy()
    P1 = polygon_impulse(x1, f.offsets, spec["kappa"])
    bs.close()
    return {"steps": rk_steps, "dt": dt, "ms": rk_ms, "ms_per_step": rk_ms / rk_steps,
            "evaluations_per_s": 4 * rk_steps / (rk_ms * 1e-3),
            "energy_rel_drift": (E1 - E0) / E0, "energy_eval": "float64 form",
            "impulse_rel_drift": float(np.linalg.norm(P1 - P0) / np.linalg.norm(P0)),
            "max_node_displacement": float(np.abs(x1 - f.nodes).max())}


def run_leapfrog(B, dev, nsteps=1000):
    """Sec. 5.2's conservation run in the paper's production setting: two
    leapfrogging elliptical rings (32 and 64 nodes each), quintic curves,
    Q = 3, subdivided local segments (f = 0.1), beta = 3.5, alpha = 7/L,
    float64, RK4 with the Kelvin-wave step; the largest relative change of
    the energy (every nsteps/10 steps) and the change of the impulse
    (kappa/2) oint s x ds on the spline."""
    import torch
    from paper_2406_07366_gb300 import workloads as W
    out = {}
    for N_l in (32, 64):
        f = W.leapfrog_ellipses(N_l=N_l)
        L = float(f.L[0])
        alpha = 7.0 / L
        K = int(math.ceil(3.5 * alpha * L / math.pi))
        p = B.make_params(f.L, kappa=1.0, a=1e-6, delta=0.25, order=6, Q=3, M=2 * K + 1, w=8,
                          precision=B.BS_FP64, alpha=alpha, flags=B.BS_WANT_PSI, local_frac=0.1)
        nodes = torch.from_numpy(f.nodes.copy()).to(dev)
        dmin = min(np.linalg.norm(np.roll(f.nodes[f.offsets[l]:f.offsets[l + 1]], -1, axis=0)
                                  - f.nodes[f.offsets[l]:f.offsets[l + 1]], axis=1).min() for l in range(f.nfil))
        dt = B.kelvin_wave_period(dmin, 1.0, 1e-6, 0.25)
        s = torch.cuda.Stream(device=dev)
        bs = B.BiotSavart(p, f.offsets, f.closing, stream=s)
        def impulse():
            # (kappa/2) oint s x ds on the spline: sum over the quadrature points
            # of s_q x q_q, each point at the image nearest its node
            qX, qq = bs.quadrature(nodes)
            x = nodes.cpu().numpy()
            qX, qq = qX.cpu().numpy(), qq.cpu().numpy()
            xn = np.repeat(x, 3, axis=0)
            qX = qX - f.L[None, :] * np.round((qX - xn) / f.L[None, :])
            return 0.5 * np.cross(qX, qq).sum(axis=0)
        with torch.cuda.stream(s):
            E0 = bs.energy(nodes)
            P0 = impulse()
            Es = [E0]
            bs.rk4_capture(nodes, dt)
            for _ in range(10):
                bs.rk4_launch(nsteps // 10)
                bs.status()
                Es.append(bs.energy(nodes))
            x1 = nodes.cpu().numpy()
            P1 = impulse()
        bs.close()
        out[f"N_l={N_l}"] = {"steps": nsteps, "dt": dt, "time": nsteps * dt,
                             "energy_max_rel_change": float(max(abs(e - E0) for e in Es) / abs(E0)),
                             "impulse_rel_change": float(np.linalg.norm(P1 - P0) / np.linalg.norm(P0)),
                             "max_node_displacement": float(np.abs(x1 - f.nodes).max())}
    out["setting"] = ("two leapfrogging elliptical rings, quintic curves, Q = 3, local segments subdivided "
                      "(f = 0.1), beta = 3.5, alpha = 7/L, float64, RK4 at the Kelvin-wave step")
    out["paper"] = "energy and impulse variations within 1e-6 (Sec. 5.2)"
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


def oracle_subset(f, nfil_sub):
    """The first nfil_sub filaments of a workload (the same curves and sizes),
    the source sample on which the oracle is timed."""
    from paper_2406_07366_gb300 import workloads as W
    k = min(int(nfil_sub), f.nfil)
    off = f.offsets[:k + 1].copy()
    return W.Filaments(f.nodes[:off[-1]].copy(), off, f.closing[:k].copy(), f.L.copy(), f.name + f"[:{k}]")


def oracle_fixed(f, spec, nfil_sub):
    """Time the oracle's per-evaluation fixed work on a sample of filaments:
    the spline fit and quadrature (per filament) and the Fourier coefficients
    (per source, over the oracle's mode cube); both scale linearly, so the
    full evaluation's share is the sample's times nfil / nfil_sub."""
    import oracle
    fs = oracle_subset(f, nfil_sub)
    t0 = time.perf_counter()
    g = oracle.geometry(fs.nodes, fs.offsets, fs.closing, fs.L, 4, spec["Q"])
    t_geom = time.perf_counter() - t0
    alpha, K = oracle.converged_params(f.L)
    t0 = time.perf_counter()
    om = oracle.fourier_coefs(g, f.L, spec["kappa"], K)
    t_coef = time.perf_counter() - t0
    scale = f.nfil / fs.nfil
    return dict(g=g, fs=fs, alpha=alpha, K=K, om=om, scale=scale, sample_s=t_geom + t_coef,
                fixed_s=(t_geom + t_coef) * scale, threads=oracle.get_threads())


def oracle_targets(f, spec, fx, tg):
    """Time the oracle's per-target work for targets tg of the sample: the
    short range over all sample sources and 27 images (scaled by NQ / NQ_sample
    to all sources: its cost per source is uniform), the Fourier synthesis
    over the oracle's modes, the self and local terms."""
    import oracle
    g = fx["g"]
    t0 = time.perf_counter()
    oracle.short_range(g, f.L, spec["kappa"], fx["alpha"], 0.0, all_images=True, targets=tg)
    t_short = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.fourier_eval(g, f.L, fx["alpha"], fx["K"], fx["om"], targets=tg)
    oracle.self_term(g, spec["kappa"], fx["alpha"], targets=tg)
    oracle.local(g, spec["kappa"], spec["a"], spec["delta"], targets=tg)
    t_rest = time.perf_counter() - t0
    return (t_short * fx["scale"] + t_rest) / tg.size, t_short + t_rest


def oracle_rate(f, spec, nfil_sub, n_targets, seed=0):
    """Nodes/s of a full oracle evaluation extrapolated from a bounded sample:
    fixed work on nfil_sub filaments, per-target work on n_targets targets."""
    fx = oracle_fixed(f, spec, nfil_sub)
    rng = np.random.default_rng(seed)
    tg = np.sort(rng.choice(fx["fs"].N, min(n_targets, fx["fs"].N), replace=False))
    per_target, tt = oracle_targets(f, spec, fx, tg)
    full = fx["fixed_s"] + per_target * f.N
    return dict(full_s=full, value=f.N / full, threads=fx["threads"], fixed_s=fx["fixed_s"], per_target_s=per_target,
                sample_s=fx["sample_s"] + tt, n_targets=int(tg.size), nfil_sub=fx["fs"].nfil)


# filaments of the oracle's timing sample per workload (about 1e5 nodes)
ORACLE_SUB = {"tangle4e6": 500, "tangle1e5": 1000}


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
    # the same evaluation replayed from a CUDA graph (context without stage events)
    graph_ms, _, _ = time_form(B, stream, flush, spec, f, nodes, prec, 10, graph=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = Clocks(dev.index if dev.index is not None else 0)
    clocks.start()
    stages = []
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
    vhead = vel.cpu().numpy()

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
    bs.close()
    del hn, hv

    extras = {}
    if world == 1:
        # the float64 form on the same workload (the metric's "vs FP64")
        if not args.no_fp64_form and prec == B.BS_MIXED:
            ms64, v64, p64 = time_form(B, stream, flush, spec, f, nodes, B.BS_FP64, 3)
            extras["fp64_form"] = {"value": f.N / (ms64 * 1e-3), "ms_per_step": ms64, "steps": 3,
                                   "nufft_w": p64.nufft_w, "accuracy": accuracy_of(B, args.workload, f, p64, v64)}
            torch.cuda.empty_cache()
            # the mixed form at w = 6: faster, inside the 1e-5 float32 budget in rms, not at 1e-6
            spec6 = dict(spec, w=6)
            ms6, v6, p6 = time_form(B, stream, flush, spec6, f, nodes, B.BS_MIXED, 10)
            extras["mixed_w6"] = {"value": f.N / (ms6 * 1e-3), "ms_per_step": ms6, "steps": 10,
                                  "nufft_w": p6.nufft_w, "accuracy": accuracy_of(B, args.workload, f, p6, v6)}
            torch.cuda.empty_cache()
        if not args.no_large_form and args.rk4_steps > 0:
            extras["rk4"] = run_rk4(B, dev, stream, spec, f, args.rk4_steps)
            torch.cuda.empty_cache()
            extras["leapfrog"] = run_leapfrog(B, dev)
        if not args.no_secondary and args.workload != "tangle1e5":
            s2, f2 = workload("tangle1e5")
            n2 = torch.from_numpy(f2.nodes).to(dev)
            msm, vm, pm = time_form(B, stream, flush, s2, f2, n2, B.BS_MIXED, 20)
            msd, vd, pd = time_form(B, stream, flush, s2, f2, n2, B.BS_FP64, 5)
            extras["tangle1e5"] = {
                "workload": "tangle1e5: 1000 closed filaments x 100 nodes, N=1e5, M=256^3 modes (384^3 grid)",
                "mixed": {"value": f2.N / (msm * 1e-3), "ms_per_step": msm, "nufft_w": pm.nufft_w,
                          "accuracy": accuracy_of(B, "tangle1e5", f2, pm, vm)},
                "fp64": {"value": f2.N / (msd * 1e-3), "ms_per_step": msd, "nufft_w": pd.nufft_w,
                         "accuracy": accuracy_of(B, "tangle1e5", f2, pd, vd)}}
            del n2
        if not args.no_batched_form:
            extras["batched_form"] = run_batched_form(B, dev, stream, flush, min(args.steps, 20))
            # many small members: the staged group's one launch per stage
            extras["batched_form_small"] = run_batched_form(B, dev, stream, flush, min(args.steps, 20), nconf=1024,
                                                            lo=2.4, hi=2.8, N_l=50, gold=None)
        if not args.no_autotune:
            extras["autotuned"] = run_autotuned(B, dev, spec, f, prec)
            extras["tiles_autotuned"] = run_tile_autotune(B, dev, spec, f, prec)

    result = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            n_t = args.cpu_sample or 4 * oracle.get_threads()
            o = oracle_rate(f, spec, ORACLE_SUB.get(args.workload, f.nfil), n_t)
            cpu = {"value": o["value"], "unit": UNIT, "cores": o["threads"], "kind": "oracle",
                   "sample": (f"timed on the first {o['nfil_sub']} of {f.nfil} filaments ({o['sample_s']:.1f} s): "
                              f"spline fit and Fourier coefficients of their sources, and {o['n_targets']} random "
                              f"targets in full over their sources (27 images, Fourier synthesis, self and local "
                              f"terms); fixed work scaled by the filament count, short range by the source "
                              f"count; full evaluation extrapolated as {o['fixed_s']:.1f} s + N x "
                              f"{o['per_target_s']:.3f} s"),
                   "ms_per_step_kind": "extrapolated full evaluation"}
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
                       "l2": "512 MiB L2 flush between timed steps (outside the events); the workspace is far "
                             "larger than L2",
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
            "ms_per_step_graph_replay": graph_ms,
            "clocks": clk,
            "stages_ms": stage_mean,
            "stage_roofline": stage_roof,
            "short_range": short,
            "fma_peak": fma_peak,
            "accuracy": accuracy_of(B, args.workload, f, p, vhead),
        }
        result.update(extras)
    return result


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args):
    """The oracle as the reference arm, timed like cpu_baseline: its fixed work
    (spline fit, Fourier coefficients) on a sample of filaments, scaled to the
    workload; each step then evaluates a fresh random sample of targets in full
    over the sample's sources, and the full-evaluation rate is
    N / (fixed + N x mean per-target time)."""
    import oracle
    spec, f = workload(args.workload)
    n = args.cpu_sample or oracle.get_threads()
    fx = oracle_fixed(f, spec, ORACLE_SUB.get(args.workload, f.nfil))
    rng = np.random.default_rng(1234)
    for _ in range(args.warmup):
        oracle_targets(f, spec, fx, np.sort(rng.choice(fx["fs"].N, n, replace=False)))
    per = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pt, _ = oracle_targets(f, spec, fx, np.sort(rng.choice(fx["fs"].N, n, replace=False)))
        per.append(pt)
    wall = time.perf_counter() - t0
    full = fx["fixed_s"] + statistics.mean(per) * f.N
    v = f.N / full
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": full * 1e3, "ms_per_step_kind": "extrapolated full evaluation",
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random-phase Fourier tangles, no dataset)",
            "impl": "reference",
            "config": {"workload": f"{args.workload}: {f.nfil} closed filaments x {f.N // max(f.nfil, 1)} nodes, "
                                   f"N={f.N}, L=2pi, M={spec['M']}^3 modes, beta={spec['beta']}",
                       "N": f.N, "M": spec["M"]},
            "cpu_baseline": {"kind": "oracle", "cores": fx["threads"], "value": v, "unit": UNIT,
                             "sample": (f"fixed work timed once on the first {fx['fs'].nfil} of {f.nfil} filaments "
                                        f"({fx['sample_s']:.1f} s, scaled by the filament count); each of "
                                        f"{args.steps} steps: {n} random targets in full over those filaments' "
                                        f"sources ({wall:.1f} s total, short range scaled by the source count); "
                                        f"ms_per_step = extrapolated full evaluation")},
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
