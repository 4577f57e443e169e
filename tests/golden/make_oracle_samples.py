"""Write the converged-oracle velocities of sampled nodes of the benchmarked
workloads, so that the GPU tests and the benchmark can check the full-size
evaluations without re-running the oracle over every source each time.

    python tests/golden/make_oracle_samples.py [tangle1e5|tangle4e6|tangle_batch ...]

Each output file tests/golden/oracle_<workload>.json holds the sampled node
indices, the velocities there from ``oracle.velocity_converged`` (the
quadrature-discretised periodic Biot-Savart sum with the oracle's own
converged Ewald split: 27 images, mode cube K_o, Sec. 3 Eq.
ewald_velocity_splitting), a checksum of the generated nodes (so a reader
can tell that the seeded generator still draws the same curves), and the
command that wrote it.  Only ``oracle`` and the seeded input generators are
used; nothing here touches the CUDA library.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2406_07366_gb300 import workloads as W  # noqa: E402

KAPPA, A_CORE, DELTA = 1.0, 1e-6, 0.25
# sampled nodes per workload (per member for the batch) and the sampling seed
SAMPLES = {"tangle1e5": (256, 11), "tangle4e6": (256, 12), "tangle_batch": (32, 13)}


def node_checksum(nodes):
    """Sum of |x| over the nodes and the sum of x weighted by the row index
    mod 97: both change if the generator draws different curves."""
    x = np.asarray(nodes, dtype=np.float64)
    w = (np.arange(x.shape[0]) % 97).astype(np.float64)
    return [float(np.abs(x).sum()), float((w[:, None] * x).sum())]


def sample(f, Q, n, seed):
    rng = np.random.default_rng(seed)
    tg = np.sort(rng.choice(f.N, min(n, f.N), replace=False))
    g = oracle.geometry(f.nodes, f.offsets, f.closing, f.L, 4, Q)
    v, _ = oracle.velocity_converged(g, f.L, KAPPA, A_CORE, DELTA, targets=tg)
    return tg, v


def write(name):
    n, seed = SAMPLES[name]
    t0 = time.time()
    if name == "tangle_batch":
        fs = W.tangle_batch(nconf=64, seed=5)
        members = []
        for i, f in enumerate(fs):
            tg, v = sample(f, 2, n, seed + i)
            members.append({"N": f.N, "targets": tg.tolist(), "velocity": v.tolist(),
                            "nodes_checksum": node_checksum(f.nodes)})
        doc = {"workload": "tangle_batch: 64 Fourier tangles, W.tangle_batch(nconf=64, seed=5)", "Q": 2,
               "members": members}
    else:
        spec = W.WORKLOADS[name]
        f = spec["gen"]()
        tg, v = sample(f, spec["Q"], n, seed)
        doc = {"workload": name, "N": f.N, "Q": spec["Q"], "targets": tg.tolist(), "velocity": v.tolist(),
               "nodes_checksum": node_checksum(f.nodes)}
    doc["_doc"] = ("Converged-oracle velocities (oracle.velocity_converged: beta_o = 6, 27 images, mode cube K_o; "
                   "kappa = 1, a = 1e-6, Delta = 1/4, cubic splines) at sampled nodes of the seeded workload.")
    doc["command"] = f"python tests/golden/make_oracle_samples.py {name}"
    doc["oracle_threads"] = oracle.get_threads()
    doc["oracle_seconds"] = round(time.time() - t0, 1)
    with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as fh:
        json.dump(doc, fh, separators=(",", ":"))
    print(name, "written in", doc["oracle_seconds"], "s", flush=True)


def load(name):
    """The stored samples of a workload (None if the file is absent)."""
    path = os.path.join(HERE, f"oracle_{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        return json.load(fh)


if __name__ == "__main__":
    oracle.build()
    for nm in (sys.argv[1:] or list(SAMPLES)):
        write(nm)
