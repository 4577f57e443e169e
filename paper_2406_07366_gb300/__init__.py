"""GB300 (sm_103a) Ewald-split periodic Biot-Savart velocity on vortex filaments.

Thin ctypes binding of the C ABI in ``include/bsewald.h``: the functions
below carry the same names as the C entry points and only marshal
arguments; every step of the computation runs in the CUDA library
``lib/libbsewald.so``, loaded on the first call.  That call raises if the
library is missing: there is no CPU fallback.  PyTorch is used only for device memory
and streams (``BiotSavart`` takes and returns torch tensors).

Method: J. I. Polanco, "Fast and accurate evaluation of Biot-Savart
integrals over spatial curves in periodic domains", arXiv:2406.07366.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libbsewald.so")

BS_OK, BS_ERR_ARG, BS_ERR_RC_GT_HALF_L, BS_ERR_NET_VORTICITY, BS_ERR_SPLINE = 0, 1, 2, 3, 4
BS_ERR_NONFINITE, BS_ERR_OOM, BS_ERR_CUDA, BS_ERR_CUFFT, BS_ERR_TIMEOUT = 5, 6, 7, 8, 9
BS_ERR_STATE, BS_ERR_GEOMETRY = 10, 11
BS_FP64, BS_MIXED = 0, 1
BS_WANT_PSI, BS_TIMING, BS_FFT_CUFFT, BS_DETERMINISTIC = 1, 2, 4, 8
BS_SHORT_TILED, BS_SHORT_PER_NODE, BS_BATCH_PER_MEMBER, BS_BATCH_STAGED = 16, 32, 64, 128

STAGES = ["geometry", "sr_sort", "short_range", "lr_sort", "spread", "fft_fwd", "kspace", "fft_inv", "interp",
          "total"]

# Every exported symbol of include/bsewald.h.
EXPORTS = ["bs_params_from_beta", "bs_error_estimate", "bs_nufft_setup", "bs_create", "bs_set_stream",
           "bs_set_filaments", "bs_compute", "bs_compute_host", "bs_compute_parts", "bs_get_quadrature",
           "bs_status", "bs_stage_times", "bs_workspace_bytes", "bs_destroy", "bs_last_error",
           "bs_short_range_static", "bs_graph_capture", "bs_graph_launch", "bs_compute_energy",
           "bs_batch_create", "bs_batch_set", "bs_batch_node_offsets", "bs_batch_staged_members", "bs_batch_compute", "bs_batch_status",
           "bs_batch_member", "bs_batch_destroy", "bs_rk4_step", "bs_rk4_capture", "bs_rk4_launch",
           "bs_autotune_alpha", "bs_energy_spectrum", "bs_coarse_velocity", "bs_fma_peak", "bs_erfc_f32",
           "bs_autotune_tiles"]


class bs_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double * 3), ("kappa", ctypes.c_double), ("a", ctypes.c_double),
                ("delta", ctypes.c_double), ("alpha", ctypes.c_double), ("rc", ctypes.c_double),
                ("M", ctypes.c_int * 3), ("quad_Q", ctypes.c_int), ("spline_order", ctypes.c_int),
                ("nufft_sigma", ctypes.c_double), ("nufft_w", ctypes.c_int), ("precision", ctypes.c_int),
                ("flags", ctypes.c_int), ("cell_div", ctypes.c_int), ("local_frac", ctypes.c_double),
                ("block_x", ctypes.c_int), ("block_y", ctypes.c_int), ("block_threads", ctypes.c_int)]

    def as_dict(self):
        return dict(L=list(self.L), kappa=self.kappa, a=self.a, delta=self.delta, alpha=self.alpha, rc=self.rc,
                    M=list(self.M), quad_Q=self.quad_Q, spline_order=self.spline_order,
                    nufft_sigma=self.nufft_sigma, nufft_w=self.nufft_w, precision=self.precision,
                    flags=self.flags, cell_div=self.cell_div, local_frac=self.local_frac, block_x=self.block_x,
                    block_y=self.block_y, block_threads=self.block_threads)


class BSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bsewald error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    sig = {
        "bs_params_from_beta": ([ctypes.c_double, P(ctypes.c_double), ctypes.c_int, ctypes.c_longlong,
                                 P(bs_params)], ctypes.c_int),
        "bs_error_estimate": ([P(bs_params), ctypes.c_double, P(ctypes.c_double), P(ctypes.c_double)], ctypes.c_int),
        "bs_nufft_setup": ([P(bs_params), P(ctypes.c_int), P(ctypes.c_double)], ctypes.c_int),
        "bs_create": ([P(vp), P(bs_params), vp], ctypes.c_int),
        "bs_set_stream": ([vp, vp], ctypes.c_int),
        "bs_set_filaments": ([vp, ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int32)], ctypes.c_int),
        "bs_compute": ([vp, vp, vp, vp], ctypes.c_int),
        "bs_compute_host": ([vp, vp, vp, vp], ctypes.c_int),
        "bs_compute_parts": ([vp, vp, vp, vp], ctypes.c_int),
        "bs_get_quadrature": ([vp, vp, vp, vp], ctypes.c_int),
        "bs_status": ([vp], ctypes.c_int),
        "bs_stage_times": ([vp, P(ctypes.c_float), ctypes.c_int, P(ctypes.c_int)], ctypes.c_int),
        "bs_workspace_bytes": ([vp, P(ctypes.c_longlong)], ctypes.c_int),
        "bs_fma_peak": ([ctypes.c_int, P(ctypes.c_double)], ctypes.c_int),
        "bs_erfc_f32": ([ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "bs_destroy": ([vp], None),
        "bs_last_error": ([], ctypes.c_char_p),
        "bs_graph_capture": ([vp, vp, vp, vp], ctypes.c_int),
        "bs_compute_energy": ([vp, vp, vp, vp, P(ctypes.c_double)], ctypes.c_int),
        "bs_graph_launch": ([vp], ctypes.c_int),
        "bs_batch_create": ([P(vp), ctypes.c_int, P(bs_params), vp], ctypes.c_int),
        "bs_batch_set": ([vp, ctypes.c_int, ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int32)], ctypes.c_int),
        "bs_batch_node_offsets": ([vp, P(ctypes.c_int64)], ctypes.c_int),
        "bs_batch_staged_members": ([vp, P(ctypes.c_int32)], ctypes.c_int),
        "bs_batch_compute": ([vp, vp, vp], ctypes.c_int),
        "bs_batch_status": ([vp], ctypes.c_int),
        "bs_batch_member": ([vp, ctypes.c_int, P(vp)], ctypes.c_int),
        "bs_batch_destroy": ([vp], None),
        "bs_rk4_step": ([vp, vp, ctypes.c_double], ctypes.c_int),
        "bs_rk4_capture": ([vp, vp, ctypes.c_double], ctypes.c_int),
        "bs_rk4_launch": ([vp, ctypes.c_int], ctypes.c_int),
        "bs_coarse_velocity": ([vp, vp, vp, P(ctypes.c_int)], ctypes.c_int),
        "bs_energy_spectrum": ([vp, vp, ctypes.c_int, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double)],
                               ctypes.c_int),
        "bs_autotune_alpha": ([P(bs_params), ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int32), vp, ctypes.c_int,
                               P(ctypes.c_double), ctypes.c_int, P(bs_params), P(ctypes.c_float)], ctypes.c_int),
        "bs_autotune_tiles": ([P(bs_params), ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int32), vp, ctypes.c_int,
                               P(ctypes.c_int), ctypes.c_int, P(bs_params), P(ctypes.c_float)], ctypes.c_int),
        "bs_short_range_static": ([P(ctypes.c_double), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, vp, vp, vp, ctypes.c_int, vp, vp, vp, vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib_handle = None


def lib():
    """The loaded CUDA library (loaded on first use; raises if missing)."""
    global _lib_handle
    if _lib_handle is None:
        _lib_handle = _load()
    return _lib_handle


def _check(rc):
    if rc != BS_OK:
        raise BSError(rc, bs_last_error())
    return rc


def _ptr(x):
    """Device/host address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x)


# ------------------------------------------------------------- C entry points
def bs_last_error() -> str:
    return (lib().bs_last_error() or b"").decode()


def bs_params_from_beta(beta, L, M=0, N=0) -> bs_params:
    p = bs_params()
    Lc = (ctypes.c_double * 3)(*np.broadcast_to(np.asarray(L, dtype=float), (3,)))
    _check(lib().bs_params_from_beta(float(beta), Lc, int(M), int(N), ctypes.byref(p)))
    return p


def bs_error_estimate(p: bs_params, total_length: float):
    ev, ep = ctypes.c_double(), ctypes.c_double()
    _check(lib().bs_error_estimate(ctypes.byref(p), float(total_length), ctypes.byref(ev), ctypes.byref(ep)))
    return ev.value, ep.value


def bs_nufft_setup(p: bs_params, want_table=True):
    ng = (ctypes.c_int * 3)()
    K = [(m - 1) // 2 for m in p.M]
    tab = np.zeros(sum(k + 1 for k in K)) if want_table else None
    _check(lib().bs_nufft_setup(ctypes.byref(p), ng,
                               tab.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_table else None))
    if not want_table:
        return list(ng), None
    out, o = [], 0
    for k in K:
        out.append(tab[o:o + k + 1].copy())
        o += k + 1
    return list(ng), out


def bs_create(p: bs_params, stream=None):
    ctx = ctypes.c_void_p()
    _check(lib().bs_create(ctypes.byref(ctx), ctypes.byref(p), stream))
    return ctx


def bs_set_stream(ctx, stream):
    _check(lib().bs_set_stream(ctx, stream))


def bs_set_filaments(ctx, offsets, closing=None):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nfil = off.size - 1
    cl = None if closing is None else np.ascontiguousarray(closing, dtype=np.int32).reshape(nfil, 3)
    _check(lib().bs_set_filaments(ctx, nfil, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 None if cl is None else cl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))


def bs_compute(ctx, nodes, vel, psi=None):
    _check(lib().bs_compute(ctx, _ptr(nodes), _ptr(vel), _ptr(psi)))


def bs_compute_host(ctx, nodes, vel, psi=None):
    _check(lib().bs_compute_host(ctx, _ptr(nodes), _ptr(vel), _ptr(psi)))


def bs_compute_parts(ctx, nodes, parts, psi_parts=None):
    _check(lib().bs_compute_parts(ctx, _ptr(nodes), _ptr(parts), _ptr(psi_parts)))


def bs_get_quadrature(ctx, nodes, qX, qq):
    _check(lib().bs_get_quadrature(ctx, _ptr(nodes), _ptr(qX), _ptr(qq)))


def bs_compute_energy(ctx, nodes, vel=None, psi=None):
    e = ctypes.c_double()
    _check(lib().bs_compute_energy(ctx, _ptr(nodes), _ptr(vel), _ptr(psi), ctypes.byref(e)))
    return e.value


def bs_graph_capture(ctx, nodes, vel, psi=None):
    _check(lib().bs_graph_capture(ctx, _ptr(nodes), _ptr(vel), _ptr(psi)))


def bs_graph_launch(ctx):
    _check(lib().bs_graph_launch(ctx))


def bs_status(ctx):
    return _check(lib().bs_status(ctx))


def bs_rk4_step(ctx, nodes, dt):
    _check(lib().bs_rk4_step(ctx, _ptr(nodes), float(dt)))


def bs_rk4_capture(ctx, nodes, dt):
    _check(lib().bs_rk4_capture(ctx, _ptr(nodes), float(dt)))


def bs_rk4_launch(ctx, nsteps):
    _check(lib().bs_rk4_launch(ctx, int(nsteps)))


def bs_coarse_velocity(ctx, nodes, grid=None):
    """Grid shape (n0, n1, n2); with a device tensor ``grid`` (3 x n0 x n1 x n2
    float64) also fills it with the coarse-grained long-range velocity."""
    ng = (ctypes.c_int * 3)()
    _check(lib().bs_coarse_velocity(ctx, _ptr(nodes), _ptr(grid), ng))
    return tuple(ng)


def bs_energy_spectrum(ctx, nodes, nbins, smoothed=False):
    """(k_m, E(k_m)) for m = 0..nbins-1 (Eq. def_energy_spectrum)."""
    Ek = np.zeros(int(nbins), dtype=np.float64)
    dk = ctypes.c_double()
    _check(lib().bs_energy_spectrum(ctx, _ptr(nodes), int(bool(smoothed)), int(nbins),
                                   Ek.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(dk)))
    return dk.value * np.arange(int(nbins)), Ek


def bs_autotune_alpha(base, offsets, closing, nodes, cbeta, reps=3):
    """Time each candidate C_beta on these filaments; returns (best params, ms list)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nfil = off.size - 1
    cl = None if closing is None else np.ascontiguousarray(closing, dtype=np.int32).reshape(nfil, 3)
    cb = np.ascontiguousarray(cbeta, dtype=np.float64)
    ms = np.zeros(cb.size, dtype=np.float32)
    best = bs_params()
    _check(lib().bs_autotune_alpha(ctypes.byref(base), nfil, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  None if cl is None else cl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  _ptr(nodes), cb.size, cb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  int(reps), ctypes.byref(best), ms.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return best, [float(x) for x in ms]


def bs_autotune_tiles(base, offsets, closing, nodes, cand, reps=3):
    """Time each candidate (block_x, block_y, block_threads, cell_div) on these
    filaments; returns (best params, ms list, -1 for skipped candidates)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nfil = off.size - 1
    cl = None if closing is None else np.ascontiguousarray(closing, dtype=np.int32).reshape(nfil, 3)
    cd = np.ascontiguousarray(np.asarray(cand, dtype=np.int32).reshape(-1, 4))
    ms = np.zeros(cd.shape[0], dtype=np.float32)
    best = bs_params()
    _check(lib().bs_autotune_tiles(ctypes.byref(base), nfil, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  None if cl is None else cl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  _ptr(nodes), cd.shape[0], cd.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  int(reps), ctypes.byref(best), ms.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return best, [float(x) for x in ms]


def kelvin_wave_period(lam, kappa=1.0, a=1e-6, delta=0.25):
    """Period of a Kelvin wave of wavelength lam on a straight vortex
    (Sec. 5.2): T = (2 lam^2 / kappa) / [ln(lam / (pi a)) + 1/2 - (delta + gamma)],
    gamma the Euler-Mascheroni constant.  The paper's stable RK4 step is
    T at the smallest node spacing."""
    gamma = 0.57721566490153286061
    return 2.0 * lam * lam / kappa / (math.log(lam / (math.pi * a)) + 0.5 - (delta + gamma))


def bs_batch_create(params, stream=None):
    arr = (bs_params * len(params))(*params)
    b = ctypes.c_void_p()
    _check(lib().bs_batch_create(ctypes.byref(b), len(params), arr, stream))
    return b


def bs_batch_set(b, i, offsets, closing=None):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nfil = off.size - 1
    cl = None if closing is None else np.ascontiguousarray(closing, dtype=np.int32).reshape(nfil, 3)
    _check(lib().bs_batch_set(b, i, nfil, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             None if cl is None else cl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))


def bs_batch_node_offsets(b, nconf):
    off = np.zeros(nconf + 1, dtype=np.int64)
    _check(lib().bs_batch_node_offsets(b, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return off


def bs_batch_staged_members(b, nconf):
    st = np.zeros(nconf, dtype=np.int32)
    _check(lib().bs_batch_staged_members(b, st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return st.astype(bool)


def bs_batch_compute(b, nodes, vel):
    _check(lib().bs_batch_compute(b, _ptr(nodes), _ptr(vel)))


def bs_batch_status(b):
    return _check(lib().bs_batch_status(b))


def bs_batch_member(b, i):
    c = ctypes.c_void_p()
    _check(lib().bs_batch_member(b, i, ctypes.byref(c)))
    return c


def bs_batch_destroy(b):
    lib().bs_batch_destroy(b)


def bs_stage_times(ctx):
    ms = (ctypes.c_float * 16)()
    n = ctypes.c_int()
    _check(lib().bs_stage_times(ctx, ms, 16, ctypes.byref(n)))
    return {STAGES[i]: float(ms[i]) for i in range(n.value)}


def bs_fma_peak(precision):
    """Measured FMA throughput of the current device in flop/s (BS_FP64 or BS_MIXED = float32)."""
    f = ctypes.c_double()
    _check(lib().bs_fma_peak(int(precision), ctypes.byref(f)))
    return f.value


def bs_erfc_f32(x, out, stream=None):
    """The short-range kernels' float32 erfc at the device float32 tensor x,
    written to the device float32 tensor out (same length)."""
    import torch
    for t in (x, out):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise BSError(BS_ERR_ARG, "bs_erfc_f32: contiguous CUDA float32 tensors expected")
    if x.numel() != out.numel():
        raise BSError(BS_ERR_ARG, "bs_erfc_f32: x and out differ in length")
    if stream is None:
        stream = torch.cuda.current_stream(x.device).cuda_stream
    _check(lib().bs_erfc_f32(int(x.numel()), _ptr(x), _ptr(out), ctypes.c_void_p(stream)))


def bs_workspace_bytes(ctx):
    b = ctypes.c_longlong()
    _check(lib().bs_workspace_bytes(ctx, ctypes.byref(b)))
    return b.value


def bs_destroy(ctx):
    if ctx:
        lib().bs_destroy(ctx)


def bs_short_range_static(L, kappa, alpha, rc, src_pos, src_q, src_seg, tgt_pos, tgt_omit, vel, stream=None):
    """Short-range velocity sum with the library's fixed scratch (no device
    allocation; for callers that cannot allocate).  Arrays are contiguous device
    tensors on one device: src_pos, src_q (nsrc x 3 float64), src_seg (nsrc
    int32), tgt_pos (ntgt x 3 float64), tgt_omit (ntgt x 2 int32), vel (ntgt x 3
    float64, written); anything else raises BSError(BS_ERR_ARG) before the
    call.  stream: a torch stream or a cudaStream_t handle, default torch's
    current stream on that device."""
    import torch
    ns, nt = int(src_pos.shape[0]), int(tgt_pos.shape[0])
    want = ((src_pos, torch.float64, (ns, 3), "src_pos"), (src_q, torch.float64, (ns, 3), "src_q"),
            (src_seg, torch.int32, (ns,), "src_seg"), (tgt_pos, torch.float64, (nt, 3), "tgt_pos"),
            (tgt_omit, torch.int32, (nt, 2), "tgt_omit"), (vel, torch.float64, (nt, 3), "vel"))
    for t, dt, shape, name in want:
        # the kernels index these arrays by the counts taken from src_pos and
        # tgt_pos: a wrong dtype, shape or placement would read or write out
        # of bounds, so it is refused here
        if not isinstance(t, torch.Tensor) or t.dtype != dt or tuple(t.shape) != shape or not t.is_cuda \
                or not t.is_contiguous() or t.device != src_pos.device:
            raise BSError(BS_ERR_ARG, f"bs_short_range_static: {name} must be a contiguous CUDA {dt} tensor of "
                                      f"shape {shape} on {src_pos.device}")
    if stream is None:
        stream = torch.cuda.current_stream(src_pos.device).cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    Lc = (ctypes.c_double * 3)(*np.broadcast_to(np.asarray(L, dtype=float), (3,)))
    _check(lib().bs_short_range_static(Lc, float(kappa), float(alpha), float(rc), ns, _ptr(src_pos), _ptr(src_q),
                                       _ptr(src_seg), nt, _ptr(tgt_pos), _ptr(tgt_omit), _ptr(vel),
                                       ctypes.c_void_p(stream)))


# ------------------------------------------------------------- convenience
def make_params(L, kappa=1.0, a=1e-6, delta=0.25, beta=3.5, M=32, Q=2, order=4, sigma=1.5, w=8,
                precision=BS_FP64, flags=0, cell_div=0, alpha=None, rc=None, local_frac=0.0) -> bs_params:
    """Parameters from beta and M (Sec. 4): k_max = (2 pi/L) floor((M-1)/2),
    alpha = k_max / (2 beta), r_c = beta / alpha, unless alpha / rc are given."""
    p = bs_params_from_beta(beta, L, M=M)
    p.kappa, p.a, p.delta = kappa, a, delta
    p.quad_Q, p.spline_order = Q, order
    p.nufft_sigma, p.nufft_w = sigma, w
    p.precision, p.flags, p.cell_div = precision, flags, cell_div
    p.local_frac = local_frac
    if alpha is not None:
        p.alpha = alpha
        p.rc = beta / alpha if rc is None else rc
    elif rc is not None:
        p.rc = rc
    return p


def tangle_params(N, L, beta=3.5, M_min=32, M_max=128, **kw) -> bs_params:
    """Parameters of one member of a batch of tangles: alpha = C_beta N^(1/3) / L
    (Eq. alpha_optimal_performance, Table tab:performance), M the smallest odd
    count with k_max >= 2 beta alpha, clamped to [M_min, M_max], then alpha
    re-derived from k_max (so the accuracy coefficient stays beta)."""
    M = bs_params_from_beta(beta, L, M=0, N=int(N)).M[0]
    M = int(min(max(M, M_min), M_max))
    return make_params(L, beta=beta, M=M, **kw)


def workload_params(spec, L, precision=BS_MIXED, flags=0) -> bs_params:
    """Parameters of a named workload (a ``workloads.WORKLOADS`` entry): its
    beta, M, Q and sigma; the width w of the entry for the mixed form and at
    least 8 for the float64 form (Table tab:performance: w = 8 for 1e-6)."""
    w = spec["w"] if precision == BS_MIXED else max(spec["w"], 8)
    return make_params(L, kappa=spec["kappa"], a=spec["a"], delta=spec["delta"], beta=spec["beta"], M=spec["M"],
                       Q=spec["Q"], order=spec.get("order", 4), w=w, sigma=spec["sigma"], precision=precision,
                       flags=flags)


def tangle_batch_params(filaments, precision=BS_MIXED, flags=0, w=8):
    """Parameters of the members of a batch of tangles: beta = 3.5, grids of
    32..128 modes matched to k_max (``tangle_params``), Q = 2, kernel width w
    (8: the 1e-6 setting of Table tab:performance, in both forms), sigma = 1.5."""
    return [tangle_params(f.N, f.L, beta=3.5, M_min=32, M_max=128, Q=2, w=w, sigma=1.5, precision=precision,
                          flags=flags) for f in filaments]


class BiotSavartBatch:
    """Independent configurations evaluated together (one CUDA graph per call
    pattern); node and velocity tensors hold the members back to back."""

    def __init__(self, params, filaments, stream=None):
        import torch
        self.torch = torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.params = list(params)
        self.b = bs_batch_create(self.params, ctypes.c_void_p(stream.cuda_stream))
        for i, f in enumerate(filaments):
            bs_batch_set(self.b, i, f.offsets, f.closing)
        self.offsets = bs_batch_node_offsets(self.b, len(self.params))
        self.staged = bs_batch_staged_members(self.b, len(self.params))
        self.N = int(self.offsets[-1])

    def velocity(self, nodes, vel=None):
        vel = self.torch.empty((self.N, 3), dtype=self.torch.float64, device="cuda") if vel is None else vel
        bs_batch_compute(self.b, nodes, vel)
        return vel

    def member(self, i):
        return bs_batch_member(self.b, i)

    def status(self):
        return bs_batch_status(self.b)

    def close(self):
        if self.b:
            bs_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BiotSavart:
    """Context holder working on torch tensors (device memory and streams only)."""

    def __init__(self, params: bs_params, offsets, closing=None, stream=None):
        import torch
        self.torch = torch
        self.params = params
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.ctx = bs_create(params, ctypes.c_void_p(stream.cuda_stream))
        bs_set_filaments(self.ctx, offsets, closing)
        self.N = int(np.asarray(offsets)[-1])

    def _out(self):
        return self.torch.empty((self.N, 3), dtype=self.torch.float64, device="cuda")

    def velocity(self, nodes, vel=None, psi=None, want_psi=False):
        vel = self._out() if vel is None else vel
        if want_psi and psi is None:
            psi = self._out()
        bs_compute(self.ctx, nodes, vel, psi)
        return (vel, psi) if want_psi else vel

    def parts(self, nodes, want_psi=False):
        parts = self.torch.empty((4, self.N, 3), dtype=self.torch.float64, device="cuda")
        pp = self.torch.empty((4, self.N, 3), dtype=self.torch.float64, device="cuda") if want_psi else None
        bs_compute_parts(self.ctx, nodes, parts, pp)
        return (parts, pp) if want_psi else parts

    def energy(self, nodes, vel=None, psi=None):
        """Kinetic energy (and optionally velocity / streamfunction) of one evaluation."""
        return bs_compute_energy(self.ctx, nodes, vel, psi)

    def coarse_velocity(self, nodes):
        """The long-range velocity on the spread grid, 3 x n0 x n1 x n2 float64."""
        shape = bs_coarse_velocity(self.ctx, None, None)
        grid = self.torch.empty((3,) + shape, dtype=self.torch.float64, device="cuda")
        bs_coarse_velocity(self.ctx, nodes, grid)
        return grid

    def energy_spectrum(self, nodes, nbins, smoothed=False):
        """(k, E(k)) on the context's Fourier modes (Eq. def_energy_spectrum)."""
        return bs_energy_spectrum(self.ctx, nodes, nbins, smoothed)

    def capture(self, nodes, vel, psi=None):
        """Capture one evaluation into a CUDA graph (replay with launch())."""
        bs_graph_capture(self.ctx, nodes, vel, psi)

    def launch(self):
        bs_graph_launch(self.ctx)

    def rk4_step(self, nodes, dt):
        """One RK4 step of the nodes in place."""
        bs_rk4_step(self.ctx, nodes, dt)

    def rk4_capture(self, nodes, dt):
        """Capture one in-place RK4 step into a CUDA graph (replay with rk4_launch)."""
        bs_rk4_capture(self.ctx, nodes, dt)

    def rk4_launch(self, nsteps):
        bs_rk4_launch(self.ctx, nsteps)

    def quadrature(self, nodes):
        Q = self.params.quad_Q
        qX = self.torch.empty((self.N * Q, 3), dtype=self.torch.float64, device="cuda")
        qq = self.torch.empty((self.N * Q, 3), dtype=self.torch.float64, device="cuda")
        bs_get_quadrature(self.ctx, nodes, qX, qq)
        return qX, qq

    def status(self):
        return bs_status(self.ctx)

    def stage_times(self):
        return bs_stage_times(self.ctx)

    def close(self):
        if self.ctx:
            bs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
