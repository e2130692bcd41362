"""Thin Python binding of libtomo (include/tomo.h).

Argument marshalling only: tensors become device pointers, the current torch
stream becomes the call's stream, numpy host arrays become host pointers.
Every computation runs in the library's CUDA kernels; there is no CPU or
eager fallback, and every call raises TomoError if the library or a GPU is
missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtomo.so")

DADMM_Q_NONE, DADMM_Q_KMEANS, DADMM_Q_JPEG = 0, 1, 2
MODE_BATCHED, MODE_PLAIN = 0, 1
NSTAT = 5
STAT_NAMES = ("gap2", "chg2", "nrm2", "res2", "bytes")

_lib = None


class TomoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libtomo error %d: %s" % (code, msg))
        self.code = code


class DadmmConfig(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("n_bins", C.c_int), ("n_angles", C.c_int), ("S", C.c_int), ("M", C.c_int),
        ("node_ang_ptr", C.c_void_p), ("node_ang", C.c_void_p), ("seg_row_ptr", C.c_void_p),
        ("adj", C.c_void_p), ("edge_q", C.c_void_p), ("home_q", C.c_void_p), ("eta1", C.c_void_p),
        ("eta2", C.c_double), ("rho", C.c_double), ("E1", C.c_int), ("E2", C.c_int),
        ("km_k", C.c_int), ("km_iters", C.c_int), ("jpeg_quality", C.c_int),
        ("seed", C.c_uint64), ("mode", C.c_int), ("max_stale", C.c_int), ("variant", C.c_int),
        ("tune", C.c_int),
    ]


class DadmmState(C.Structure):
    _fields_ = [("u", C.c_void_p), ("lam", C.c_void_p), ("xseg", C.c_void_p),
                ("hist", C.c_void_p), ("iter", C.c_void_p)]


SIGNATURES = {
    "tomo_last_error": (C.c_char_p, []),
    "tomo_version": (C.c_int, []),
    "tomo_geometry_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "tomo_geometry_destroy": (C.c_int, [C.c_void_p]),
    "tomo_project": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                               C.c_void_p, C.c_void_p]),
    "tomo_project_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                       C.c_void_p, C.c_void_p]),
    "tomo_backproject": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                   C.c_float, C.c_void_p]),
    "tomo_opnorm_workspace_size": (C.c_size_t, [C.c_void_p, C.c_int]),
    "tomo_opnorm_sq": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_uint64, C.c_void_p,
                                 C.c_size_t, C.c_void_p, C.c_void_p]),
    "quant_kmeans": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_uint64, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "quant_kmeans_key": (C.c_uint64, [C.c_uint64, C.c_int, C.c_int, C.c_int]),
    "quant_jpeg": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_void_p, C.c_void_p]),
    "quant_jpeg_entropy_bound": (C.c_size_t, [C.c_int, C.c_int]),
    "quant_jpeg_entropy_workspace_size": (C.c_size_t, [C.c_int, C.c_int]),
    "quant_jpeg_entropy": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p,
                                     C.c_void_p, C.c_size_t, C.c_void_p]),
    "dadmm_create": (C.c_int, [C.c_void_p, C.POINTER(DadmmConfig), C.c_void_p]),
    "dadmm_destroy": (C.c_int, [C.c_void_p]),
    "dadmm_ring_depth": (C.c_int, [C.c_void_p]),
    "dadmm_launch_shape": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dadmm_state_size": (C.c_size_t, [C.c_void_p]),
    "dadmm_state_init": (C.c_int, [C.c_void_p, C.POINTER(DadmmState), C.c_void_p]),
    "dadmm_workspace_size": (C.c_size_t, [C.c_void_p]),
    "dadmm_state_modified": (C.c_int, [C.c_void_p]),
    "dadmm_step": (C.c_int, [C.c_void_p, C.POINTER(DadmmState), C.c_void_p, C.c_int, C.c_void_p,
                             C.c_size_t, C.c_void_p, C.c_void_p]),
    "dadmm_home_view": (C.c_int, [C.c_void_p, C.POINTER(DadmmState), C.c_void_p, C.c_void_p]),
    "dadmm_step_lossy": (C.c_int, [C.c_void_p, C.POINTER(DadmmState), C.c_void_p, C.c_int, C.c_void_p,
                                   C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "tomo_lincomb": (C.c_int, [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tomo_dot": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tomo_sync_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tomo_selftest_wait": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "dadmm_sync_status": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dadmm_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "dadmm_num_phases": (C.c_int, [C.c_void_p]),
    "dadmm_phase_times": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "tomo_fp32_peak": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tomo_smem_peak": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p]),
    "tomo_geometry_plan": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "tomo_geometry_cache_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
}


def lib():
    """Load libtomo.so (built in-tree by paper_2410_06106_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TomoError(-2, "libtomo.so is not built (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise TomoError(rc, lib().tomo_last_error().decode())


def _require_cuda(*tensors):
    if not torch.cuda.is_available():
        raise TomoError(-2, "no CUDA device: libtomo has no CPU path")
    for t in tensors:
        if t is not None:
            if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
                raise TomoError(-1, "expected a contiguous float32 CUDA tensor")


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def fp32_peak(target_ms=50):
    """Measured FP32 FMA throughput of the current GPU (tomo_fp32_peak):
    {"scalar_tflops", "packed_tflops", "sm_mhz"}"""
    _require_cuda()
    v = (C.c_double * 3)()
    _check(lib().tomo_fp32_peak(int(target_ms), C.byref(v, 0), C.byref(v, 8), C.byref(v, 16), _stream()))
    return {"scalar_tflops": v[0], "packed_tflops": v[1], "sm_mhz": v[2]}


def smem_peak(target_ms=50):
    """Measured shared-memory load bandwidth of the current GPU in GB/s (tomo_smem_peak)"""
    _require_cuda()
    v = C.c_double()
    _check(lib().tomo_smem_peak(int(target_ms), C.byref(v), _stream()))
    return v.value


def _host_i32(a):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return arr, arr.ctypes.data_as(C.c_void_p)


class Geometry:
    """Parallel-beam geometry (N x N pixels, B bins, angles theta)."""

    def __init__(self, N, B, theta=None, A=None):
        if theta is None:
            A = int(A)
            th = None
        else:
            th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
            A = len(th)
        self.N, self.B, self.A = int(N), int(B), int(A)
        self._theta = th
        h = C.c_void_p()
        tp = th.ctypes.data_as(C.c_void_p) if th is not None else None
        _check(lib().tomo_geometry_create(self.N, self.B, self.A, tp, C.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().tomo_geometry_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sel(self, angle_idx):
        if angle_idx is None:
            return None, None, self.A
        arr, p = _host_i32(angle_idx)
        return arr, p, len(arr)

    def project(self, img, angle_idx=None, subtract=None, out=None):
        """img [..., N, N] -> sino [..., n_sel, B] (Eq. 4), minus `subtract`"""
        _require_cuda(img, subtract, out)
        lead = img.shape[:-2]
        batch = int(np.prod(lead)) if len(lead) else 1
        arr, p, n_sel = self._sel(angle_idx)
        if out is None:
            out = torch.empty(*lead, n_sel, self.B, device=img.device, dtype=torch.float32)
        _check(lib().tomo_project(self.handle, _ptr(img), _ptr(out), p, n_sel, batch, _ptr(subtract),
                                  _stream()))
        return out

    def backproject(self, sino, angle_idx=None, out=None, beta=0.0):
        """sino [..., n_sel, B] -> img [..., N, N] (P^T); out = beta out + P^T sino"""
        _require_cuda(sino, out)
        lead = sino.shape[:-2]
        batch = int(np.prod(lead)) if len(lead) else 1
        arr, p, n_sel = self._sel(angle_idx)
        if out is None:
            out = torch.empty(*lead, self.N, self.N, device=sino.device, dtype=torch.float32)
            beta = 0.0
        _check(lib().tomo_backproject(self.handle, _ptr(sino), _ptr(out), p, n_sel, batch, float(beta),
                                      _stream()))
        return out

    def sync_status(self):
        """raise TomoError if a device-side failure was recorded by an operator
        call on this geometry since the last check (synchronizes the stream)"""
        _check(lib().tomo_sync_status(self.handle, _stream()))

    def plan(self, angle_idx=None, batch=1):
        """build the work lists of a selection now (tomo_geometry_plan), so that
        the operator calls that use it allocate no device memory"""
        _require_cuda()
        arr, p, n_sel = self._sel(angle_idx)
        _check(lib().tomo_geometry_plan(self.handle, p, n_sel, int(batch)))

    def cache_stats(self):
        """{"allocs", "frees", "entries", "bytes"} of the geometry's work-list cache"""
        v = (C.c_int64 * 4)()
        _check(lib().tomo_geometry_cache_stats(self.handle, C.byref(v, 0), C.byref(v, 8), C.byref(v, 16),
                                               C.byref(v, 24)))
        return {"allocs": v[0], "frees": v[1], "entries": v[2], "bytes": v[3]}

    def opnorm_sq(self, angle_idx=None, iters=100, seed=1):
        """||P_sel||^2 by power iteration on the GPU"""
        _require_cuda()
        arr, p, n_sel = self._sel(angle_idx)
        nb = lib().tomo_opnorm_workspace_size(self.handle, n_sel)
        work = torch.empty(nb, dtype=torch.uint8, device="cuda")
        out = C.c_double()
        _check(lib().tomo_opnorm_sq(self.handle, p, n_sel, int(iters), int(seed), _ptr(work), nb,
                                    C.byref(out), _stream()))
        return out.value


def kmeans_key(seed, slice_, owner, iteration):
    return lib().quant_kmeans_key(int(seed), int(slice_), int(owner), int(iteration))


def quant_kmeans(x, k, iters, key, objective=False):
    """Algorithm 5 on a float32 CUDA vector -> (codes u8, centroids, deq, objective|None)"""
    _require_cuda(x)
    x = x.reshape(-1)
    n = x.numel()
    codes = torch.empty(n, dtype=torch.uint8, device=x.device)
    cent = torch.empty(k, dtype=torch.float32, device=x.device)
    deq = torch.empty(n, dtype=torch.float32, device=x.device)
    obj = torch.empty(iters + 1, dtype=torch.float64, device=x.device) if objective else None
    _check(lib().quant_kmeans(_ptr(x), n, int(k), int(iters), int(key), _ptr(codes), _ptr(cent), _ptr(deq),
                              _ptr(obj), _stream()))
    return codes, cent, deq, obj


def quant_jpeg(x, quality):
    """JPEG-style codec of a [rows, cols] float32 CUDA segment -> (coefs, lohi, deq, nnz)"""
    _require_cuda(x)
    rows, cols = x.shape
    coefs = torch.empty((rows // 8) * (cols // 8), 64, dtype=torch.int16, device=x.device)
    lohi = torch.empty(2, dtype=torch.float32, device=x.device)
    deq = torch.empty_like(x)
    nnz = torch.zeros(1, dtype=torch.int64, device=x.device)
    _check(lib().quant_jpeg(_ptr(x), rows, cols, int(quality), _ptr(coefs), _ptr(lohi), _ptr(deq), _ptr(nnz),
                            _stream()))
    return coefs, lohi, deq, nnz


def jpeg_entropy(coefs, rows, cols, stream=True):
    """Baseline Huffman entropy-coded segment of quantized blocks [nblk, 64]
    (CUDA int16, natural order, blocks in raster order of a rows x cols
    image). Returns the stuffed stream as bytes (stream=True) or its length"""
    if not torch.cuda.is_available():
        raise TomoError(-2, "no CUDA device: libtomo has no CPU path")
    if not coefs.is_cuda or coefs.dtype != torch.int16 or coefs.numel() != (rows // 8) * (cols // 8) * 64:
        raise TomoError(-1, "expected int16 CUDA coefficients [rows/8 * cols/8, 64]")
    coefs = coefs.contiguous()
    lib_ = lib()
    ws = torch.empty(lib_.quant_jpeg_entropy_workspace_size(rows, cols), dtype=torch.uint8, device=coefs.device)
    cap = lib_.quant_jpeg_entropy_bound(rows, cols)
    out = torch.empty(cap, dtype=torch.uint8, device=coefs.device) if stream else None
    n = torch.empty(1, dtype=torch.int64, device=coefs.device)
    _check(lib_.quant_jpeg_entropy(_ptr(coefs), rows, cols, _ptr(out), cap if stream else 0, _ptr(n),
                                   _ptr(ws), ws.numel(), _stream()))
    nb = int(n.item())
    if nb < 0:
        raise TomoError(-1, "coefficient outside the baseline JPEG range")
    return out[:nb].cpu().numpy().tobytes() if stream else nb


def lincomb(xs, coefs, out=None):
    """out = sum_j coefs[j] * xs[j] (CUDA float32 tensors of equal size, 1..4 terms)"""
    _require_cuda(*xs)
    k = len(xs)
    n = xs[0].numel()
    for t in xs:
        assert t.numel() == n
    if out is None:
        out = torch.empty_like(xs[0])
    ptrs = (C.c_void_p * k)(*[t.data_ptr() for t in xs])
    cf = (C.c_float * k)(*[float(c) for c in coefs])
    _check(lib().tomo_lincomb(n, k, ptrs, cf, _ptr(out), _stream()))
    return out


def dot(x, y, scratch=None):
    """FP64 dot product of two CUDA float32 tensors, as a 0-dim CUDA float64 tensor"""
    _require_cuda(x, y)
    assert x.numel() == y.numel()
    if scratch is None:
        scratch = torch.empty(257, dtype=torch.float64, device=x.device)
    _check(lib().tomo_dot(x.numel(), _ptr(x), _ptr(y), _ptr(scratch), _stream()))
    return scratch[0]


class DADMM:
    """Decentralized ADMM solver (Algorithm 4) over S slices x M nodes.

    `prob` is a problem dict as produced by synth.make_problem (geometry,
    partition, graph, quantizers, solver settings). The device state (u, lam,
    xseg, hist, iter) and the workspace are torch tensors owned by this object.
    """

    def __init__(self, prob, eta1, mode="batched", geometry=None, tune="auto"):
        """tune: launch shapes, "auto" (timed at the first step, cached per
        problem shape in the process), "wide", "narrow", "pairs" (slice pairs of
        both operators, even S), "quads" (projector items of 4 slices, S % 4
        == 0) or "widepairs" (quads with wide backprojector tiles in slice
        pairs); see dadmm_config"""
        g = prob["geometry"]
        self.N, self.B, self.A = g["N"], g["B"], g["A"]
        self.S, self.M = int(prob["S"]), int(prob["M"])
        self.geometry = geometry or Geometry(self.N, self.B, g["theta"])
        self._keep = {}

        def keep(name, a, dt):
            arr = np.ascontiguousarray(np.asarray(a, dtype=dt))
            self._keep[name] = arr
            return arr.ctypes.data_as(C.c_void_p)

        cfg = DadmmConfig()
        cfg.N, cfg.n_bins, cfg.n_angles, cfg.S, cfg.M = self.N, self.B, self.A, self.S, self.M
        cfg.node_ang_ptr = keep("nap", prob["node_ang_ptr"], np.int32)
        cfg.node_ang = keep("na", prob["node_ang"], np.int32)
        cfg.seg_row_ptr = keep("srp", prob["seg_row_ptr"], np.int32)
        cfg.adj = keep("adj", prob["adj"], np.int32)
        cfg.edge_q = keep("eq", prob["edge_q"], np.int32)
        cfg.home_q = keep("hq", prob["home_q"], np.int32)
        cfg.eta1 = keep("eta1", eta1, np.float64)
        cfg.eta2, cfg.rho = float(prob["eta2"]), float(prob["rho"])
        cfg.E1, cfg.E2 = int(prob["E1"]), int(prob["E2"])
        cfg.km_k, cfg.km_iters = int(prob["km_k"]), int(prob["km_iters"])
        cfg.jpeg_quality = int(prob["jpeg_quality"])
        cfg.seed = int(prob["seed"])
        cfg.mode = MODE_BATCHED if mode == "batched" else MODE_PLAIN
        cfg.max_stale = int(prob.get("max_stale", 0))
        self.variant = prob.get("variant", "segments")
        if self.variant not in ("segments", "consensus"):
            raise TomoError(-1, "variant must be 'segments' or 'consensus'")
        cfg.variant = 1 if self.variant == "consensus" else 0
        tunes = {"wide": 0, "auto": 1, "narrow": 2, "pairs": 3, "quads": 4, "widepairs": 5}
        if tune not in tunes:
            raise TomoError(-1, "tune must be 'auto', 'wide', 'narrow', 'pairs', 'quads' or 'widepairs'")
        cfg.tune = tunes[tune]
        self.mode = mode
        self.cfg = cfg
        h = C.c_void_p()
        _check(lib().dadmm_create(self.geometry.handle, C.byref(cfg), C.byref(h)))
        self.handle = h
        self.D = lib().dadmm_ring_depth(h)
        dev = torch.device("cuda")
        n = self.N * self.N
        self.u = torch.zeros(self.S, self.M, self.N, self.N, device=dev)
        self.lam = torch.zeros(self.S, self.M, self.N, self.N, device=dev)
        if self.variant == "consensus":  # every node's x, and the message planes of one exchange
            self.xseg = torch.zeros(self.S, self.M, self.N, self.N, device=dev)
            self.hist = torch.zeros(3, self.S, self.M, self.N, self.N, device=dev)
        else:
            self.xseg = torch.zeros(self.S, self.N, self.N, device=dev)
            self.hist = torch.zeros(self.D, 3, self.S, self.N, self.N, device=dev)
        self.iter = torch.zeros(1, dtype=torch.int32, device=dev)
        self.ws_bytes = lib().dadmm_workspace_size(h)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self._state = DadmmState(self.u.data_ptr(), self.lam.data_ptr(), self.xseg.data_ptr(),
                                 self.hist.data_ptr(), self.iter.data_ptr())
        del n

    def close(self):
        if getattr(self, "handle", None):
            lib().dadmm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        _check(lib().dadmm_state_init(self.handle, C.byref(self._state), _stream()))

    def step(self, sino, n_iters=1, stats=True, drop=None):
        """Run n_iters iterations on sino [S, A, B] (CUDA float32). Returns the
        statistics [n_iters, S, 5] (numpy) when stats=True (synchronizes).
        drop: optional [n_iters, M, M] (or [M, M] for every iteration) array,
        drop[i, s, m] != 0 when node m loses owner s's message in iteration i
        (needs max_stale > 0 in the problem)"""
        _require_cuda(sino)
        st = np.empty((n_iters, self.S, NSTAT), np.float64) if stats else None
        sp = st.ctypes.data_as(C.c_void_p) if stats else None
        if drop is None:
            _check(lib().dadmm_step(self.handle, C.byref(self._state), _ptr(sino), int(n_iters),
                                    _ptr(self.workspace), self.ws_bytes, sp, _stream()))
        else:
            d = np.asarray(drop, np.uint8)
            if d.ndim == 2:
                d = np.broadcast_to(d, (n_iters, self.M, self.M))
            d = np.ascontiguousarray(d)
            assert d.shape == (n_iters, self.M, self.M)
            _check(lib().dadmm_step_lossy(self.handle, C.byref(self._state), _ptr(sino), int(n_iters),
                                          d.ctypes.data_as(C.c_void_p), _ptr(self.workspace), self.ws_bytes, sp,
                                          _stream()))
        return st

    def sync_status(self):
        """raise TomoError if a device-side failure (bounded wait that gave up,
        non-finite statistics) was recorded since the last check"""
        _check(lib().dadmm_sync_status(self.handle, _ptr(self.workspace), self.ws_bytes, _stream()))

    def set_profiling(self, enable=True):
        _check(lib().dadmm_set_profiling(self.handle, int(bool(enable))))

    def phase_names(self):
        E1 = int(self.cfg.E1)
        names = []
        for e in range(E1):
            names += ["project_%d" % e, "backproject_ustep_%d" % e]
        return names + ["xstep", "kmeans", "jpeg", "dual", "stats"]

    def phase_times(self):
        """per-phase milliseconds of the most recent iteration (synchronizes)"""
        n = lib().dadmm_num_phases(self.handle)
        out = np.empty(n, np.float32)
        _check(lib().dadmm_phase_times(self.handle, out.ctypes.data_as(C.c_void_p), n))
        return out

    def home_view(self, out=None):
        out = out if out is not None else torch.empty(self.S, self.N, self.N, device="cuda")
        _check(lib().dadmm_home_view(self.handle, C.byref(self._state), _ptr(out), _stream()))
        return out

    def launch_shape(self):
        """(backprojector tile width, slices per batched backprojector item,
        bins of 4-angle projector items, slices per projector item) in use"""
        tx, sl, nb, ps = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(lib().dadmm_launch_shape(self.handle, C.byref(tx), C.byref(sl), C.byref(nb), C.byref(ps)))
        return tx.value, sl.value, nb.value, ps.value

    @property
    def k(self):
        return int(self.iter.item())

    def state_dict(self):
        """checkpoint of the full iteration state (bit-exact resume)"""
        return {"u": self.u.clone(), "lam": self.lam.clone(), "xseg": self.xseg.clone(),
                "hist": self.hist.clone(), "iter": self.iter.clone()}

    def load_state_dict(self, sd):
        for name in ("u", "lam", "xseg", "hist", "iter"):
            getattr(self, name).copy_(sd[name])
        _check(lib().dadmm_state_modified(self.handle))

    def load_state(self, u, lam, xseg, hist, k):
        """set the state from arrays (numpy or torch) in the oracle's layout"""
        for name, v in (("u", u), ("lam", lam), ("xseg", xseg), ("hist", hist)):
            getattr(self, name).copy_(torch.as_tensor(np.asarray(v, np.float32)))
        self.iter.fill_(int(k))
        _check(lib().dadmm_state_modified(self.handle))

    def reconstruct(self, sino_host, n_iters):
        """End-to-end call: host sinograms in, host reconstruction out.
        Copies [S, A, B] float32 host data to the device, runs n_iters
        iterations and returns the owners' home view [S, N, N] on the host."""
        pinned = sino_host if (isinstance(sino_host, torch.Tensor) and sino_host.is_pinned()) else \
            torch.as_tensor(np.asarray(sino_host, np.float32)).pin_memory()
        d = pinned.to("cuda", non_blocking=True)
        self.step(d, n_iters, stats=False)
        return self.home_view().to("cpu")
