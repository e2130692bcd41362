"""Python access to the FP64 CPU oracle (ctypes over liboracle.so).

TEST INFRASTRUCTURE: only tests/, the smoke check and the benchmark's
CPU-baseline leg import this package. It never imports the CUDA package and
the CUDA package never imports it.

Every function takes and returns numpy arrays; conversion to the C layouts
(float64 / float32 / int32, C-contiguous) happens here and nowhere else.
"""
import ctypes as C
import numpy as np

from . import build as _build

_lib = None

KIND_NONE, KIND_KMEANS, KIND_JPEG = 0, 1, 2
NSTAT = 5


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        d, i32, i64, u64 = C.c_double, C.c_int, C.c_int64, C.c_uint64
        p = C.c_void_p
        sig = {
            "orc_num_threads": (i32, []),
            "orc_set_num_threads": (None, [i32]),
            "orc_trig": (None, [i32, p, p, p]),
            "orc_chord": (d, [d, d, d, d, d]),
            "orc_project": (None, [i32, i32, p, p, i32, p, i32, p, p]),
            "orc_backproject": (None, [i32, i32, p, p, i32, p, i32, p, p]),
            "orc_project_rays": (None, [i32, i32, p, p, i32, p, p, p, p]),
            "orc_backproject_pixels": (None, [i32, i32, p, p, i32, p, p, i32, p, p]),
            "orc_opnorm_sq": (d, [i32, i32, p, p, i32, p, i32, u64]),
            "orc_alg2_node": (d, [i32, i32, p, p, i32, p, p, p, p, d, d, i32, p]),
            "orc_ctr": (None, [i32, i32, i32, p, p, i32, p, d, i32, p]),
            "orc_mix64": (u64, [u64]),
            "orc_kmeans_key": (u64, [u64, i32, i32, i32]),
            "orc_kmeans": (None, [p, i64, i32, i32, u64, p, p, p, p]),
            "orc_jpeg_qtable": (None, [i32, p]),
            "orc_dct8x8": (None, [p, p]),
            "orc_idct8x8": (None, [p, p]),
            "orc_jpeg": (i64, [p, i32, i32, i32, p, p, p]),
            "orc_jpeg_entropy": (i64, [p, i64, p]),
            "orc_jpeg_entropy_decode": (i32, [p, i64, i64, p]),
            "orc_huff_code": (None, [i32, i32, p, p]),
            "orc_zigzag": (None, [p]),
            "orc_relay_tables": (None, [i32, p, p, p]),
            "orc_consensus_iterate": (i32, [i32, i32, i32, i32, i32, p, p, p, p, p, p, p,
                                            d, p, i32, i32, i32, i32, u64, p, p, p, p, p, p]),
            "orc_dadmm_iterate": (i32, [i32, i32, i32, i32, i32, p, p, p, p, p, p, p, p,
                                        d, p, d, i32, i32, i32, i32, i32, u64, i32,
                                        p, p, p, p, p, p, p, p, p, p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    """threads of the oracle's parallel loops (results do not depend on it)"""
    lib().orc_set_num_threads(int(n))


def trig(theta):
    th = _f64(theta)
    c = np.empty_like(th)
    s = np.empty_like(th)
    lib().orc_trig(len(th), _ptr(th), _ptr(c), _ptr(s))
    return c, s


def chord(c, s, t, xc, yc):
    return lib().orc_chord(float(c), float(s), float(t), float(xc), float(yc))


class Geometry:
    """N x N pixels, B unit bins, angles theta (radians)."""

    def __init__(self, N, B, theta):
        self.N, self.B = int(N), int(B)
        self.theta = _f64(theta)
        self.A = len(self.theta)
        self.c, self.s = trig(self.theta)

    def _sel(self, aidx):
        return _i32(np.arange(self.A) if aidx is None else aidx)

    def project(self, img, aidx=None):
        """img [..., N, N] -> sino [..., nsel, B] (Eq. 4)"""
        img = _f64(img)
        lead = img.shape[:-2]
        batch = int(np.prod(lead)) if lead else 1
        sel = self._sel(aidx)
        out = np.empty(lead + (len(sel), self.B), np.float64)
        lib().orc_project(self.N, self.B, _ptr(self.c), _ptr(self.s), len(sel), _ptr(sel),
                          batch, _ptr(img), _ptr(out))
        return out

    def backproject(self, sino, aidx=None):
        """sino [..., nsel, B] -> img [..., N, N] (P^T)"""
        sino = _f64(sino)
        lead = sino.shape[:-2]
        batch = int(np.prod(lead)) if lead else 1
        sel = self._sel(aidx)
        assert sino.shape[-2] == len(sel)
        out = np.empty(lead + (self.N, self.N), np.float64)
        lib().orc_backproject(self.N, self.B, _ptr(self.c), _ptr(self.s), len(sel), _ptr(sel),
                              batch, _ptr(sino), _ptr(out))
        return out

    def project_rays(self, img, ray_a, ray_b):
        img = _f64(img)
        ra, rb = _i32(ray_a), _i32(ray_b)
        out = np.empty(len(ra), np.float64)
        lib().orc_project_rays(self.N, self.B, _ptr(self.c), _ptr(self.s), len(ra), _ptr(ra),
                               _ptr(rb), _ptr(img), _ptr(out))
        return out

    def backproject_pixels(self, sino, pix, aidx=None):
        sino = _f64(sino)
        sel = self._sel(aidx)
        px = _i32(pix)
        out = np.empty(len(px), np.float64)
        lib().orc_backproject_pixels(self.N, self.B, _ptr(self.c), _ptr(self.s), len(sel),
                                     _ptr(sel), _ptr(sino), len(px), _ptr(px), _ptr(out))
        return out

    def alg2_node(self, u, xview, lam, sino, aidx, rho, eta1, E1):
        """Algorithm 2 for one node (E1 steps from u, view and dual fixed):
        returns (u after the steps, residual norm^2 at the last step)"""
        uu = _f64(u).copy()
        sel = _i32(aidx)
        res = lib().orc_alg2_node(self.N, self.B, _ptr(self.c), _ptr(self.s), len(sel), _ptr(sel),
                                  _ptr(_f64(sino)), _ptr(_f64(xview)), _ptr(_f64(lam)), float(rho),
                                  float(eta1), int(E1), _ptr(uu))
        return uu, res

    def ctr(self, sino, eta, E, u0=None):
        """Algorithm 1: E steps u <- u - eta P^T (P u - d) over every angle, from u0
        (zero by default); sino [..., A, B] -> u [..., N, N]"""
        d = _f64(sino)
        lead = d.shape[:-2]
        batch = int(np.prod(lead)) if lead else 1
        u = np.zeros(lead + (self.N, self.N)) if u0 is None else _f64(u0).copy()
        lib().orc_ctr(self.N, self.B, self.A, _ptr(self.c), _ptr(self.s), batch, _ptr(d), float(eta), int(E),
                      _ptr(u))
        return u

    def opnorm_sq(self, aidx=None, iters=100, seed=1):
        sel = self._sel(aidx)
        return lib().orc_opnorm_sq(self.N, self.B, _ptr(self.c), _ptr(self.s), len(sel),
                                   _ptr(sel), int(iters), int(seed))


def mix64(z):
    return lib().orc_mix64(int(z) & 0xFFFFFFFFFFFFFFFF)


def kmeans_key(seed, slice_, owner, it):
    return lib().orc_kmeans_key(int(seed), int(slice_), int(owner), int(it))


def kmeans(v, k, iters, key):
    """Algorithm 5 -> (codes u8, centres f32, dequantized f32, objective f64[iters+1])"""
    v = _f32(v).ravel()
    codes = np.empty(v.size, np.uint8)
    cent = np.empty(k, np.float32)
    deq = np.empty(v.size, np.float32)
    obj = np.empty(iters + 1, np.float64)
    lib().orc_kmeans(_ptr(v), v.size, int(k), int(iters), int(key), _ptr(codes), _ptr(cent),
                     _ptr(deq), _ptr(obj))
    return codes, cent, deq, obj


def jpeg_qtable(quality):
    qt = np.empty(64, np.int32)
    lib().orc_jpeg_qtable(int(quality), _ptr(qt))
    return qt.reshape(8, 8)


def dct8x8(block):
    b = _f64(block).reshape(64)
    out = np.empty(64, np.float64)
    lib().orc_dct8x8(_ptr(b), _ptr(out))
    return out.reshape(8, 8)


def idct8x8(block):
    b = _f64(block).reshape(64)
    out = np.empty(64, np.float64)
    lib().orc_idct8x8(_ptr(b), _ptr(out))
    return out.reshape(8, 8)


def jpeg(v, quality):
    """JPEG-style codec of a [rows, cols] segment -> (coefs i16, lohi f32[2], deq f32, nnz)"""
    v = _f32(v)
    rows, cols = v.shape
    coefs = np.empty(((rows // 8) * (cols // 8), 64), np.int16)
    lohi = np.empty(2, np.float32)
    deq = np.empty_like(v)
    nnz = lib().orc_jpeg(_ptr(v), rows, cols, int(quality), _ptr(coefs), _ptr(lohi), _ptr(deq))
    return coefs, lohi, deq, int(nnz)


def jpeg_entropy(coefs):
    """baseline Huffman-coded bytes (stuffed, padded) of quantized blocks [nblk, 64]"""
    c = np.ascontiguousarray(coefs, np.int16).reshape(-1, 64)
    n = lib().orc_jpeg_entropy(_ptr(c), len(c), None)
    if n < 0:
        raise ValueError("coefficient outside the baseline range")
    out = np.empty(max(n, 1), np.uint8)
    lib().orc_jpeg_entropy(_ptr(c), len(c), _ptr(out))
    return out[:n].tobytes()


def jpeg_entropy_decode(data, nblk):
    buf = np.frombuffer(bytes(data), np.uint8).copy()
    out = np.empty((nblk, 64), np.int16)
    if lib().orc_jpeg_entropy_decode(_ptr(buf), len(buf), int(nblk), _ptr(out)) != 0:
        raise ValueError("malformed entropy-coded segment")
    return out


def huff_code(ac, symbol):
    """(code, length) of a DC category (ac=False) or AC run/size symbol"""
    code, ln = np.zeros(1, np.int32), np.zeros(1, np.int32)
    lib().orc_huff_code(int(bool(ac)), int(symbol), _ptr(code), _ptr(ln))
    return int(code[0]), int(ln[0])


def zigzag():
    zz = np.empty(64, np.int32)
    lib().orc_zigzag(_ptr(zz))
    return zz


def relay_tables(adj):
    a = _i32(adj)
    M = a.shape[0]
    dist = np.empty((M, M), np.int32)
    first = np.empty((M, M), np.int32)
    lib().orc_relay_tables(M, _ptr(a), _ptr(dist), _ptr(first))
    return dist, first


class DADMM:
    """Oracle state of S independent slices x M nodes (Algorithm 4).

    State arrays (float64): u, lam [S, M, N, N]; xseg [S, N, N];
    hist [D, 3, S, N, N]; k = completed iterations.
    """

    def __init__(self, prob, eta1, S=None):
        self.p = prob
        g = prob["geometry"]
        self.N, self.B, self.A = g["N"], g["B"], g["A"]
        self.M = prob["M"]
        self.S = prob["S"] if S is None else S
        self.theta = _f64(g["theta"])
        self.c, self.s = trig(self.theta)
        self.node_ang_ptr = _i32(prob["node_ang_ptr"])
        self.node_ang = _i32(prob["node_ang"])
        self.seg_row_ptr = _i32(prob["seg_row_ptr"])
        self.adj = _i32(prob["adj"])
        self.edge_q = _i32(prob["edge_q"])
        self.home_q = _i32(prob["home_q"])
        self.eta1 = _f64(eta1)
        dist, _ = relay_tables(self.adj)
        self.max_stale = int(prob.get("max_stale", 0))
        self.D = max(1, int(dist.max())) + 1 + self.max_stale  # max relay lag + 2 + staleness allowed
        self.lag = np.where(np.eye(self.M, dtype=bool), 0, dist - 1).astype(np.int32)  # [s, m]
        self.held = None  # versions held [s, m] once messages may be lost
        N, M, S = self.N, self.M, self.S
        self.u = np.zeros((S, M, N, N))
        self.lam = np.zeros((S, M, N, N))
        self.xseg = np.zeros((S, N, N))
        self.hist = np.zeros((self.D, 3, S, N, N))
        self.k = 0

    def load_state(self, u, lam, xseg, hist, k):
        self.u = _f64(u).copy()
        self.lam = _f64(lam).copy()
        self.xseg = _f64(xseg).copy()
        self.hist = _f64(hist).copy()
        assert self.hist.shape[0] == self.D
        self.k = int(k)

    def iterate(self, sino, drop=None, msgs=None):
        """one iteration on sinograms [S, A, B]; returns stats [S, NSTAT].
        drop [M, M] (s, m): node m loses owner s's message in this exchange.
        msgs [3, S, N, N]: dequantized K-means / JPEG messages to use in place
        of the oracle's own quantizers' output (plane 0 is ignored)"""
        p = self.p
        d = _f64(sino)
        it = np.array([self.k], np.int32)
        stats = np.empty((self.S, NSTAT), np.float64)
        if drop is not None and self.held is None:  # the versions every node holds without losses
            self.held = np.maximum(self.k - self.lag, 0).astype(np.int32)
        dr = None if drop is None else np.ascontiguousarray(drop, np.uint8)
        if msgs is not None:
            mi = _f64(msgs)
            assert mi.shape == (3, self.S, self.N, self.N)
        rc = lib().orc_dadmm_iterate(
            self.N, self.B, self.A, self.S, self.M, _ptr(self.c), _ptr(self.s),
            _ptr(self.node_ang_ptr), _ptr(self.node_ang), _ptr(self.seg_row_ptr),
            _ptr(self.adj), _ptr(self.edge_q), _ptr(self.home_q),
            float(p["rho"]), _ptr(self.eta1), float(p["eta2"]), int(p["E1"]), int(p["E2"]),
            int(p["km_k"]), int(p["km_iters"]), int(p["jpeg_quality"]), int(p["seed"]),
            self.D, _ptr(d), _ptr(self.u), _ptr(self.lam), _ptr(self.xseg), _ptr(self.hist),
            _ptr(it), _ptr(stats), None if dr is None else _ptr(dr), None if self.held is None else _ptr(self.held),
            None if msgs is None else _ptr(mi))
        if rc != 0:
            raise ValueError("orc_dadmm_iterate failed: %d" % rc)
        self.k = int(it[0])
        return stats

    def home_view(self):
        """conc over owners of their home-quantized segment at the current k"""
        N = self.N
        out = np.zeros((self.S, N, N))
        if self.k < 1:
            return out
        slot = self.k % self.D
        for m in range(self.M):
            r0, r1 = self.seg_row_ptr[m], self.seg_row_ptr[m + 1]
            out[:, r0:r1] = self.hist[slot, self.home_q[m], :, r0:r1]
        return out


class Consensus:
    """Oracle state of the neighbour-averaged consensus variant: u, lam and
    every node's own x, all [S, M, N, N] float64; k completed iterations."""

    def __init__(self, prob, eta1, S=None):
        self.p = prob
        g = prob["geometry"]
        self.N, self.B, self.A = g["N"], g["B"], g["A"]
        self.M = prob["M"]
        self.S = prob["S"] if S is None else S
        self.c, self.s = trig(_f64(g["theta"]))
        self.node_ang_ptr = _i32(prob["node_ang_ptr"])
        self.node_ang = _i32(prob["node_ang"])
        self.adj = _i32(prob["adj"])
        self.edge_q = _i32(prob["edge_q"])
        self.home_q = _i32(prob["home_q"])
        self.eta1 = _f64(eta1)
        N, M, S = self.N, self.M, self.S
        self.u = np.zeros((S, M, N, N))
        self.lam = np.zeros((S, M, N, N))
        self.x = np.zeros((S, M, N, N))
        self.k = 0

    def load_state(self, u, lam, x, k):
        self.u, self.lam, self.x = _f64(u).copy(), _f64(lam).copy(), _f64(x).copy()
        self.k = int(k)

    def iterate(self, sino):
        p = self.p
        d = _f64(sino)
        it = np.array([self.k], np.int32)
        stats = np.empty((self.S, NSTAT), np.float64)
        rc = lib().orc_consensus_iterate(
            self.N, self.B, self.A, self.S, self.M, _ptr(self.c), _ptr(self.s),
            _ptr(self.node_ang_ptr), _ptr(self.node_ang), _ptr(self.adj), _ptr(self.edge_q), _ptr(self.home_q),
            float(p["rho"]), _ptr(self.eta1), int(p["E1"]), int(p["km_k"]), int(p["km_iters"]),
            int(p["jpeg_quality"]), int(p["seed"]), _ptr(d), _ptr(self.u), _ptr(self.lam), _ptr(self.x),
            _ptr(it), _ptr(stats))
        if rc != 0:
            raise ValueError("orc_consensus_iterate failed: %d" % rc)
        self.k = int(it[0])
        return stats
