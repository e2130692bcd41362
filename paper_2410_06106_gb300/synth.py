"""Seeded synthetic inputs: random-ellipse phantoms, analytic sinograms,
noise, angle partitions, node graphs and the five benchmark problem shapes.

This module holds none of the reconstruction method's arithmetic (no system
matrix, no ADMM step, no quantizer). It produces the inputs that both the CUDA
path and the FP64 CPU oracle consume, so it imports neither of them.

Conventions match the operator's: pixel (i, j) is centred at
x = j - (N-1)/2, y = (N-1)/2 - i; ray (a, b) is x cos(theta_a) + y sin(theta_a)
= t_b with t_b = b - (B-1)/2; theta_a = a pi / A.

The sinograms are ANALYTIC line integrals of the ellipses (Kak & Slaney,
"Principles of Computerized Tomographic Imaging", ch. 3, the reference the
paper cites for the x-ray transform, Eq. 1), so the data never comes from the
discrete operator being tested.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2410_06106

KIND_NONE, KIND_KMEANS, KIND_JPEG = 0, 1, 2


# --------------------------------------------------------------------------
# phantoms and data
# --------------------------------------------------------------------------

def angles(A: int) -> np.ndarray:
    """A angles uniform on [0, pi): theta_a = a pi / A."""
    return np.arange(A, dtype=np.float64) * (math.pi / A)


def random_ellipses(N: int, count: int, rng: np.random.Generator) -> np.ndarray:
    """count ellipses as rows (cx, cy, a, b, phi, density), pixel units.

    Centres uniform in the disk inscribed in the image (r = sqrt(U)),
    semi-axes U[0.05, 0.4] x N/2, rotation U[0, pi), density U[0.1, 1]."""
    R = N / 2.0
    r = np.sqrt(rng.random(count)) * R
    ang = 2.0 * math.pi * rng.random(count)
    a = rng.uniform(0.05, 0.4, count) * R
    b = rng.uniform(0.05, 0.4, count) * R
    phi = rng.uniform(0.0, math.pi, count)
    rho = rng.uniform(0.1, 1.0, count)
    return np.stack([r * np.cos(ang), r * np.sin(ang), a, b, phi, rho], axis=1)


def ellipse_sinogram(ell: np.ndarray, theta: np.ndarray, B: int) -> np.ndarray:
    """Exact line integrals [A, B] of a sum of uniform ellipses.

    For an ellipse with semi-axes (a, b) rotated by phi and centred at
    (cx, cy): shift t' = t - (cx cos th + cy sin th), relative angle
    th' = th - phi, s2 = a^2 cos^2 th' + b^2 sin^2 th'; the chord integral is
    2 rho a b sqrt(s2 - t'^2) / s2 for |t'| < sqrt(s2), else 0."""
    t = np.arange(B, dtype=np.float64) - 0.5 * (B - 1)
    out = np.zeros((len(theta), B), np.float64)
    ct, st = np.cos(theta)[:, None], np.sin(theta)[:, None]
    for cx, cy, a, b, phi, rho in ell:
        tp = t[None, :] - (cx * ct + cy * st)
        thr = theta[:, None] - phi
        s2 = (a * np.cos(thr)) ** 2 + (b * np.sin(thr)) ** 2
        arg = np.clip(s2 - tp * tp, 0.0, None)
        out += 2.0 * rho * a * b * np.sqrt(arg) / s2
    return out


def rasterize(ell: np.ndarray, N: int, ss: int = 4) -> np.ndarray:
    """Pixel-average density of the ellipses on an ss x ss subgrid [N, N]."""
    off = (np.arange(ss) + 0.5) / ss - 0.5
    x = (np.arange(N) - 0.5 * (N - 1))
    y = (0.5 * (N - 1) - np.arange(N))
    img = np.zeros((N, N), np.float64)
    for oy in off:
        Y = (y + oy)[:, None]
        for ox in off:
            X = (x + ox)[None, :]
            for cx, cy, a, b, phi, rho in ell:
                dx, dy = X - cx, Y - cy
                cp, sp = math.cos(phi), math.sin(phi)
                u = (dx * cp + dy * sp) / a
                v = (-dx * sp + dy * cp) / b
                img += rho * ((u * u + v * v) <= 1.0)
    return img / (ss * ss)


def add_noise(d: np.ndarray, frac: float, rng: np.random.Generator) -> np.ndarray:
    """Additive Gaussian noise with sigma = frac * max(d)."""
    if frac <= 0.0:
        return d.copy()
    return d + rng.normal(0.0, frac * float(d.max()), d.shape)


# --------------------------------------------------------------------------
# partitions and graphs
# --------------------------------------------------------------------------

def partition_contiguous(counts) -> list:
    """consecutive angle blocks of the given sizes, in node order"""
    out, a0 = [], 0
    for c in counts:
        out.append(np.arange(a0, a0 + c, dtype=np.int32))
        a0 += c
    return out


def partition_even_blocks(A: int, M: int) -> list:
    """contiguous near-equal blocks (the first A mod M nodes get one more)"""
    base, extra = divmod(A, M)
    return partition_contiguous([base + (m < extra) for m in range(M)])


def partition_interleaved(A: int, M: int) -> list:
    """node m holds angles m, m+M, m+2M, ... (the 2- and 10-node splits of Sec. 3.2)"""
    return [np.arange(m, A, M, dtype=np.int32) for m in range(M)]


def uneven_counts(A: int, M: int, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    """M counts drawn from U{lo..hi}, repaired by +-1 on random nodes (within
    the bounds) until they sum to A."""
    assert lo * M <= A <= hi * M
    c = rng.integers(lo, hi + 1, M)
    while c.sum() != A:
        i = int(rng.integers(M))
        if c.sum() > A and c[i] > lo:
            c[i] -= 1
        elif c.sum() < A and c[i] < hi:
            c[i] += 1
    return c


def ring(M: int) -> np.ndarray:
    adj = np.zeros((M, M), np.int32)
    for m in range(M):
        adj[m, (m + 1) % M] = adj[(m + 1) % M, m] = 1
    np.fill_diagonal(adj, 0)
    return adj


def complete(M: int) -> np.ndarray:
    adj = np.ones((M, M), np.int32)
    np.fill_diagonal(adj, 0)
    return adj


def connected(adj: np.ndarray) -> bool:
    M = adj.shape[0]
    seen = np.zeros(M, bool)
    stack = [0]
    seen[0] = True
    while stack:
        x = stack.pop()
        for y in np.nonzero(adj[x])[0]:
            if not seen[y]:
                seen[y] = True
                stack.append(int(y))
    return bool(seen.all())


def random_geometric_graph(M: int, mean_degree: int, seed: int) -> np.ndarray:
    """Nodes uniform in the unit square; keep the M*deg/2 shortest pairs
    (exact mean degree); a disconnected draw moves on to seed+1."""
    n_edges = M * mean_degree // 2
    while True:
        rng = np.random.default_rng(seed)
        pts = rng.random((M, 2))
        iu, ju = np.triu_indices(M, 1)
        d = np.hypot(*(pts[iu] - pts[ju]).T)
        order = np.lexsort((ju, iu, d))[:n_edges]
        adj = np.zeros((M, M), np.int32)
        adj[iu[order], ju[order]] = 1
        adj[ju[order], iu[order]] = 1
        if connected(adj):
            return adj
        seed += 1


def uniform_edge_kinds(adj: np.ndarray, kind: int) -> np.ndarray:
    """every edge uses the same quantizer; -1 marks a non-edge"""
    return np.where(adj > 0, kind, -1).astype(np.int32)


def alternating_edge_kinds(adj: np.ndarray) -> np.ndarray:
    """undirected edges in (min id, max id) order; even position -> K-means,
    odd -> JPEG"""
    M = adj.shape[0]
    q = np.full((M, M), -1, np.int32)
    e = 0
    for i in range(M):
        for j in range(i + 1, M):
            if adj[i, j]:
                q[i, j] = q[j, i] = KIND_KMEANS if e % 2 == 0 else KIND_JPEG
                e += 1
    return q


def csr(parts) -> tuple:
    ptr = np.zeros(len(parts) + 1, np.int32)
    ptr[1:] = np.cumsum([len(p) for p in parts])
    idx = np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)
    return ptr, idx


def even_segments(N: int, M: int) -> np.ndarray:
    """contiguous row bands, near-equal (the first N mod M get one more row)"""
    base, extra = divmod(N, M)
    rows = [base + (m < extra) for m in range(M)]
    return np.concatenate([[0], np.cumsum(rows)]).astype(np.int32)


# --------------------------------------------------------------------------
# the five problem shapes
# --------------------------------------------------------------------------

CONFIGS = {
    # name: N, A, B, M, slices, ellipses, noise, graph, partition, quantizer, iterations
    "c1_tiny": dict(idx=1, N=64, A=90, B=91, M=4, S=1, ellipses=5, noise=0.01,
                    graph=("ring",), part=("even_blocks",), quant="none", iters=50),
    "c2_kmeans": dict(idx=2, N=256, A=360, B=367, M=8, S=1, ellipses=10, noise=0.01,
                      graph=("ring",), part=("interleaved",), quant="kmeans", iters=100),
    "c3_batch_jpeg": dict(idx=3, N=512, A=720, B=725, M=16, S=1, ellipses=20, noise=0.01,
                          graph=("rgg", 4), part=("uneven", 10, 80), quant="jpeg", iters=100),
    "c4_diff": dict(idx=4, N=1024, A=1440, B=1449, M=8, S=1, ellipses=30, noise=0.01,
                    graph=("complete",), part=("interleaved",), quant="none", iters=10),
    "c5_stress": dict(idx=5, N=2048, A=1800, B=2897, M=64, S=8, ellipses=40, noise=0.01,
                      graph=("rgg", 6), part=("uneven", 8, 60), quant="alternate", iters=200),
}

SOLVER = dict(rho=1.0, eta2=0.2, E1=10, E2=10, km_iters=10)


def make_problem(name: str, slices: int | None = None, with_phantom: bool = False,
                 **override) -> dict:
    """Build one of the five problems (or a variant via keyword overrides of
    the CONFIGS entry). Returns a dict of plain numpy arrays and scalars."""
    cfg = dict(CONFIGS[name])
    cfg.update(override)
    N, A, B, M = cfg["N"], cfg["A"], cfg["B"], cfg["M"]
    S = cfg["S"] if slices is None else slices
    base = SEED_BASE + 1000 * cfg["idx"]
    theta = angles(A)

    kind = cfg["part"][0]
    if kind == "even_blocks":
        parts = partition_even_blocks(A, M)
    elif kind == "interleaved":
        parts = partition_interleaved(A, M)
    else:
        counts = uneven_counts(A, M, cfg["part"][1], cfg["part"][2],
                               np.random.default_rng(base + 500))
        parts = partition_contiguous(counts)
    ptr, idx = csr(parts)

    g = cfg["graph"][0]
    if g == "ring":
        adj = ring(M)
    elif g == "complete":
        adj = complete(M)
    else:
        adj = random_geometric_graph(M, cfg["graph"][1], base + 600)

    q = cfg["quant"]
    if q == "none":
        edge_q, home_q = uniform_edge_kinds(adj, KIND_NONE), np.zeros(M, np.int32)
    elif q == "kmeans":
        edge_q, home_q = uniform_edge_kinds(adj, KIND_KMEANS), np.full(M, KIND_KMEANS, np.int32)
    elif q == "jpeg":
        edge_q, home_q = uniform_edge_kinds(adj, KIND_JPEG), np.full(M, KIND_JPEG, np.int32)
    else:
        edge_q = alternating_edge_kinds(adj)
        home_q = np.where(np.arange(M) % 2 == 0, KIND_KMEANS, KIND_JPEG).astype(np.int32)

    km_k = {"c2_kmeans": 16, "c5_stress": 32}.get(name, 16)
    jpeg_q = {"c3_batch_jpeg": 50, "c5_stress": 75}.get(name, 50)

    sino = np.empty((S, A, B), np.float32)
    ells = []
    for sl in range(S):
        rng = np.random.default_rng(base + sl)
        ell = random_ellipses(N, cfg["ellipses"], rng)
        d = ellipse_sinogram(ell, theta, B)
        sino[sl] = add_noise(d, cfg["noise"], rng).astype(np.float32)
        ells.append(ell)

    prob = dict(
        name=name, geometry=dict(N=N, A=A, B=B, theta=theta), M=M, S=S,
        node_ang_ptr=ptr, node_ang=idx, seg_row_ptr=even_segments(N, M),
        adj=adj, edge_q=edge_q, home_q=home_q, km_k=km_k, jpeg_quality=jpeg_q,
        seed=base + 700, iters=cfg["iters"], sino=sino, ellipses=ells, **SOLVER)
    prob.update({k: v for k, v in override.items() if k in SOLVER or k in ("km_k", "jpeg_quality", "seed")})
    if with_phantom:
        prob["phantom"] = np.stack([rasterize(e, N) for e in ells]).astype(np.float32)
    return prob

