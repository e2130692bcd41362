"""Seeded random configurations against the FP64 oracle, beyond the fixed
shapes: operator geometries (odd and even N, detectors narrower and wider
than the image diagonal, arbitrary angles including negative ones, exact
multiples of pi/4, repeated and unordered angle selections, batches,
subtraction), and dADMM problems (random graphs, partitions with empty
nodes, ragged segments, every quantizer mix, two slices, random solver
settings) checked by state injection (one GPU iteration replayed by the
oracle from the same state)."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import cuda, need_gpu, rel_l2
from paper_2410_06106_gb300 import api, synth
from test_gpu_dadmm import compare_states, gpu_state

pytestmark = pytest.mark.gpu
TOL = 1e-5


AXIS_GAP = 1.5e-3  # non-axis angles keep min(|cos|, |sin|) above this (uniform sets up to 2000 angles do)


def random_geometry(rng):
    N = int(rng.integers(3, 300))
    diag = int(np.ceil(N * np.sqrt(2)))
    B = int(rng.integers(max(1, diag // 2), diag + 40))
    A = int(rng.integers(1, 160))
    theta = rng.uniform(-np.pi, 2 * np.pi, A)
    near = np.minimum(np.abs(np.cos(theta)), np.abs(np.sin(theta))) < AXIS_GAP
    theta[near] += 4 * AXIS_GAP  # off the axis (the near-axis envelope has its own test)
    special = rng.random(A) < 0.2  # exact multiples of pi/4
    theta[special] = rng.integers(-4, 9, special.sum()) * (np.pi / 4)
    return N, B, theta


@pytest.mark.parametrize("seed", range(24))
def test_random_operator_geometries(seed):
    need_gpu()
    rng = np.random.default_rng(1000 + seed)
    N, B, theta = random_geometry(rng)
    A = len(theta)
    g = api.Geometry(N, B, theta)
    og = O.Geometry(N, B, theta)
    n_sel = int(rng.integers(1, 2 * A + 1))
    sel = rng.integers(0, A, n_sel).astype(np.int32)  # unordered, with repeats
    batch = int(rng.integers(1, 4))
    img = rng.standard_normal((batch, N, N)).astype(np.float32)
    sub = rng.standard_normal((batch, n_sel, B)).astype(np.float32) if rng.random() < 0.5 else None
    d = g.project(cuda(img), sel, subtract=cuda(sub) if sub is not None else None).cpu().numpy()
    ref = og.project(img, sel) - (sub if sub is not None else 0.0)
    assert rel_l2(d, ref) <= TOL, (N, B, A, n_sel, batch)
    r = rng.standard_normal((batch, n_sel, B)).astype(np.float32)
    bp = g.backproject(cuda(r), sel).cpu().numpy()
    assert rel_l2(bp, og.backproject(r, sel)) <= TOL, (N, B, A, n_sel, batch)
    g.close()


def test_near_axis_angles_accuracy_envelope():
    """Angles a little off an axis (min(|cos|, |sin|) = 3e-4 .. 1.5e-3) have
    trapezoid ramps of slope 1/min(|cos|, |sin|) up to ~3300 in minor units.
    The FP32 weights resolve positions to 2^-23, so inside a ramp a weight
    is off by up to that slope x 1.2e-7; rays land in a ramp with
    probability ~1/slope. The projection's relative error therefore grows
    like sqrt(slope) x ~5e-7. It stays below 1e-5 for the uniform angle sets
    of the shapes (slope <= 573), and below 4e-5 here"""
    need_gpu()
    N, B = 96, 137
    rng = np.random.default_rng(77)
    off = np.array([3e-4, -5e-4, 8e-4, -1.2e-3, 1.5e-3])
    theta = np.concatenate([off, np.pi / 2 + off, np.pi + off, rng.uniform(0, np.pi, 11)])
    g = api.Geometry(N, B, theta)
    og = O.Geometry(N, B, theta)
    img = rng.standard_normal((N, N)).astype(np.float32)
    ep = rel_l2(g.project(cuda(img)).cpu().numpy(), og.project(img))
    r = rng.standard_normal((len(theta), B)).astype(np.float32)
    eb = rel_l2(g.backproject(cuda(r)).cpu().numpy(), og.backproject(r))
    print("near-axis envelope: projector %.2e, backprojector %.2e" % (ep, eb))
    assert ep <= 4e-5 and eb <= 4e-5
    g.close()


def random_problem(rng, seed):
    quant = ["none", "kmeans", "jpeg", "alternate"][seed % 4]
    jpeg = quant in ("jpeg", "alternate")
    M = int(rng.integers(2, 10))
    if jpeg:  # JPEG segments are whole 8-row blocks
        rows = rng.integers(1, 4, M) * 8
        N = int(rows.sum())
        seg = np.concatenate([[0], np.cumsum(rows)]).astype(np.int32)
    else:  # ragged bands
        N = int(rng.integers(M, 80))
        cuts = np.sort(rng.choice(np.arange(1, N), M - 1, replace=False))
        seg = np.concatenate([[0], cuts, [N]]).astype(np.int32)
    A = int(rng.integers(M, 6 * M))
    B = int(np.ceil(N * np.sqrt(2))) + int(rng.integers(0, 5))
    theta = synth.angles(A) + rng.uniform(0, 0.05)
    counts = rng.multinomial(A, rng.dirichlet(np.ones(M)))  # may leave nodes without angles
    if rng.random() < 0.5:
        parts = synth.partition_contiguous(counts)
    else:
        perm = rng.permutation(A).astype(np.int32)
        parts = [np.sort(perm[a:b]) for a, b in zip(np.r_[0, np.cumsum(counts)[:-1]], np.cumsum(counts))]
    ptr, idx = synth.csr(parts)
    graph = ["ring", "complete", "rgg"][int(rng.integers(3))]
    adj = {"ring": lambda: synth.ring(M), "complete": lambda: synth.complete(M),
           "rgg": lambda: synth.random_geometric_graph(M, min(M - 1, 2 + int(rng.integers(0, 3))), 7 + seed)}[graph]()
    kinds = {"none": 0, "kmeans": 1, "jpeg": 2}
    if quant == "alternate":
        edge_q = synth.alternating_edge_kinds(adj)
        home_q = np.where(np.arange(M) % 2 == 0, 1, 2).astype(np.int32)
    else:
        edge_q = synth.uniform_edge_kinds(adj, kinds[quant])
        home_q = np.full(M, kinds[quant], np.int32)
    S = int(rng.integers(1, 3))
    sino = np.empty((S, A, B), np.float32)
    for sl in range(S):
        ell = synth.random_ellipses(N, 4, rng)
        sino[sl] = synth.add_noise(synth.ellipse_sinogram(ell, theta, B), 0.01, rng)
    return dict(name="fuzz", geometry=dict(N=N, A=A, B=B, theta=theta), M=M, S=S, node_ang_ptr=ptr,
                node_ang=idx, seg_row_ptr=seg, adj=adj, edge_q=edge_q, home_q=home_q,
                km_k=int(rng.integers(2, 33)), jpeg_quality=int(rng.integers(10, 96)), seed=99 + seed,
                iters=4, sino=sino, rho=float(rng.uniform(0.5, 2.0)), eta2=float(rng.uniform(0.05, 0.4)),
                E1=int(rng.integers(1, 6)), E2=int(rng.integers(1, 6)), km_iters=int(rng.integers(0, 12)))


@pytest.mark.parametrize("seed", range(8))
def test_random_dadmm_problems_state_injection(seed):
    need_gpu()
    rng = np.random.default_rng(2000 + seed)
    p = random_problem(rng, seed)
    og = O.Geometry(p["geometry"]["N"], p["geometry"]["B"], p["geometry"]["theta"])
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    L = np.array([og.opnorm_sq(idx[ptr[m]:ptr[m + 1]], iters=40) if ptr[m + 1] > ptr[m] else 0.0
                  for m in range(p["M"])])
    eta = 1.0 / (L + p["rho"])
    s = api.DADMM(p, eta)
    sino = torch.as_tensor(p["sino"]).cuda()
    s.step(sino, 3)
    before = gpu_state(s)
    s.step(sino, 1)
    after = gpu_state(s)
    o = O.DADMM(p, eta)
    o.load_state(*before)
    o.iterate(p["sino"])
    compare_states(after, o, p)
