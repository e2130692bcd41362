"""GPU parity of the dADMM iteration (Algorithms 2-4, Eq. 15-18, 21-24)
against the FP64 oracle.

(i) state injection: the GPU's iterate k is loaded into the oracle, which runs
one iteration; the GPU's iterate k+1 must match (u, lambda, x segments:
relative L2 <= 1e-5; quantized messages: levels identical except at
rounding ties);
(ii) the tiny shape's full trajectory: the reconstruction within 1e-3 after
its 50 iterations (the other shapes' trajectories, against stored oracle
runs, are in test_gpu_trajectories.py);
plus: the batched (persistent, graph-captured) and plain (per-node launch)
forms are bit-identical, and a checkpoint resumes bit-identically."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import need_gpu, rel_l2
from paper_2410_06106_gb300 import api, synth
from problems import oracle_eta1, small_problem

pytestmark = pytest.mark.gpu


def gpu_state(s):
    return (s.u.cpu().numpy(), s.lam.cpu().numpy(), s.xseg.cpu().numpy(), s.hist.cpu().numpy(), s.k)


def compare_states(g_next, o, prob, tol=1e-5, msg_frac=1e-4):
    """u and x segments at tol; the new messages: identity plane at tol,
    quantized planes identical except at rounding ties (<= msg_frac of the
    entries); lambda at tol on every pixel whose new messages agree (a
    message that differs by one quantization level moves lambda there by
    rho times that level)"""
    u, lam, xseg, hist, k = g_next
    assert k == o.k
    assert rel_l2(u, o.u) <= tol
    assert rel_l2(xseg, o.xseg) <= tol
    slot = o.k % o.D
    kinds = set(np.asarray(prob["home_q"]).tolist()) | set(
        np.asarray(prob["edge_q"])[np.asarray(prob["adj"]) > 0].tolist())
    agree = np.ones(hist.shape[2:], bool)
    for q in kinds:
        a, b = hist[slot, q], o.hist[slot, q]
        if q == 0:
            assert rel_l2(a, b) <= tol
        else:  # quantized planes: identical levels except at rounding ties
            bad = np.abs(a - b) > 1e-4 * (np.abs(b).max() + 1e-30)
            # a K-means code sets one value; a JPEG code sets its 8 x 8 block
            per_code = 1 if q == 1 else 64
            assert bad.mean() <= msg_frac * per_code, (q, bad.mean())
            agree &= ~bad
    m = np.broadcast_to(agree[:, None], lam.shape)
    assert rel_l2(lam[m], o.lam[m]) <= 10 * tol


@pytest.mark.parametrize("quant,graph,M", [("none", "ring", 4), ("kmeans", "ring", 4),
                                          ("jpeg", "complete", 4), ("alternate", "ring", 8)])
def test_state_injection_small(quant, graph, M):
    need_gpu()
    p = small_problem(N=64, A=48, B=91, M=M, graph=graph, quant=quant, part="blocks",
                      noise=0.01, seed=M, km_k=16, jpeg_quality=50)
    eta = oracle_eta1(p, iters=60)
    s = api.DADMM(p, eta)
    sino = torch.as_tensor(p["sino"]).cuda()
    s.step(sino, 6)
    before = gpu_state(s)
    st = s.step(sino, 1)
    after = gpu_state(s)
    o = O.DADMM(p, eta)
    o.load_state(*before)
    ost = o.iterate(p["sino"])
    compare_states(after, o, p)
    compare_stats(st[0], ost, quant != "none")


def compare_stats(st, ost, quantized):
    """all five FP64 statistics [S, 5] of one iteration: the residual norm and
    node 0's previous view norm come from continuous state (1e-5); the gap and
    change norms also see the new messages, which at a rounding tie differ by
    one quantization level (1e-5 unquantized, 1e-3 quantized); bytes: exact
    sizes (K-means, identity) and entropy-coded JPEG messages, which a code at
    a rounding tie may change by a few bits"""
    tol_msg = 1e-3 if quantized else 1e-5
    for j, tol in ((0, tol_msg), (1, tol_msg), (2, 1e-5), (3, 1e-5)):
        assert rel_l2(st[:, j], ost[:, j]) <= tol, (j, st[:, j], ost[:, j])
    assert abs(st[:, 4] - ost[:, 4]).max() <= 1e-3 * ost[:, 4].max()


@pytest.mark.parametrize("name", ["c2_kmeans", "c3_batch_jpeg"])
def test_state_injection_full_config(name):
    """one iteration of the full-size problem, injected after 3 GPU iterations"""
    need_gpu()
    p = synth.make_problem(name)
    g = api.Geometry(p["geometry"]["N"], p["geometry"]["B"], p["geometry"]["theta"])
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    L = np.array([g.opnorm_sq(idx[ptr[m]:ptr[m + 1]], iters=30) for m in range(p["M"])])
    eta = 1.0 / (L + p["rho"])  # any step works: both sides get the same input
    s = api.DADMM(p, eta, geometry=g)
    sino = torch.as_tensor(p["sino"]).cuda()
    s.step(sino, 3)
    before = gpu_state(s)
    st = s.step(sino, 1)
    after = gpu_state(s)
    o = O.DADMM(p, eta)
    o.load_state(*before)
    ost = o.iterate(p["sino"])
    compare_states(after, o, p)
    compare_stats(st[0], ost, True)


def test_c1_trajectory_matches_oracle():
    need_gpu()
    p = synth.make_problem("c1_tiny")
    eta = oracle_eta1(p, iters=60)
    s = api.DADMM(p, eta)
    st = s.step(torch.as_tensor(p["sino"]).cuda(), p["iters"])
    o = O.DADMM(p, eta)
    ost = [o.iterate(p["sino"]) for _ in range(p["iters"])]
    x = s.home_view().cpu().numpy()
    assert rel_l2(x, o.home_view()) <= 1e-3
    ost = np.stack(ost)
    assert rel_l2(st[:, :, 0], ost[:, :, 0]) <= 1e-3  # primal gap trajectory
    assert np.all(st[:, :, 4] == ost[:, :, 4])        # bytes on the wire


@pytest.mark.parametrize("quant", ["none", "alternate"])
def test_batched_and_plain_forms_are_bit_identical(quant):
    need_gpu()
    p = small_problem(N=64, A=48, B=91, M=8, S=2, graph="ring", quant=quant, part="blocks", noise=0.01,
                      km_k=16)
    eta = oracle_eta1(p, iters=30)
    sino = torch.as_tensor(p["sino"]).cuda()
    a = api.DADMM(p, eta, mode="batched")
    b = api.DADMM(p, eta, mode="plain")
    sa = a.step(sino, 5)
    sb = b.step(sino, 5)
    for name in ("u", "lam", "xseg", "hist"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
    assert np.array_equal(sa, sb)


@pytest.mark.parametrize("tune,shape", [("wide", (64, 1, 128, 1)), ("narrow", (32, 1, 64, 1)),
                                        ("pairs", (32, 2, 128, 2)), ("quads", (64, 1, 128, 4)),
                                        ("widepairs", (64, 2, 128, 4))])
def test_launch_shapes_follow_the_oracle(tune, shape):
    """every launch shape of the operators (64 x 64 backprojector tiles with
    128-bin projector items; 32 x 64 tiles with 64-bin items for runs of 4
    angles; slice pairs of both operators; projector items of 4 slices) by
    state injection, on four slices; N = 96 leaves ragged tiles in all"""
    need_gpu()
    p = small_problem(N=96, A=64, B=139, M=4, S=4, graph="ring", quant="alternate", noise=0.02, seed=12, km_k=16)
    eta = oracle_eta1(p)
    s = api.DADMM(p, eta, tune=tune)
    assert s.launch_shape() == shape
    sino = torch.as_tensor(p["sino"]).cuda()
    s.step(sino, 2)
    before = gpu_state(s)
    st = s.step(sino, 1)
    o = O.DADMM(p, eta)
    o.load_state(*before)
    ost = o.iterate(p["sino"])
    compare_states(gpu_state(s), o, p)
    compare_stats(st[0], ost, True)
    assert s.launch_shape() == shape


def test_autotuned_shape_is_shared_by_the_solvers_of_a_problem():
    """the first step of an auto-tuned solver times both shapes and caches the
    choice for the problem: a second solver, plain or batched, runs the same
    shapes, so the two forms stay bit-identical"""
    need_gpu()
    p = small_problem(N=64, A=40, B=93, M=4, graph="complete", quant="kmeans", noise=0.02, seed=13, km_k=8)
    eta = oracle_eta1(p)
    a, b = api.DADMM(p, eta, mode="batched"), api.DADMM(p, eta, mode="plain")
    sino = torch.as_tensor(p["sino"]).cuda()
    assert a.launch_shape() == (64, 1, 128, 1)  # until the first step
    a.step(sino, 3)
    b.step(sino, 3)
    sa, sb = a.launch_shape(), b.launch_shape()
    assert (sa[0], sa[2], sa[3]) == (sb[0], sb[2], sb[3])
    assert sa[0] in (32, 64) and sa[1] == 1 and sa[2] in (64, 128) and sa[3] == 1  # one slice: no pairs
    for name in ("u", "lam", "xseg", "hist", "iter"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name


def test_slice_pairs_batched_and_plain_are_bit_identical():
    """with slice-pair items of both operators, the batched form (backprojector
    pairs) and the plain form (single-slice backprojector tiles of the same
    shape; the same projector pairs, one launch per slice pair and node) give
    the same iterates bit for bit, over four slices"""
    need_gpu()
    p = small_problem(N=64, A=48, B=93, M=4, S=4, graph="ring", quant="alternate", noise=0.02, seed=21, km_k=8)
    eta = oracle_eta1(p)
    sino = torch.as_tensor(p["sino"]).cuda()
    runs = [api.DADMM(p, eta, tune="pairs"), api.DADMM(p, eta, tune="pairs", mode="plain")]
    assert runs[0].launch_shape() == (32, 2, 128, 2) == runs[1].launch_shape()
    quads = [api.DADMM(p, eta, tune="widepairs"), api.DADMM(p, eta, tune="widepairs", mode="plain")]
    assert quads[0].launch_shape() == (64, 2, 128, 4)  # the plain form runs single-slice wide tiles
    qst = [r.step(sino, 4) for r in quads]
    for name in ("u", "lam", "xseg", "hist", "iter"):
        assert torch.equal(getattr(quads[0], name), getattr(quads[1], name)), name
    assert np.array_equal(qst[0], qst[1])
    stats = [r.step(sino, 4) for r in runs]
    for r, st in zip(runs[1:], stats[1:]):
        for name in ("u", "lam", "xseg", "hist", "iter"):
            assert torch.equal(getattr(runs[0], name), getattr(r, name)), name
        assert np.array_equal(stats[0], st)


def test_alternating_input_buffers():
    """a caller that alternates input buffers (double-buffered host copies)
    gets the same iterates as one that passes one buffer: each buffer keeps
    its own captured iteration"""
    need_gpu()
    p = small_problem(N=64, A=48, B=93, M=4, graph="ring", quant="alternate", noise=0.02, seed=6, km_k=16)
    eta = oracle_eta1(p)
    a, b = api.DADMM(p, eta), api.DADMM(p, eta)
    bufs = [torch.as_tensor(p["sino"]).cuda() for _ in range(3)]
    for i in range(7):
        a.step(bufs[0], 1)
        b.step(bufs[i % 3], 1)
    for name in ("u", "lam", "xseg", "hist", "iter"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name


def test_checkpoint_resume_is_bit_identical():
    need_gpu()
    p = small_problem(N=64, A=48, B=91, M=4, graph="ring", quant="alternate", part="blocks", noise=0.01,
                      km_k=16)
    eta = oracle_eta1(p, iters=30)
    sino = torch.as_tensor(p["sino"]).cuda()
    s = api.DADMM(p, eta)
    s.step(sino, 4)
    ck = s.state_dict()
    s.step(sino, 5)
    x_a = s.home_view().clone()
    s.load_state_dict(ck)
    s.step(sino, 5)
    assert torch.equal(s.home_view(), x_a)


def test_stress_config_sampled_parity():
    """the 8 x 2048^2, 64-node problem (random geometric graph, alternating
    K-means / JPEG edges) in the batched launch configuration the benchmark
    times, with one Algorithm 2 step per iteration so that single pixels can
    be recomputed by the oracle:
    iteration 1 from zero gives u_m = eta1_m P_m^T d_m;
    iteration 2 takes the step Delta = P_m^T (P_m u_m - d_m) + rho (u_m - x_m) + lambda_m
    with x_m = u_m - lambda_m / rho (Eq. 24 with lambda^0 = 0), i.e.
    Delta = P_m^T (P_m u_m - d_m) + 2 lambda_m, checked at sampled pixels of four
    (slice, node) images from the GPU's own u and lambda after iteration 1"""
    need_gpu()
    p = dict(synth.make_problem("c5_stress"), E1=1)
    N, B, rho = p["geometry"]["N"], p["geometry"]["B"], p["rho"]
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    eta = 1.0 / (1.2 * np.diff(ptr) * N + rho)  # any step: both sides get the same
    og = O.Geometry(N, B, p["geometry"]["theta"])
    hB, hN = 0.5 * (B - 1), 0.5 * (N - 1)
    rng = np.random.default_rng(11)
    picks = [(0, 0), (3, 17), (5, 42), (7, 63)]
    pix = {k: rng.integers(0, N * N, 8) for k in picks}
    s = api.DADMM(p, eta)
    sino = torch.as_tensor(p["sino"]).cuda()
    st = s.step(sino, 1)
    assert np.all(np.isfinite(st)) and np.all(st[:, :, 4] > 0)
    u1, lam1 = {}, {}
    for (sl, m) in picks:
        angs = idx[ptr[m]:ptr[m + 1]]
        u1[sl, m] = s.u[sl, m].cpu().numpy().astype(np.float64)
        lam1[sl, m] = s.lam[sl, m].cpu().numpy().ravel()[pix[sl, m]].astype(np.float64)
        want = eta[m] * og.backproject_pixels(p["sino"][sl][angs], pix[sl, m], angs)
        assert rel_l2(u1[sl, m].ravel()[pix[sl, m]], want) <= 1e-5, (sl, m)
    s.step(sino, 1)
    for (sl, m) in picks:
        angs = idx[ptr[m]:ptr[m + 1]]
        q = pix[sl, m]
        # residual lines through the sampled pixels: 4 bins around each pixel's position
        rk, rb = [], []
        for e in q:
            xc, yc = e % N - hN, hN - e // N
            for k, a in enumerate(angs):
                t = xc * np.cos(p["geometry"]["theta"][a]) + yc * np.sin(p["geometry"]["theta"][a]) + hB
                for b in range(int(np.floor(t)) - 1, int(np.floor(t)) + 3):
                    if 0 <= b < B:
                        rk.append(k)
                        rb.append(b)
        rk, rb = np.asarray(rk), np.asarray(rb)
        key = np.unique(rk * B + rb)
        rk, rb = key // B, key % B
        r = og.project_rays(u1[sl, m], angs[rk], rb) - p["sino"][sl][angs[rk], rb]
        res = np.zeros((len(angs), B))
        res[rk, rb] = r
        delta = og.backproject_pixels(res, q, angs) + 2.0 * lam1[sl, m]
        got = (u1[sl, m].ravel()[q] - s.u[sl, m].cpu().numpy().ravel()[q].astype(np.float64)) / eta[m]
        assert rel_l2(got, delta) <= 1e-4, (sl, m)


def node_view(hist, k, D, sl, m, p, dist, first):
    """node m's view x_m^k of slice sl, assembled from the GPU's message ring by
    the relay rule: segment s holds the message of iteration k - max(dist - 1, 0),
    in the plane of the path's first edge (the home plane for the node's own
    segment), zero before the first message arrives"""
    N, M, seg = p["geometry"]["N"], p["M"], p["seg_row_ptr"]
    out = np.zeros((N, N))
    for s in range(M):
        lag = 0 if s == m else dist[s, m] - 1
        ver = k - lag
        if ver < 1:
            continue
        kind = p["home_q"][m] if s == m else p["edge_q"][s, first[s, m]]
        out[seg[s]:seg[s + 1]] = hist[ver % D, kind, sl, seg[s]:seg[s + 1]].cpu().numpy()
    return out


def test_stress_config_inner_loop_by_state_injection():
    """the 8 x 2048^2, 64-node problem with the benchmark's E1 = 10 inner steps,
    in the launch configuration the benchmark times (batched, auto-tuned
    shapes): after two iterations, the GPU's u_m of the third iteration equals
    the oracle's Algorithm 2 (ten steps, whole 2048^2 image) from the GPU's
    u_m, lambda_m and the node's view of x (assembled from the message ring)
    for four (slice, node) pairs, at the state-injection tolerance 1e-5"""
    need_gpu()
    p = synth.make_problem("c5_stress")
    N, B, rho, E1 = p["geometry"]["N"], p["geometry"]["B"], p["rho"], p["E1"]
    assert E1 == 10
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    eta = 1.0 / (1.2 * np.diff(ptr) * N + rho)  # any step: both sides get the same
    og = O.Geometry(N, B, p["geometry"]["theta"])
    dist, first = O.relay_tables(p["adj"])
    s = api.DADMM(p, eta)
    sino = torch.as_tensor(p["sino"]).cuda()
    s.step(sino, 2, stats=False)
    k = int(s.iter.item())
    D = s.hist.shape[0]
    picks = [(0, 0), (2, 9), (5, 42), (7, 63)]
    before = {}
    for sl, m in picks:
        before[sl, m] = (s.u[sl, m].cpu().numpy(), s.lam[sl, m].cpu().numpy(),
                         node_view(s.hist, k, D, sl, m, p, dist, first))
    s.step(sino, 1, stats=False)
    for sl, m in picks:
        u0, l0, xv = before[sl, m]
        want, _ = og.alg2_node(u0, xv, l0, p["sino"][sl], idx[ptr[m]:ptr[m + 1]], rho, eta[m], E1)
        err = rel_l2(s.u[sl, m].cpu().numpy(), want)
        assert err <= 1e-5, (sl, m, err)
    del s
