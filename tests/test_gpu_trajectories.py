"""Full-trajectory parity of the dADMM iteration (Algorithm 4 with Algorithms
2, 3, 5 and Eq. 15-18, 21-24) at the stated iteration counts of the
benchmark shapes, against FP64 oracle trajectories stored by
tests/golden/make_trajectory_goldens.py (which calls only the oracle and the
seeded input generators):

- 256^2, 360 angles, 8 nodes on a ring, K-means messages (k = 16), 100 iterations;
- 512^2, 720 angles, 16 nodes on a random geometric graph with uneven angle
  counts, JPEG messages (quality 50), 100 iterations;
- 1024^2, 1440 angles, 8 nodes on a complete graph, no quantizer, 10 iterations.

Both sides get the oracle's step sizes eta1 (stored with the trajectory).

Unquantized: the reconstruction, u and lambda within the protocol's 1e-3
(relative L2; at seeded sample positions where the full arrays are too large
to store). Quantized: a message is not a continuous function of the iterate
(a value at a K-means decision boundary or a JPEG rounding tie changes by a
whole level), so FP32 and FP64 states a rounding apart take a few different
decisions, lambda accumulates them, and free-running trajectories drift apart
(measured: u 1.5e-3, x 1.6e-1 after the K-means ring's 100 iterations). So
the quantized shapes are checked three ways: (1) with the same decisions on
both sides (the oracle takes the GPU's messages), every continuous state
stays within 1e-3 of the FP64 iteration; (2) free-running, the last of the
100 iterations is replayed by the oracle from the GPU's state at the kernel
tolerance; (3) free-running, the reconstruction is held to the bound that
follows from the quantizers' steps:

  ||Q_gpu(x_gpu) - Q_orc(x_orc)|| <= ||x_gpu - x_orc|| + b_gpu + b_orc,

where b is the worst-case quantization error of that side's messages, derived
from the quantizer, not fitted: for K-means every value lies within half the
gap between the neighbouring centres (or within the distance from the
segment's extreme value to the outermost centre); for JPEG a block of 64
samples is off by at most 4 (rounding to 8-bit samples) + ||Qt||_F / 2
(rounding the orthonormal DCT coefficients to multiples of the table) + 4
(rounding the inverse), in units of (hi - lo) / 255. Each side's realized
quantization error is also checked against its own bound."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import need_gpu, rel_l2
from paper_2410_06106_gb300 import api, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    path = os.path.join(GOLDEN, "%s_trajectory.npz" % name)
    assert os.path.exists(path), "missing %s: run tests/golden/make_trajectory_goldens.py %s" % (path, name)
    return np.load(path)


def run_gpu(name, z):
    p = synth.make_problem(name)
    s = api.DADMM(p, z["eta1"])
    st = s.step(torch.as_tensor(p["sino"]).cuda(), int(z["iters"]))
    return p, s, st


def sampled_rel(full, idx, val):
    return rel_l2(full.reshape(-1)[idx], val)


def kmeans_bound(v, q):
    """worst-case |v - Q(v)| over a K-means-coded segment: the largest half gap
    between neighbouring used centres, or the distance from an extreme value to
    the outermost centre"""
    c = np.unique(q)
    d = max(c[0] - v.min(), v.max() - c[-1], 0.0)
    if len(c) > 1:
        d = max(d, 0.5 * np.diff(c).max())
    return d


def jpeg_block_bound(v, quality):
    """worst-case L2 error of one 8x8 block of a JPEG-coded segment"""
    lo, hi = float(v.min()), float(v.max())
    if hi == lo:
        return 0.0
    qt = O.jpeg_qtable(quality).astype(np.float64)
    return (hi - lo) / 255.0 * (4.0 + 0.5 * np.linalg.norm(qt) + 4.0)


def quantization_bounds(p, xs, q):
    """per-side worst-case ||x - Q(x)|| over the home-quantized segments, and the
    realized error of each segment against its own bound"""
    seg = p["seg_row_ptr"]
    N = p["geometry"]["N"]
    tot2 = 0.0
    for m in range(p["M"]):
        v = xs[seg[m]:seg[m + 1]].astype(np.float64)
        qm = q[seg[m]:seg[m + 1]].astype(np.float64)
        # the codec sees the segment in FP32; allow its rounding (2^-24 relative)
        slack = 2.0 ** -23 * np.abs(v).max()
        if p["home_q"][m] == synth.KIND_KMEANS:
            b_val = kmeans_bound(v.astype(np.float32).astype(np.float64), qm) + slack
            assert np.abs(v - qm).max() <= b_val * (1 + 1e-6), (m, np.abs(v - qm).max(), b_val)
            b2 = v.size * b_val * b_val
        else:
            nblk = v.size // 64
            b_blk = jpeg_block_bound(v.astype(np.float32), p["jpeg_quality"]) * (1 + 1e-4) + 8 * slack
            err = (v - qm).reshape(v.shape[0] // 8, 8, N // 8, 8).transpose(0, 2, 1, 3).reshape(-1, 64)
            assert np.linalg.norm(err, axis=1).max() <= b_blk, (m, np.linalg.norm(err, axis=1).max(), b_blk)
            b2 = nblk * b_blk * b_blk
        tot2 += b2
    return np.sqrt(tot2)


@pytest.mark.parametrize("name,iters", [("c2_kmeans", 100), ("c3_batch_jpeg", 25)])
def test_quantized_shapes_follow_the_oracle_given_the_same_decisions(name, iters):
    """the continuous arithmetic over many iterations: the oracle runs Algorithm 4
    live with the GPU's dequantized messages in place of its own quantizers'
    output (the same discrete decisions on both sides), so u, lambda, the owners'
    segments x and the reconstruction must stay within the protocol's 1e-3 of the
    FP64 iteration: all 100 stated iterations of the K-means ring, 25 of the
    JPEG graph (an FP64 iteration of the 512^2, 16-node problem takes seconds)"""
    need_gpu()
    z = golden(name)
    p = synth.make_problem(name)
    s = api.DADMM(p, z["eta1"])
    o = O.DADMM(p, z["eta1"])
    sino = torch.as_tensor(p["sino"]).cuda()
    D = s.hist.shape[0]
    for _ in range(iters):
        s.step(sino, 1, stats=False)
        o.iterate(p["sino"], msgs=s.hist[s.k % D].cpu().numpy())
    errs = {"u": rel_l2(s.u.cpu().numpy(), o.u), "lambda": rel_l2(s.lam.cpu().numpy(), o.lam),
            "x": rel_l2(s.xseg.cpu().numpy(), o.xseg), "reconstruction": rel_l2(s.home_view().cpu().numpy(),
                                                                                o.home_view())}
    print("%s, %d iterations with the GPU's decisions: %s" % (name, iters, {k: "%.2e" % v for k, v in errs.items()}))
    for k, v in errs.items():
        assert v <= 1e-3, (k, v)


@pytest.mark.parametrize("name", ["c2_kmeans", "c3_batch_jpeg"])
def test_quantized_shapes_free_running_for_100_iterations(name):
    """each side with its own decisions, against the stored FP64 trajectory. The
    reconstruction is held to the bound derived from the quantizers' steps (the
    module docstring); the last iteration is replayed by the oracle from the
    GPU's state (state injection: the kernels agree at the state the GPU
    reached); the drift of u, lambda and x from the stored trajectory, which
    grows through decisions that flip between FP32 and FP64 states, is printed"""
    need_gpu()
    from test_gpu_dadmm import compare_states, gpu_state
    z = golden(name)
    p = synth.make_problem(name)
    assert int(z["iters"]) == p["iters"] == 100
    s = api.DADMM(p, z["eta1"])
    sino = torch.as_tensor(p["sino"]).cuda()
    s.step(sino, 99, stats=False)
    before = gpu_state(s)
    s.step(sino, 1, stats=False)
    o = O.DADMM(p, z["eta1"])
    o.load_state(*before)
    o.iterate(p["sino"])
    compare_states(gpu_state(s), o, p)
    u, lam = s.u.cpu().numpy(), s.lam.cpu().numpy()
    xs, home = s.xseg.cpu().numpy()[0], s.home_view().cpu().numpy()[0]
    xo, ho = z["xseg"][0].astype(np.float64), z["home"][0].astype(np.float64)
    drift = float(np.linalg.norm(home - ho))
    b_gpu = quantization_bounds(p, xs, home)
    b_orc = quantization_bounds(p, xo, ho)
    dx = float(np.linalg.norm(xs - xo))
    print("%s after 100 free-running iterations: rel-L2 u %.3e, x %.3e, lambda %.3e; reconstruction drift %.3e "
          "(relative %.3e) <= bound %.3e = ||dx|| %.3e + b_gpu %.3e + b_orc %.3e; realized quantization "
          "errors %.3e / %.3e" % (name, sampled_rel(u, z["u_idx"], z["u_val"]), rel_l2(xs, xo),
                                  sampled_rel(lam, z["u_idx"], z["lam_val"]), drift, drift / np.linalg.norm(ho),
                                  dx + b_gpu + b_orc, dx, b_gpu, b_orc, np.linalg.norm(xs - home),
                                  np.linalg.norm(xo - ho)))
    assert drift <= dx + b_gpu + b_orc
    assert np.all(np.isfinite(u)) and np.all(np.isfinite(lam))


def test_unquantized_1024_follows_the_oracle_for_10_iterations():
    """1024^2, 1440 angles, 8 nodes (interleaved angles, complete graph), no
    quantizer, 10 iterations of the batched graph-captured form: the
    reconstruction at 65536 seeded pixels, <w, x> over all pixels, ||x||^2,
    u and lambda at seeded positions, and every statistic of the last
    iteration within 1e-3 of the FP64 oracle"""
    need_gpu()
    name = "c4_diff"
    z = golden(name)
    p, s, st = run_gpu(name, z)
    assert int(z["iters"]) == p["iters"] == 10
    x = s.home_view().cpu().numpy()[0].astype(np.float64)
    N = p["geometry"]["N"]
    w = np.random.default_rng(int(z["w_seed"])).standard_normal((N, N))
    assert abs(w.sum() - float(z["w_sum"])) <= 1e-9 * abs(float(z["w_sum"])) + 1e-9
    err_x = sampled_rel(x, z["x_idx"], z["x_val"])
    err_loss = abs(np.sum(w * x) - float(z["loss"])) / abs(float(z["loss"]))
    err_n2 = abs(np.sum(x * x) - float(z["x_norm2"])) / float(z["x_norm2"])
    err_u = sampled_rel(s.u.cpu().numpy(), z["u_idx"], z["u_val"])
    err_l = sampled_rel(s.lam.cpu().numpy(), z["u_idx"], z["lam_val"])
    print("c4 after 10 iterations: rel-L2 x %.3e (sampled), <w,x> %.3e, ||x||^2 %.3e, u %.3e, lambda %.3e"
          % (err_x, err_loss, err_n2, err_u, err_l))
    assert err_x <= 1e-3 and err_loss <= 1e-3 and err_n2 <= 1e-3
    assert err_u <= 1e-3 and err_l <= 1e-3
    for j in range(4):
        assert rel_l2(st[:, 0, j], z["stats"][:, 0, j]) <= 1e-3, j
    assert np.array_equal(st[:, 0, 4], z["stats"][:, 0, 4])
