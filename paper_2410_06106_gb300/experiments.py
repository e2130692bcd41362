"""The paper's experiments (Sec. 3) on synthetic data, run on the library's kernels.

- Algorithm 1 (CTR, Eq. 5), the centralized baseline: E gradient steps
  u <- u - eta P^T (P u - d) from zero, every step in libtomo kernels (projector
  with subtraction, backprojector, linear combination).
- Sec. 3.2 / Fig. 4: CTR against dADMM without quantization on 2 and 10 nodes
  holding interleaved angles (node m takes angles m, m + M, ...).
- Sec. 3.3 / Fig. 5: the elbow sweep of dADMM-K over the number of centres K,
  and the JPEG quality sweep of dADMM-J, RMSE against the message size.
- Sec. 3.3 / Figs. 6-7: dADMM-K and dADMM-J at the paper's noise levels
  NSD = sigma / x_peak (0, 0.24 %, 0.77 %, 2.43 %), x_peak the largest value of
  the noise-free sinogram.
- Sec. 3.3 / Fig. 8: RMSE after every outer iteration.

The paper's Phantom and Barbara images are not available: random-ellipse
phantoms stand in for them, shaped like its setup (512 x 512 pixels, 804
angles uniform on [0, 180 deg), 725 unit bins so that the unpadded image's
diagonal is covered), with RMSE and PSNR taken against the 4 x 4
supersampled phantom (Sec. 3, the RMSE and PSNR definitions).

Run: python -m paper_2410_06106_gb300.experiments [--iters K] [--out results.json]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import api, synth

PAPER_SHAPE = dict(N=512, A=804, B=725, ellipses=20)
NSD_LEVELS = (0.0, 0.0024, 0.0077, 0.0243)


# --------------------------------------------------------------------------
# Algorithm 1 and the image quality measures
# --------------------------------------------------------------------------

def ctr(sino, geom, eta, E, u0=None, every=None):
    """Algorithm 1: E steps of u <- u - eta P^T (P u - d) over every angle from
    u0 (zero by default). sino [..., A, B] CUDA float32; returns u [..., N, N]
    (and, with every=(k, f), the values f(u) after every k-th step)"""
    lead = sino.shape[:-2]
    u = torch.zeros(*lead, geom.N, geom.N, device=sino.device) if u0 is None else u0.clone()
    trace = []
    for e in range(E):
        r = geom.project(u, subtract=sino)
        g = geom.backproject(r)
        u = api.lincomb([u, g], [1.0, -float(eta)], out=u)
        if every is not None and (e + 1) % every[0] == 0:
            trace.append(every[1](u))
    return (u, trace) if every is not None else u


def rmse(x, truth):
    """root mean square error over the pixels (Sec. 3)"""
    x = np.asarray(x, np.float64)
    t = np.asarray(truth, np.float64)
    return float(np.sqrt(np.mean((x - t) ** 2)))


def psnr(x, truth):
    """20 log10(I_max / RMSE), I_max the largest value of the true image (Sec. 3)"""
    e = rmse(x, truth)
    imax = float(np.max(truth))
    return float("inf") if e == 0 else 20.0 * math.log10(imax / e)


# --------------------------------------------------------------------------
# problems shaped like the paper's setup
# --------------------------------------------------------------------------

def paper_data(seed=0, shape=PAPER_SHAPE):
    """noise-free analytic sinogram [A, B], the phantom [N, N] and the angles"""
    rng = np.random.default_rng(synth.SEED_BASE + 9000 + seed)
    N, A, B = shape["N"], shape["A"], shape["B"]
    theta = synth.angles(A)
    ell = synth.random_ellipses(N, shape["ellipses"], rng)
    return synth.ellipse_sinogram(ell, theta, B), synth.rasterize(ell, N), theta


def noisy(d, nsd, seed):
    """d + N(0, (nsd x_peak)^2), x_peak = max d: the paper's NSD (Sec. 3.3)"""
    if nsd == 0:
        return np.asarray(d, np.float32)
    rng = np.random.default_rng(synth.SEED_BASE + 9500 + seed)
    return synth.add_noise(d, nsd, rng).astype(np.float32)


def segments_of_8(N, M):
    """row bands of whole 8-row blocks (what JPEG messages need), near-equal: the
    first (N / 8) mod M owners take one block more"""
    base, extra = divmod(N // 8, M)
    rows = [8 * (base + (m < extra)) for m in range(M)]
    rows[-1] += N - sum(rows)  # N not a multiple of 8: the last band takes the rest
    return np.concatenate([[0], np.cumsum(rows)]).astype(np.int32)


def dadmm_problem(sino, theta, N, M, quant="none", km_k=16, jpeg_quality=50, E1=10, E2=10, rho=1.0,
                  eta2=0.2, seed=0):
    """M nodes with interleaved angles on a complete graph (the paper's all-to-all
    exchange), one slice, segments of whole 8-row blocks; quant: none, kmeans or
    jpeg on every message"""
    A, B = sino.shape
    ptr, idx = synth.csr(synth.partition_interleaved(A, M))
    adj = synth.complete(M) if M > 1 else np.zeros((1, 1), np.int32)
    kind = {"none": synth.KIND_NONE, "kmeans": synth.KIND_KMEANS, "jpeg": synth.KIND_JPEG}[quant]
    return dict(name="paper", geometry=dict(N=N, A=A, B=B, theta=theta), M=M, S=1, node_ang_ptr=ptr,
                node_ang=idx, seg_row_ptr=segments_of_8(N, M), adj=adj,
                edge_q=synth.uniform_edge_kinds(adj, kind), home_q=np.full(M, kind, np.int32), km_k=km_k,
                jpeg_quality=jpeg_quality, seed=synth.SEED_BASE + 9700 + seed, sino=sino[None], rho=rho,
                eta2=eta2, E1=E1, E2=E2, km_iters=10)


def step_sizes(geom, prob, iters=30):
    """eta1_m = 1 / (||P_m||^2 + rho), ||P_m||^2 by power iteration on the GPU"""
    ptr, idx = prob["node_ang_ptr"], prob["node_ang"]
    L = np.array([geom.opnorm_sq(idx[ptr[m]:ptr[m + 1]], iters=iters) for m in range(prob["M"])])
    return 1.0 / (L + prob["rho"])


def run_dadmm(geom, prob, truth, iters, trace=False):
    """iters outer iterations; returns the final RMSE / PSNR, the best RMSE and
    its iteration, the message bytes per iteration and (trace) RMSE per iteration"""
    s = api.DADMM(prob, step_sizes(geom, prob), geometry=geom)
    sino = torch.as_tensor(prob["sino"]).cuda()
    hist, nbytes = [], 0.0
    for _ in range(iters):
        st = s.step(sino, 1, stats=True)
        nbytes = float(st[0, 0, 4])
        if trace:
            hist.append(rmse(s.home_view().cpu().numpy()[0], truth))
    x = s.home_view().cpu().numpy()[0]
    out = {"rmse": rmse(x, truth), "psnr": psnr(x, truth), "bytes_per_iteration": nbytes}
    if trace:
        out["rmse_per_iteration"] = hist
        b = int(np.argmin(hist))
        out["best_rmse"], out["best_iteration"] = hist[b], b + 1
    del s
    return out


# --------------------------------------------------------------------------
# the experiments
# --------------------------------------------------------------------------

def exp_ctr_vs_dadmm(iters, seed=0):
    """Fig. 4: CTR and unquantized dADMM on 2 and 10 interleaved nodes, noise-free;
    CTR runs E1 x iters steps (the same number of operator applies per node)"""
    d, truth, theta = paper_data(seed)
    N, A, B = PAPER_SHAPE["N"], PAPER_SHAPE["A"], PAPER_SHAPE["B"]
    geom = api.Geometry(N, B, theta)
    sino = noisy(d, 0.0, seed)
    L = geom.opnorm_sq(None, iters=30)
    out = {}
    u = ctr(torch.as_tensor(sino).cuda(), geom, 1.0 / L, 10 * iters)
    x = u.cpu().numpy()
    out["CTR"] = {"rmse": rmse(x, truth), "psnr": psnr(x, truth), "steps": 10 * iters}
    for M in (2, 10):
        out["dADMM, %d nodes" % M] = run_dadmm(geom, dadmm_problem(sino, theta, N, M), truth, iters, trace=True)
    geom.close()
    return out


def exp_elbow(iters, seed=0, ks=(2, 3, 4, 5, 6, 8, 16, 32), qualities=(10, 30, 50, 75, 90)):
    """Fig. 5: dADMM-K over K and dADMM-J over the JPEG quality, 10 nodes,
    noise-free; RMSE against the message size (bits per value)"""
    d, truth, theta = paper_data(seed)
    N, A, B = PAPER_SHAPE["N"], PAPER_SHAPE["A"], PAPER_SHAPE["B"]
    geom = api.Geometry(N, B, theta)
    sino = noisy(d, 0.0, seed)
    values = N * N * 9  # values sent per iteration: every segment to the 9 other nodes
    out = {"kmeans": {}, "jpeg": {}}
    for k in ks:
        r = run_dadmm(geom, dadmm_problem(sino, theta, N, 10, "kmeans", km_k=k), truth, iters)
        r["bits_per_value"] = 8.0 * r["bytes_per_iteration"] / values
        out["kmeans"][k] = r
    for q in qualities:
        r = run_dadmm(geom, dadmm_problem(sino, theta, N, 10, "jpeg", jpeg_quality=q), truth, iters)
        r["bits_per_value"] = 8.0 * r["bytes_per_iteration"] / values
        out["jpeg"][q] = r
    geom.close()
    return out


def exp_noise(iters, km_k, jpeg_quality, seed=0):
    """Figs. 6-8: dADMM-K and dADMM-J (10 nodes) at the paper's NSD levels, RMSE
    per iteration; plain K-means of the phantom with the same K for reference"""
    d, truth, theta = paper_data(seed)
    N, A, B = PAPER_SHAPE["N"], PAPER_SHAPE["A"], PAPER_SHAPE["B"]
    geom = api.Geometry(N, B, theta)
    out = {"kmeans_of_phantom": None, "levels": {}}
    t = torch.as_tensor(truth.astype(np.float32)).cuda()
    _, _, deq, _ = api.quant_kmeans(t.reshape(-1), km_k, 10, 12345)
    out["kmeans_of_phantom"] = {"K": km_k, "rmse": rmse(deq.cpu().numpy().reshape(N, N), truth)}
    for nsd in NSD_LEVELS:
        sino = noisy(d, nsd, seed)
        lv = {}
        for quant in ("kmeans", "jpeg"):
            lv[quant] = run_dadmm(geom, dadmm_problem(sino, theta, N, 10, quant, km_k=km_k,
                                                      jpeg_quality=jpeg_quality), truth, iters, trace=True)
        out["levels"]["%.2f%%" % (100 * nsd)] = lv
    geom.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=200, help="outer dADMM iterations of every run")
    ap.add_argument("--km-k", type=int, default=16)
    ap.add_argument("--jpeg-quality", type=int, default=50)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    t0 = time.time()
    res = {"shape": PAPER_SHAPE, "iters": args.iters,
           "ctr_vs_dadmm": exp_ctr_vs_dadmm(args.iters),
           "elbow": exp_elbow(args.iters),
           "noise": exp_noise(args.iters, args.km_k, args.jpeg_quality)}
    res["seconds"] = time.time() - t0

    def brief(r):
        return {k: v for k, v in r.items() if k != "rmse_per_iteration"}

    print("CTR vs dADMM (noise-free):")
    for k, v in res["ctr_vs_dadmm"].items():
        print("  %-18s %s" % (k, json.dumps(brief(v))))
    print("elbow (10 nodes, noise-free):")
    for kind in ("kmeans", "jpeg"):
        for k, v in res["elbow"][kind].items():
            print("  %-6s %-3s %s" % (kind, k, json.dumps(brief(v))))
    print("noise levels (10 nodes, K = %d, quality %d):" % (args.km_k, args.jpeg_quality))
    print("  K-means of the phantom itself: %s" % json.dumps(res["noise"]["kmeans_of_phantom"]))
    for lvl, v in res["noise"]["levels"].items():
        for quant, r in v.items():
            print("  NSD %-6s %-6s %s" % (lvl, quant, json.dumps(brief(r))))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1, default=float)


if __name__ == "__main__":
    main()
