#!/usr/bin/env python
"""Write the FP64 oracle trajectories that the full-size GPU parity tests
compare against: tests/golden/<shape>_trajectory.npz.

Only the FP64 oracle (oracle/) and the seeded input generators
(paper_2410_06106_gb300.synth, which hold none of the method's arithmetic)
are called, so no stored value comes from the CUDA path. The step sizes
eta1_m = 1 / (||P_m||^2 + rho) come from the oracle's own power iteration
and are stored with the trajectory: the GPU test passes them to its solver
(the paper treats eta1 as an input of Algorithm 2).

Per shape (Algorithm 4 with Algorithms 2, 3, 5 and Eq. 15-18, 21-24, run
from zero for the shape's stated iteration count):
  eta1, opnorm2, power_iters    the step sizes and the norms they came from
  stats [iters, S, 5]           every iteration's FP64 statistics
  u_idx, u_val, lam_val         u and lambda at seeded flat positions of
                                [S, M, N, N] (the full arrays are too large
                                to store), with u_norm2 / lam_norm2 of the
                                full arrays
  xseg, home  (c2, c3)          the owners' unquantized segments and the
                                home-quantized reconstruction, float32
  x_idx, x_val, x_norm2, loss   (c4) the reconstruction at seeded pixels,
                                its squared norm and <w, x> with
                                w = default_rng(W_SEED).standard_normal
  loss_plus, loss_minus, h      (c4) <w, x> at rho (1 + h) and rho (1 - h),
                                eta1 held fixed: the FP64 central difference
                                of the loss in rho (the differentiation
                                check of the unrolled 10-iteration form)

Usage: python tests/golden/make_trajectory_goldens.py c2_kmeans c3_batch_jpeg c4_diff
Cost on 8 x86 cores: c2 ~5 min, c3 ~40 min, c4 ~100 min (three trajectories).
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2410_06106_gb300 import synth  # noqa: E402

SAMPLE = 65536
SAMPLE_SEED = 2410
W_SEED = 5
FD_H = 1e-4
POWER_ITERS = {"c2_kmeans": 60, "c3_batch_jpeg": 60, "c4_diff": 20}


def path(name):
    return os.path.join(HERE, "%s_trajectory.npz" % name)


def step_sizes(prob, iters):
    g = prob["geometry"]
    geo = O.Geometry(g["N"], g["B"], g["theta"])
    ptr, idx = prob["node_ang_ptr"], prob["node_ang"]
    L = np.array([geo.opnorm_sq(idx[ptr[m]:ptr[m + 1]], iters=iters, seed=1) for m in range(prob["M"])])
    return 1.0 / (L + prob["rho"]), L


def sample_index(n, seed):
    return np.sort(np.random.default_rng(seed).choice(n, min(SAMPLE, n), replace=False)).astype(np.int64)


def run(prob, eta, rho=None):
    o = O.DADMM(prob if rho is None else dict(prob, rho=rho), eta)
    stats = np.stack([o.iterate(prob["sino"]) for _ in range(prob["iters"])])
    return o, stats


def make(name):
    t0 = time.time()
    prob = synth.make_problem(name)
    eta, L = step_sizes(prob, POWER_ITERS[name])
    print("%s: step sizes (%.0f s)" % (name, time.time() - t0), flush=True)
    o, stats = run(prob, eta)
    print("%s: trajectory of %d iterations (%.0f s)" % (name, prob["iters"], time.time() - t0), flush=True)
    ui = sample_index(o.u.size, SAMPLE_SEED)
    out = dict(eta1=eta, opnorm2=L, power_iters=POWER_ITERS[name], iters=prob["iters"], stats=stats,
               u_idx=ui, u_val=o.u.ravel()[ui], lam_val=o.lam.ravel()[ui],
               u_norm2=float(np.sum(o.u * o.u)), lam_norm2=float(np.sum(o.lam * o.lam)))
    home = o.home_view()
    if name == "c4_diff":
        N = prob["geometry"]["N"]
        w = np.random.default_rng(W_SEED).standard_normal((N, N))
        xi = sample_index(N * N, SAMPLE_SEED + 1)
        out.update(x_idx=xi, x_val=home[0].ravel()[xi], x_norm2=float(np.sum(home * home)),
                   loss=float(np.sum(w * home[0])), w_seed=W_SEED, w_sum=float(w.sum()), h=FD_H)
        rho = float(prob["rho"])
        for key, r in (("loss_plus", rho * (1 + FD_H)), ("loss_minus", rho * (1 - FD_H))):
            o2, _ = run(prob, eta, r)
            out[key] = float(np.sum(w * o2.home_view()[0]))
            print("%s: %s (%.0f s)" % (name, key, time.time() - t0), flush=True)
    else:
        out.update(xseg=o.xseg.astype(np.float32), home=home.astype(np.float32))
    np.savez_compressed(path(name), **out)
    print("%s: wrote %s (%.0f s)" % (name, path(name), time.time() - t0), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("shapes", nargs="+", choices=sorted(POWER_ITERS))
    for name in ap.parse_args().shapes:
        make(name)


if __name__ == "__main__":
    main()
