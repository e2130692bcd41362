"""Algorithm 1 (CTR, Eq. 5) on the library's kernels against the FP64 oracle,
and one short pass of every experiment of the driver (Sec. 3) at the paper's
512 x 512, 804-angle shape."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import cuda, need_gpu, rel_l2
from paper_2410_06106_gb300 import api
from paper_2410_06106_gb300 import experiments as X
from problems import small_problem

pytestmark = pytest.mark.gpu


def test_ctr_follows_the_oracle():
    need_gpu()
    N, A, B = 64, 48, 91
    p = small_problem(N=N, A=A, B=B, noise=0.01, seed=5)
    og = O.Geometry(N, B, p["geometry"]["theta"])
    eta = 1.0 / og.opnorm_sq(iters=60)
    want = og.ctr(p["sino"][0], eta, 30)
    g = api.Geometry(N, B, p["geometry"]["theta"])
    got = X.ctr(cuda(p["sino"][0]), g, eta, 30).cpu().numpy()
    assert rel_l2(got, want) <= 1e-4
    g.close()


def test_every_experiment_runs_and_reports():
    need_gpu()
    r = X.exp_ctr_vs_dadmm(2)
    assert set(r) == {"CTR", "dADMM, 2 nodes", "dADMM, 10 nodes"}
    assert all(np.isfinite(v["rmse"]) for v in r.values())
    e = X.exp_elbow(2, ks=(2, 3), qualities=(50,))
    assert e["kmeans"][2]["bits_per_value"] < e["kmeans"][3]["bits_per_value"]
    n = X.exp_noise(2, km_k=4, jpeg_quality=50)
    assert len(n["levels"]) == len(X.NSD_LEVELS)
    assert all(len(v["kmeans"]["rmse_per_iteration"]) == 2 for v in n["levels"].values())
    torch.cuda.synchronize()
