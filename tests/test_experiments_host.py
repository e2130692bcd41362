"""Host logic of the experiment driver (Sec. 3): the image quality measures,
the noise model of the NSD sweep and the node layouts of the Fig. 4
comparison. The experiments themselves run on the GPU
(tests/test_gpu_experiments.py)."""
import math

import numpy as np

from paper_2410_06106_gb300 import experiments as X
from paper_2410_06106_gb300 import synth


def test_rmse_and_psnr_follow_their_definitions():
    truth = np.zeros((4, 4))
    truth[1, 2] = 2.0
    x = truth + np.array([[1.0, -1.0, 0, 0]] * 4)  # 8 errors of magnitude 1
    assert X.rmse(x, truth) == math.sqrt(8 / 16)
    assert X.psnr(x, truth) == 20 * math.log10(2.0 / math.sqrt(0.5))
    assert X.psnr(truth, truth) == float("inf")


def test_noise_is_nsd_times_the_peak():
    d = np.full((200, 300), 7.0)
    d[0, 0] = 410.0
    for nsd in (0.0024, 0.0243):
        e = X.noisy(d, nsd, seed=1) - d
        assert abs(np.std(e) / (nsd * 410.0) - 1.0) < 0.02
    assert np.array_equal(X.noisy(d, 0.0, seed=1), d.astype(np.float32))


def test_interleaved_nodes_on_a_complete_graph():
    sino = np.zeros((804, 725), np.float32)
    p = X.dadmm_problem(sino, synth.angles(804), 512, 10)
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    # the paper's 10-node split: node m holds m, m + 10, ...; the first four hold 81 angles
    assert [ptr[m + 1] - ptr[m] for m in range(10)] == [81] * 4 + [80] * 6
    assert list(idx[ptr[1]:ptr[1] + 3]) == [1, 11, 21]
    assert np.array_equal(p["adj"], 1 - np.eye(10, dtype=np.int32))
    seg = p["seg_row_ptr"]  # whole 8-row blocks (JPEG messages), near-equal
    assert list(np.diff(seg)) == [56] * 4 + [48] * 6 and seg[-1] == 512
    q = X.dadmm_problem(sino, synth.angles(804), 512, 2, "kmeans", km_k=3)
    assert [q["node_ang_ptr"][m + 1] - q["node_ang_ptr"][m] for m in range(2)] == [402, 402]
    assert np.all(q["home_q"] == synth.KIND_KMEANS) and q["km_k"] == 3
