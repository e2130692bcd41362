"""GPU parity of the projector and matched backprojector (Eq. 2-4) against
the FP64 oracle: full outputs at sizes the oracle finishes in seconds (several
tiles, ragged edges, odd/even sizes, subsets, batches, axis-aligned rays),
sampled rays and pixels at the full problem sizes, and the FP32 adjoint test.
Tolerance: relative L2 <= 1e-5 (FP32 arithmetic and accumulation)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import cuda, need_gpu, rel_l2
from paper_2410_06106_gb300 import api, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.mark.parametrize("N,B,A,off", [(64, 91, 90, 0.0), (37, 54, 23, 0.013), (130, 187, 60, 0.4),
                                       (256, 367, 72, 0.0), (8, 13, 16, 0.0), (5, 3, 7, 0.2)])
def test_project_and_backproject_match_oracle(N, B, A, off):
    need_gpu()
    theta = synth.angles(A) + off
    g = api.Geometry(N, B, theta)
    og = O.Geometry(N, B, theta)
    rng = np.random.default_rng(N + A)
    img = rng.random((N, N)).astype(np.float32)
    sino = rng.standard_normal((A, B)).astype(np.float32)
    d_gpu = g.project(cuda(img)).cpu().numpy()
    assert rel_l2(d_gpu, og.project(img)) <= TOL
    b_gpu = g.backproject(cuda(sino)).cpu().numpy()
    assert rel_l2(b_gpu, og.backproject(sino)) <= TOL
    g.close()


def test_axis_aligned_single_pixels_are_exact():
    need_gpu()
    N, B = 8, 13
    theta = np.array([0.0, math.pi / 2, math.pi / 4])
    g = api.Geometry(N, B, theta)
    og = O.Geometry(N, B, theta)
    for (i, j) in [(0, 0), (3, 4), (7, 7)]:
        img = np.zeros((N, N), np.float32)
        img[i, j] = 1.0
        d = g.project(cuda(img)).cpu().numpy()
        ref = og.project(img)
        assert np.array_equal(d[:2], ref[:2].astype(np.float32))  # 1/2 on pixel edges, exactly
        assert np.abs(d[2] - ref[2]).max() < 1e-6


def test_subset_batch_and_subtract():
    need_gpu()
    N, B, A = 48, 71, 40
    theta = synth.angles(A)
    g = api.Geometry(N, B, theta)
    og = O.Geometry(N, B, theta)
    rng = np.random.default_rng(7)
    sel = np.array([39, 0, 17, 20, 5, 33], np.int32)
    img = rng.random((3, N, N)).astype(np.float32)
    sub = rng.random((3, len(sel), B)).astype(np.float32)
    d = g.project(cuda(img), sel, subtract=cuda(sub)).cpu().numpy()
    assert rel_l2(d, og.project(img, sel) - sub) <= TOL
    out = cuda(img)
    g.backproject(cuda(sub), sel, out=out, beta=1.0)
    assert rel_l2(out.cpu().numpy(), img + og.backproject(sub, sel)) <= TOL


def test_fp32_adjoint_dot_product():
    need_gpu()
    N, B, A = 200, 287, 64
    g = api.Geometry(N, B, synth.angles(A) + 0.01)
    rng = np.random.default_rng(1)
    x, y = cuda(rng.standard_normal((N, N))), cuda(rng.standard_normal((A, B)))
    lhs = torch.sum(g.project(x).double() * y.double()).item()
    rhs = torch.sum(x.double() * g.backproject(y).double()).item()
    assert abs(lhs - rhs) <= 1e-5 * math.sqrt(
        torch.sum(g.project(x).double() ** 2).item() * torch.sum(y.double() ** 2).item())


def test_operator_norm_matches_oracle():
    need_gpu()
    N, B, A = 32, 47, 20
    theta = synth.angles(A)
    sel = np.arange(0, A, 3, dtype=np.int32)
    L_gpu = api.Geometry(N, B, theta).opnorm_sq(sel, iters=200)
    L_orc = O.Geometry(N, B, theta).opnorm_sq(sel, iters=200)
    assert abs(L_gpu - L_orc) <= 1e-4 * L_orc


@pytest.mark.parametrize("name", ["c4_diff", "c5_stress"])
def test_full_size_sampled_rays_and_pixels(name):
    """the full image and detector sizes of the two largest problems, every
    angle of the geometry; rays and pixels sampled for the oracle"""
    need_gpu()
    cfg = synth.CONFIGS[name]
    N, A, B = cfg["N"], cfg["A"], cfg["B"]
    theta = synth.angles(A)
    g = api.Geometry(N, B, theta)
    og = O.Geometry(N, B, theta)
    rng = np.random.default_rng(cfg["idx"])
    ell = synth.random_ellipses(N, 12, rng)
    img = (synth.rasterize(ell, N, ss=1) + 0.05 * rng.random((N, N))).astype(np.float32)
    sel = np.concatenate([[0, A // 4, A // 2, 3 * A // 4], rng.choice(A, 12, replace=False)]).astype(np.int32)
    d = g.project(cuda(img), sel).cpu().numpy()
    q = rng.integers(0, len(sel), 96)
    b = rng.integers(B // 6, 5 * B // 6, 96)
    ref = og.project_rays(img, sel[q], b)
    assert rel_l2(d[q, b], ref) <= TOL
    sino = rng.standard_normal((A, B)).astype(np.float32)
    bp = g.backproject(cuda(sino)).cpu().numpy().ravel()
    pix = rng.integers(0, N * N, 96)
    ref = og.backproject_pixels(sino, pix)
    assert rel_l2(bp[pix], ref) <= TOL
    g.close()
