"""Edge cases of the boundary against the FP64 oracle: the largest image and
detector a geometry accepts (sampled rays and pixels), the smallest ones
(one or two pixels, one bin, one angle), empty requests (refused before any
launch), a zero-iteration step (no work, state unchanged), and the
single-node problem (no messages: Algorithm 4 with M = 1)."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import cuda, need_gpu, rel_l2
from paper_2410_06106_gb300 import api, synth
from problems import oracle_eta1, small_problem

pytestmark = pytest.mark.gpu
INVALID = -1


def test_largest_image_and_detector():
    """N = 8192 pixels a side and 16384 bins (the geometry limits), 8 angles
    including the axes and the diagonal: rays and pixels sampled for the oracle"""
    need_gpu()
    N, B = 8192, 16384
    theta = np.array([0.0, 0.3, np.pi / 4, 1.2, np.pi / 2, 2.0, 2.6, 3.0])
    g = api.Geometry(N, B, theta)
    og = O.Geometry(N, B, theta)
    rng = np.random.default_rng(3)
    img = rng.random((N, N), dtype=np.float32)
    d = g.project(cuda(img)).cpu().numpy()
    ra = rng.integers(0, len(theta), 24)
    rb = rng.integers(B // 2 - N // 2, B // 2 + N // 2, 24)  # rays that cross the image
    assert rel_l2(d[ra, rb], og.project_rays(img, ra, rb)) <= 1e-5
    assert np.all(d[:, :B // 2 - int(0.71 * N) - 2] == 0)  # bins whose rays miss the image
    sino = rng.standard_normal((len(theta), B)).astype(np.float32)
    bp = g.backproject(cuda(sino)).cpu().numpy().ravel()
    pix = np.concatenate([[0, N - 1, N * N - N, N * N - 1], rng.integers(0, N * N, 28)])
    assert rel_l2(bp[pix], og.backproject_pixels(sino, pix)) <= 1e-5
    g.close()


@pytest.mark.parametrize("N,B,A", [(1, 1, 1), (1, 3, 5), (2, 1, 4), (2, 5, 7), (3, 2, 3)])
def test_smallest_geometries(N, B, A):
    need_gpu()
    theta = synth.angles(A) + 0.1
    g = api.Geometry(N, B, theta)
    og = O.Geometry(N, B, theta)
    rng = np.random.default_rng(N * 100 + B * 10 + A)
    img = rng.random((2, N, N)).astype(np.float32)
    assert rel_l2(g.project(cuda(img)).cpu().numpy(), og.project(img)) <= 1e-5
    r = rng.standard_normal((2, A, B)).astype(np.float32)
    assert rel_l2(g.backproject(cuda(r)).cpu().numpy(), og.backproject(r)) <= 1e-5
    g.close()


def test_empty_requests_are_refused():
    need_gpu()
    lib = api.lib()
    g = api.Geometry(16, 23, A=8)
    x = torch.zeros(16, 16, device="cuda")
    s = torch.zeros(8, 23, device="cuda")
    st = C.c_void_p(0)
    sel = np.array([0], np.int32)
    for n_sel, batch in [(0, 1), (1, 0)]:
        assert lib.tomo_project(g.handle, C.c_void_p(x.data_ptr()), C.c_void_p(s.data_ptr()),
                                sel.ctypes.data_as(C.c_void_p), n_sel, batch, None, st) == INVALID
        assert lib.tomo_backproject(g.handle, C.c_void_p(s.data_ptr()), C.c_void_p(x.data_ptr()),
                                    sel.ctypes.data_as(C.c_void_p), n_sel, batch, C.c_float(0.0), st) == INVALID
    g.close()


def test_zero_iterations_change_nothing():
    need_gpu()
    p = small_problem(N=32, A=24, B=47, M=4, graph="ring", quant="alternate", noise=0.02, seed=2, km_k=8)
    s = api.DADMM(p, oracle_eta1(p))
    sino = torch.as_tensor(p["sino"]).cuda()
    s.step(sino, 2)
    before = {n: getattr(s, n).clone() for n in ("u", "lam", "xseg", "hist", "iter")}
    s.step(sino, 0, stats=False)
    for n, v in before.items():
        assert torch.equal(getattr(s, n), v), n


def test_single_node_trajectory():
    """M = 1: no graph and no messages but the node's own segment (the whole
    image); Algorithm 4 then alternates a proximal gradient step and the
    x-step of Algorithm 3"""
    need_gpu()
    p = small_problem(N=32, A=40, B=47, M=1, quant="none", noise=0.02, seed=4)
    eta = oracle_eta1(p)
    s = api.DADMM(p, eta)
    st = s.step(torch.as_tensor(p["sino"]).cuda(), 15)
    o = O.DADMM(p, eta)
    ost = np.stack([o.iterate(p["sino"]) for _ in range(15)])
    assert rel_l2(s.u.cpu().numpy(), o.u) <= 1e-4
    assert rel_l2(s.home_view().cpu().numpy(), o.home_view()) <= 1e-4
    assert np.all(st[:, :, 4] == ost[:, :, 4])  # bytes on the wire: none
    assert rel_l2(st[:, :, 0], ost[:, :, 0]) <= 1e-3
