"""tomo_project_noalloc: the projection entry point for callers that cannot
allocate device memory (e.g. code that runs while a CUDA graph is captured,
or under a fixed device-memory budget). Called through the C ABI, its output
must match tomo_project's on two calls in a row (the second reuses the fixed
work-list array the first one filled), and requests beyond its fixed
capacity must be refused without launching anything.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_common import need_gpu, rel_l2
from paper_2410_06106_gb300 import api, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5  # the projector parity tolerance used by the other GPU tests

TOMO_ERR_WORKSPACE = -3


def call_noalloc(lib, geo, img, out, sel, batch, sub=None):
    arr = np.ascontiguousarray(sel, np.int32)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.tomo_project_noalloc(geo.handle, C.c_void_p(img.data_ptr()), C.c_void_p(out.data_ptr()),
                                  arr.ctypes.data_as(C.c_void_p), len(arr), batch,
                                  C.c_void_p(sub.data_ptr()) if sub is not None else None, stream)
    return rc


def test_noalloc_projection_matches_tomo_project_twice():
    need_gpu()
    lib = api.lib()
    N, B, A = 192, 273, 96
    geo = api.Geometry(N, B, synth.angles(A))
    rng = np.random.default_rng(2024)
    cases = [  # (angle selection, batch, subtract?)
        (np.arange(0, A, 3, dtype=np.int32), 2, False),
        (rng.choice(A, 40, replace=False).astype(np.int32), 3, True),
    ]
    refs, inputs = [], []
    for sel, batch, with_sub in cases:  # reference results first, with the existing entry point
        img = torch.as_tensor(rng.random((batch, N, N), dtype=np.float32)).cuda()
        sub = torch.as_tensor(rng.random((batch, len(sel), B), dtype=np.float32)).cuda() if with_sub else None
        refs.append(geo.project(img, sel, subtract=sub).cpu().numpy())
        inputs.append((img, sub))
    for (sel, batch, _), (img, sub), ref in zip(cases, inputs, refs):  # two calls in a row
        out = torch.full((batch, len(sel), B), float("nan"), device="cuda")
        assert call_noalloc(lib, geo, img, out, sel, batch, sub) == 0, lib.tomo_last_error()
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref) <= TOL
    geo.close()


def test_noalloc_rejects_requests_beyond_its_capacity():
    need_gpu()
    lib = api.lib()
    N, B, A = 64, 2048 * 4 + 1, 8  # 8193 bins: 129 runs of 64 per angle group
    geo = api.Geometry(N, B, synth.angles(A))
    sel = np.zeros(4096, np.int32)  # 4096 single-angle groups x 33+ runs > 16384 items
    img = torch.zeros(1, N, N, device="cuda")
    out = torch.zeros(1, 8, 8, device="cuda")  # never written: the call must refuse before any launch
    rc = call_noalloc(lib, geo, img, out, sel, 1)
    assert rc == TOMO_ERR_WORKSPACE
    assert b"capacity" in lib.tomo_last_error()
    too_many = np.zeros(8193, np.int32)
    assert call_noalloc(lib, geo, img, out, too_many, 1) == TOMO_ERR_WORKSPACE
    geo.close()
