"""tomo_project_noalloc: the projection entry point for callers that cannot
allocate device memory (e.g. code that runs while a CUDA graph is captured
elsewhere in the process, or under a fixed device-memory budget). Called
through the C ABI, its output must match the FP64 oracle and tomo_project's
on two calls in a row (the second reuses the fixed work-list array the first
one filled), requests right at its capacity must be accepted and correct,
requests beyond it refused without launching anything, and a stream that is
capturing a CUDA graph refused with nothing enqueued.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import need_gpu, rel_l2
from paper_2410_06106_gb300 import api, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5  # the projector parity tolerance used by the other GPU tests

TOMO_ERR_INVALID_ARG = -1
TOMO_ERR_WORKSPACE = -3
MAX_ITEMS = 16384  # the fixed array's capacity: work items and angles
MAX_ANGLES = 8192


def call_noalloc(lib, geo, img, out, sel, batch, sub=None, stream=None):
    arr = np.ascontiguousarray(sel, np.int32)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.tomo_project_noalloc(geo.handle, C.c_void_p(img.data_ptr()), C.c_void_p(out.data_ptr()),
                                  arr.ctypes.data_as(C.c_void_p), len(arr), batch,
                                  C.c_void_p(sub.data_ptr()) if sub is not None else None,
                                  C.c_void_p(st.cuda_stream))
    return rc


def oracle_project(N, B, theta, img, sel, sub=None):
    want = O.Geometry(N, B, theta).project(img.cpu().numpy(), sel)
    return want if sub is None else want - sub.cpu().numpy()


def test_noalloc_projection_matches_oracle_and_tomo_project_twice():
    need_gpu()
    lib = api.lib()
    N, B, A = 192, 273, 96
    theta = synth.angles(A)
    geo = api.Geometry(N, B, theta)
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
        got = out.cpu().numpy()
        assert rel_l2(got, oracle_project(N, B, theta, img, sel, sub)) <= TOL
        assert rel_l2(got, ref) <= TOL
    geo.close()


def test_noalloc_requests_at_the_capacity_are_accepted():
    """(a) exactly MAX_ITEMS work items: 2048 selections of one angle form 512
    four-angle groups, each split into ceil(B / 128) = 32 bin runs, in a batch
    of one; (b) MAX_ANGLES selected angles (every angle of a 4096-angle
    geometry twice) in one batch. Both match the oracle and tomo_project."""
    need_gpu()
    lib = api.lib()
    N = 48
    for A, B, sel, batch in [(16, 32 * 128, np.full(2048, 3, np.int32), 1),
                             (4096, 71, np.arange(MAX_ANGLES, dtype=np.int32) % 4096, 1)]:
        theta = synth.angles(A)
        geo = api.Geometry(N, B, theta)
        rng = np.random.default_rng(A)
        img = torch.as_tensor(rng.random((batch, N, N), dtype=np.float32)).cuda()
        out = torch.full((batch, len(sel), B), float("nan"), device="cuda")
        assert call_noalloc(lib, geo, img, out, sel, batch) == 0, lib.tomo_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert rel_l2(got, geo.project(img, sel).cpu().numpy()) <= TOL
        # the oracle on a sample of the selected rows (every row is a separate ray set)
        rows = rng.choice(len(sel), 64, replace=False)
        want = O.Geometry(N, B, theta).project(img[0].cpu().numpy(), sel[rows])
        assert rel_l2(got[0, rows], want) <= TOL
        geo.close()


def test_noalloc_rejects_requests_beyond_its_capacity():
    """MAX_ITEMS + 1 items (565 groups of 29 bin runs: 2256 selections of one
    angle form 564 four-angle groups, one more makes a single-angle group) and
    MAX_ANGLES + 1 angles are refused with TOMO_ERR_WORKSPACE before anything
    runs: an output buffer of the full request's size stays untouched"""
    need_gpu()
    lib = api.lib()
    N, B, A = 64, 29 * 128, 8
    geo = api.Geometry(N, B, synth.angles(A))
    img = torch.zeros(1, N, N, device="cuda")
    sel = np.zeros(4 * 564 + 1, np.int32)
    out = torch.full((1, len(sel), B), float("nan"), device="cuda")
    rc = call_noalloc(lib, geo, img, out, sel, 1)
    assert rc == TOMO_ERR_WORKSPACE
    assert b"capacity" in lib.tomo_last_error()
    ok = np.zeros(4 * 564, np.int32)  # one angle fewer: 564 x 29 = 16356 items, accepted
    out_ok = torch.full((1, len(ok), B), float("nan"), device="cuda")
    assert call_noalloc(lib, geo, img, out_ok, ok, 1) == 0, lib.tomo_last_error()
    too_many = np.zeros(MAX_ANGLES + 1, np.int32)
    out2 = torch.full((1, len(too_many), B), float("nan"), device="cuda")
    assert call_noalloc(lib, geo, img, out2, too_many, 1) == TOMO_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert torch.isnan(out).all() and torch.isnan(out2).all()
    assert torch.equal(out_ok, torch.zeros_like(out_ok))  # zero image: zero projection
    geo.close()


def test_noalloc_refuses_a_capturing_stream():
    """the work list is copied from host memory that lives only during the
    call, so on a stream that is capturing a graph the call is refused with
    TOMO_ERR_INVALID_ARG and enqueues nothing; the stream works normally
    afterwards"""
    need_gpu()
    lib = api.lib()
    N, B, A = 32, 47, 12
    theta = synth.angles(A)
    geo = api.Geometry(N, B, theta)
    img = torch.rand(1, N, N, device="cuda")
    sel = np.arange(A, dtype=np.int32)
    out = torch.full((1, A, B), float("nan"), device="cuda")
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        graph.capture_begin(capture_error_mode="relaxed")
        try:
            rc = call_noalloc(lib, geo, img, out, sel, 1, stream=st)
        finally:
            graph.capture_end()
    assert rc == TOMO_ERR_INVALID_ARG
    assert b"capturing" in lib.tomo_last_error()
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
    assert call_noalloc(lib, geo, img, out, sel, 1, stream=st) == 0, lib.tomo_last_error()
    st.synchronize()
    assert rel_l2(out.cpu().numpy(), oracle_project(N, B, theta, img, sel)) <= TOL
    del graph
    geo.close()
