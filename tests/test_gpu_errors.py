"""Failure handling injected on the host: invalid arguments are refused
before any launch with TOMO_ERR_INVALID_ARG, an undersized workspace is
refused, and non-finite data surfaces as TOMO_ERR_NUMERIC from the FP64
statistics (the iteration itself still runs). No GPU fault is provoked."""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_common import need_gpu
from paper_2410_06106_gb300 import api
from problems import small_problem

pytestmark = pytest.mark.gpu
INVALID, WORKSPACE, NUMERIC = -1, -3, -5


def test_invalid_arguments_are_refused():
    need_gpu()
    lib = api.lib()
    g = api.Geometry(16, 23, A=8)
    x = torch.zeros(16, 16, device="cuda")
    s = torch.zeros(8, 23, device="cuda")
    st = C.c_void_p(0)
    assert lib.tomo_project(g.handle, None, C.c_void_p(s.data_ptr()), None, 8, 1, None, st) == INVALID
    bad = np.array([0, 9], np.int32)
    assert lib.tomo_project(g.handle, C.c_void_p(x.data_ptr()), C.c_void_p(s.data_ptr()),
                            bad.ctypes.data_as(C.c_void_p), 2, 1, None, st) == INVALID
    assert b"out of range" in lib.tomo_last_error()
    assert lib.tomo_backproject(g.handle, C.c_void_p(s.data_ptr()), C.c_void_p(x.data_ptr()), None, 8, 1,
                                C.c_float(0.5), st) == INVALID
    h = C.c_void_p()
    assert lib.tomo_geometry_create(0, 23, 8, None, C.byref(h)) == INVALID
    with pytest.raises(api.TomoError):
        api.quant_jpeg(torch.zeros(12, 16, device="cuda"), 50)  # rows not a multiple of 8
    g.close()


def test_bad_configurations_are_refused_at_create():
    need_gpu()
    p = small_problem(N=16, A=16, B=23, M=4, graph="ring")
    eta = np.full(4, 0.01)
    p_disc = dict(p, adj=np.zeros((4, 4), np.int32))
    with pytest.raises(api.TomoError, match="connected"):
        api.DADMM(p_disc, eta)
    p_jpeg = small_problem(N=20, A=16, B=31, M=2, graph="ring", quant="jpeg")  # 10-row segments
    with pytest.raises(api.TomoError, match="multiples of 8"):
        api.DADMM(p_jpeg, np.full(2, 0.01))
    with pytest.raises(api.TomoError, match="positive"):
        api.DADMM(p, np.zeros(4))


def test_undersized_workspace_and_nonfinite_data():
    need_gpu()
    p = small_problem(N=16, A=16, B=23, M=2, graph="ring", quant="none")
    s = api.DADMM(p, np.full(2, 0.002))
    lib = api.lib()
    sino = torch.as_tensor(p["sino"]).cuda()
    rc = lib.dadmm_step(s.handle, C.byref(s._state), C.c_void_p(sino.data_ptr()), 1,
                        C.c_void_p(s.workspace.data_ptr()), s.ws_bytes - 1, None, C.c_void_p(0))
    assert rc == INVALID and b"workspace too small" in lib.tomo_last_error()
    assert s.k == 0  # nothing ran
    sino[0, 3, 5] = float("nan")
    with pytest.raises(api.TomoError) as e:
        s.step(sino, 1)
    assert e.value.code == NUMERIC
    assert s.k == 1


TIMEOUT = -4


def test_bounded_wait_timeout_is_reported_and_context_stays_usable():
    """the projector's bounded wait, run on a barrier that nothing completes
    (no copy in flight), gives up, the status word reports TOMO_ERR_TIMEOUT on
    the host, and the same context keeps computing correct projections"""
    need_gpu()
    lib = api.lib()
    g = api.Geometry(64, 91, A=90)
    x = torch.rand(64, 64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    ref = g.project(x)
    g.sync_status()  # clean
    assert lib.tomo_selftest_wait(g.handle, 20, C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    with pytest.raises(api.TomoError) as e:
        g.sync_status()
    assert e.value.code == TIMEOUT and b"bounded wait" in lib.tomo_last_error()
    g.sync_status()  # the read reset the word
    assert torch.equal(g.project(x), ref)
    g.sync_status()
    assert lib.tomo_selftest_wait(g.handle, 0, None) == INVALID
    g.close()


def test_dadmm_status_without_stats():
    need_gpu()
    p = small_problem(N=16, A=16, B=23, M=2, graph="ring", quant="none")
    s = api.DADMM(p, np.full(2, 0.002))
    sino = torch.as_tensor(p["sino"]).cuda()
    s.step(sino, 2, stats=False)
    s.sync_status()
    sino[0, 3, 5] = float("nan")
    s.step(sino, 1, stats=False)
    with pytest.raises(api.TomoError) as e:
        s.sync_status()
    assert e.value.code == NUMERIC
