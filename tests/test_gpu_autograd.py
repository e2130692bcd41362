"""Differentiation: the projector as a torch.autograd.Function (backward = the
matched backprojection kernel) and the unrolled 10-iteration unquantized
dADMM, differentiated with respect to rho and the sinogram with one
checkpoint per iteration. Checked against central finite differences of the
FP64 oracle (computed live on the small problem, stored by
tests/golden/make_trajectory_goldens.py at the full 1024^2 size) and of the
GPU forward (the sinogram direction, where the map is linear), and against
the oracle's adjoint."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import cuda, need_gpu, rel_l2
from paper_2410_06106_gb300 import api, autograd, synth
from problems import oracle_eta1, small_problem

pytestmark = pytest.mark.gpu


def test_project_function_adjoint_on_64_directions_full_size():
    """C4 geometry (1024^2, 1440 angles, 1449 bins): <w, P v> by central
    differences of the forward equals <P^T w, v> from autograd for 64 seeded
    directions; the autograd gradient equals the oracle's P^T w at sampled
    pixels"""
    need_gpu()
    cfg = synth.CONFIGS["c4_diff"]
    N, A, B = cfg["N"], cfg["A"], cfg["B"]
    theta = synth.angles(A)
    g = api.Geometry(N, B, theta)
    rng = np.random.default_rng(4)
    u0 = cuda(rng.random((N, N)))
    w = cuda(rng.standard_normal((A, B)))
    u = u0.clone().requires_grad_(True)
    y = autograd.project(u, g)
    (y * w).sum().backward()
    grad = u.grad.detach()
    wd = w.double()
    wn = torch.linalg.norm(wd).item()
    fd_err, dot_err = [], []
    for k in range(64):
        v = cuda(np.random.default_rng(100 + k).standard_normal((N, N)))
        yp, ym, pv = (g.project(t).double() for t in (u0 + v, u0 - v, v))
        fd = (torch.sum(yp * wd) - torch.sum(ym * wd)).item() / 2
        ad = torch.sum(grad.double() * v.double()).item()
        # errors on the scale of the FP32 values that were formed: |w| |P(u0 +- v)| for the
        # central difference, |w| |P v| for the dot test <w, P v> = <P^T w, v>
        fd_err.append(abs(fd - ad) / (wn * max(torch.linalg.norm(yp).item(), torch.linalg.norm(ym).item())))
        dot_err.append(abs(torch.sum(pv * wd).item() - ad) / (wn * torch.linalg.norm(pv).item()))
    assert max(fd_err) <= 1e-5, max(fd_err)
    assert max(dot_err) <= 1e-5, max(dot_err)
    og = O.Geometry(N, B, theta)
    pix = rng.integers(0, N * N, 64)
    ref = og.backproject_pixels(w.cpu().numpy(), pix)
    assert rel_l2(grad.cpu().numpy().ravel()[pix], ref) <= 1e-5
    g.close()


def oracle_x(p, eta, rho, sino):
    o = O.DADMM(dict(p, rho=rho), eta)
    for _ in range(10):
        o.iterate(sino)
    return o.home_view()[0]


def oracle_loss(p, eta, w, rho, sino):
    return float(np.sum(w * oracle_x(p, eta, rho, sino)))


def test_unrolled_admm_gradients_match_oracle_finite_differences():
    need_gpu()
    N, A, B, M = 32, 48, 47, 8
    p = small_problem(N=N, A=A, B=B, M=M, graph="complete", part="interleaved", noise=0.01, seed=9,
                      E1=10, E2=10, rho=1.0, eta2=0.2)
    eta = oracle_eta1(p, iters=60)
    rng = np.random.default_rng(3)
    w = rng.standard_normal((N, N))
    sino = p["sino"][0]
    g = api.Geometry(N, B, p["geometry"]["theta"])
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    sel = [idx[ptr[m]:ptr[m + 1]] for m in range(M)]
    rho = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    d = cuda(sino).requires_grad_(True)
    x = autograd.unrolled_admm(d, g, sel, p["seg_row_ptr"], rho, eta, eta2=0.2, E1=10, E2=10, iters=10)
    loss = torch.sum(x.double() * cuda(w).double())
    loss.backward()
    # forward parity with the oracle (10 unquantized iterations, complete graph)
    assert rel_l2(x.detach().cpu().numpy(), oracle_x(p, eta, 1.0, sino[None])) <= 1e-4
    # d L / d rho (eta1 fixed) by central differences of the FP64 oracle
    h = 1e-3
    fd_rho = (oracle_loss(p, eta, w, 1.0 + h, sino[None]) - oracle_loss(p, eta, w, 1.0 - h, sino[None])) / (2 * h)
    assert abs(rho.grad.item() - fd_rho) <= 1e-3 * abs(fd_rho), (rho.grad.item(), fd_rho)
    # directional derivative along a sinogram direction (the map is linear in d)
    v = rng.standard_normal((A, B)).astype(np.float32)
    fd_d = (oracle_loss(p, eta, w, 1.0, (sino + v)[None]) - oracle_loss(p, eta, w, 1.0, (sino - v)[None])) / 2
    ad_d = float(torch.sum(d.grad.double() * cuda(v).double()))
    assert abs(ad_d - fd_d) <= 1e-3 * abs(fd_d), (ad_d, fd_d)
    g.close()


def test_unrolled_admm_full_size_checkpointed():
    """1024^2, 1440 angles, 8 nodes (interleaved, complete graph), 10 unrolled
    iterations with the oracle's step sizes. Checkpointing (one per iteration)
    changes no gradient and keeps the peak memory well below the
    stored-activation run; the forward loss <w, x_10> and dL/drho (eta1 held
    fixed) match the FP64 oracle's value and central difference stored by
    tests/golden/make_trajectory_goldens.py within 1e-3; the sinogram gradient
    matches central differences of the GPU forward (the map is linear in d,
    so they are exact up to FP32 rounding)"""
    need_gpu()
    import os
    z = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c4_diff_trajectory.npz"))
    prob = synth.make_problem("c4_diff")
    gd = prob["geometry"]
    g = api.Geometry(gd["N"], gd["B"], gd["theta"])
    ptr, idx = prob["node_ang_ptr"], prob["node_ang"]
    sel = [idx[ptr[m]:ptr[m + 1]] for m in range(prob["M"])]
    eta = z["eta1"]
    w_host = np.random.default_rng(int(z["w_seed"])).standard_normal((gd["N"], gd["N"]))
    w = torch.as_tensor(w_host).cuda()  # float64
    sino = cuda(prob["sino"][0])

    def loss_of(rho_val, d, grad=False, checkpoint=True):
        rho = torch.tensor(rho_val, dtype=torch.float64, requires_grad=grad)
        x = autograd.unrolled_admm(d, g, sel, prob["seg_row_ptr"], rho, eta, iters=10, checkpoint=checkpoint)
        return torch.sum(x.double() * w), rho

    grads, peaks, losses = [], [], []
    for ck in (True, False):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        d = sino.clone().requires_grad_(True)
        loss, rho = loss_of(1.0, d, grad=True, checkpoint=ck)
        loss.backward()
        torch.cuda.synchronize()
        peaks.append(torch.cuda.max_memory_allocated() - base)
        grads.append((rho.grad.item(), d.grad.detach().clone()))
        losses.append(loss.item())
        del loss, rho, d
    assert grads[0][0] == grads[1][0] and torch.equal(grads[0][1], grads[1][1])
    assert peaks[0] < 0.25 * peaks[1], peaks
    g_rho, g_d = grads[0]
    # forward and rho-derivative against the FP64 oracle
    assert abs(losses[0] - float(z["loss"])) <= 1e-3 * abs(float(z["loss"])), (losses[0], float(z["loss"]))
    h = float(z["h"])  # rho (1 +- h) with rho = 1
    fd64 = (float(z["loss_plus"]) - float(z["loss_minus"])) / (2.0 * h)
    print("dL/drho: autograd %.9e, FP64 oracle central difference %.9e, rel %.3e"
          % (g_rho, fd64, abs(g_rho - fd64) / abs(fd64)))
    assert abs(g_rho - fd64) <= 1e-3 * abs(fd64), (g_rho, fd64)
    v = torch.randn(sino.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    with torch.no_grad():
        fdd = (loss_of(1.0, sino + v)[0] - loss_of(1.0, sino - v)[0]).item() / 2
    add = float(torch.sum(g_d.double() * v.double()))
    assert abs(add - fdd) <= 1e-3 * abs(fdd), (add, fdd)
    g.close()


def test_unrolled_admm_with_64_nodes_allocates_no_work_lists_after_setup():
    """64 nodes: the unrolled iteration plans its 64 angle selections once
    (one device allocation each) and then runs every projector and
    backprojector call of two further forward and backward passes without
    a device allocation or free of the library's work lists"""
    need_gpu()
    N, A, B, M = 64, 128, 91, 64  # one row of x per node
    p = small_problem(N=N, A=A, B=B, M=M, graph="complete", part="interleaved", noise=0.01, seed=2,
                      E1=2, E2=2)
    g = api.Geometry(N, B, p["geometry"]["theta"])
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    sel = [idx[ptr[m]:ptr[m + 1]] for m in range(M)]
    eta = np.full(M, 1e-3)
    d = cuda(p["sino"][0]).requires_grad_(True)

    def run():
        rho = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
        x = autograd.unrolled_admm(d, g, sel, p["seg_row_ptr"], rho, eta, E1=2, E2=2, iters=2)
        x.sum().backward()
        torch.cuda.synchronize()
        return rho.grad.item()

    g0 = run()
    after_setup = g.cache_stats()
    assert after_setup["allocs"] == M and after_setup["frees"] == 0 and after_setup["entries"] == M
    assert run() == g0 and run() == g0  # deterministic, and no new lists
    assert g.cache_stats() == after_setup
    g.close()
