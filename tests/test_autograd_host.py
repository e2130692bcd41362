"""Host logic of the differentiable unrolled dADMM, on CPU in float64: the
library kernels it calls (projector, backprojector, linear combination, dot)
are replaced by the oracle's dense FP64 operator and plain torch sums, so
that the coefficient algebra of Algorithms 2-3 and Eq. 18 and the backward
formulas can be checked without a GPU: the forward against the oracle's own
iteration, the gradients by torch.autograd.gradcheck."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2410_06106_gb300 import api, autograd
from problems import oracle_eta1, small_problem


class DenseGeom:
    """oracle-backed stand-in with the Geometry methods autograd calls"""

    def __init__(self, og):
        self.og, self.N = og, og.N

    def project(self, img, sel=None, subtract=None):
        y = torch.from_numpy(self.og.project(img.detach().numpy(), sel))
        return y if subtract is None else y - subtract.detach()

    def backproject(self, sino, sel=None):
        return torch.from_numpy(self.og.backproject(sino.detach().numpy(), sel))

    def plan(self, sel=None, batch=1):
        self.planned = getattr(self, "planned", 0) + 1


@pytest.fixture
def cpu_kernels(monkeypatch):
    monkeypatch.setattr(api, "lincomb", lambda xs, coefs, out=None: sum(float(c) * x for c, x in zip(coefs, xs)))
    monkeypatch.setattr(api, "dot", lambda x, y: torch.sum(x.double() * y.double()))


def setup(E1, E2, M=4):
    p = small_problem(N=8, A=16, B=13, M=M, graph="complete", part="interleaved", noise=0.02, seed=5,
                      E1=E1, E2=E2, rho=0.7, eta2=0.3)
    g = p["geometry"]
    geo = DenseGeom(O.Geometry(g["N"], g["B"], g["theta"]))
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    sel = [idx[ptr[m]:ptr[m + 1]] for m in range(M)]
    return p, geo, sel, oracle_eta1(p, iters=60)


def test_forward_equals_oracle_iteration(cpu_kernels):
    p, geo, sel, eta = setup(10, 10)
    d = torch.from_numpy(p["sino"][0].astype(np.float64))
    x = autograd.unrolled_admm(d, geo, sel, p["seg_row_ptr"], 0.7, eta, eta2=0.3, E1=10, E2=10, iters=7)
    o = O.DADMM(p, eta)
    for _ in range(7):
        o.iterate(p["sino"])
    ref = o.home_view()[0]
    assert np.max(np.abs(x.numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_gradients_by_gradcheck(cpu_kernels):
    p, geo, sel, eta = setup(3, 4)
    d = torch.from_numpy(p["sino"][0].astype(np.float64)).requires_grad_(True)
    rho = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)

    def f(rho_, d_):
        return autograd.unrolled_admm(d_, geo, sel, p["seg_row_ptr"], rho_, eta, eta2=0.3, E1=3, E2=4, iters=3)

    assert torch.autograd.gradcheck(f, (rho, d), eps=1e-6, atol=1e-8, rtol=1e-6, fast_mode=True)


def test_checkpointing_changes_no_gradient(cpu_kernels):
    p, geo, sel, eta = setup(3, 4)
    w = torch.from_numpy(np.random.default_rng(1).standard_normal((8, 8)))
    grads = []
    for ck in (True, False):
        d = torch.from_numpy(p["sino"][0].astype(np.float64)).requires_grad_(True)
        rho = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
        x = autograd.unrolled_admm(d, geo, sel, p["seg_row_ptr"], rho, eta, eta2=0.3, E1=3, E2=4, iters=4,
                                   checkpoint=ck)
        torch.sum(x * w).backward()
        grads.append((rho.grad.item(), d.grad.clone()))
    assert grads[0][0] == pytest.approx(grads[1][0], rel=1e-13)
    assert torch.allclose(grads[0][1], grads[1][1], rtol=1e-12, atol=1e-15)
