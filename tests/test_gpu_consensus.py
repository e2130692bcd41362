"""GPU parity of the neighbour-averaged consensus variant (every node keeps
its own x_m = mean over its closed neighbourhood of Q(u_j + lambda_j / rho),
the decentralized analogue of Eq. 9) against the oracle's own
implementation: one iteration replayed from the GPU's state (u, x, lambda;
quantized messages agree except at rounding ties), a free-running
unquantized trajectory, the byte statistic, and the batched and plain forms
bit for bit."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import need_gpu, rel_l2
from paper_2410_06106_gb300 import api
from problems import oracle_eta1, small_problem

pytestmark = pytest.mark.gpu


def cons_problem(quant, graph, M, seed=0, N=32):
    p = small_problem(N=N, A=48, B=int(np.ceil(N * np.sqrt(2))) + 2, M=M, graph=graph, quant=quant,
                      noise=0.02, seed=seed, km_k=16, jpeg_quality=60)
    return dict(p, variant="consensus")


def state(s):
    return s.u.cpu().numpy(), s.lam.cpu().numpy(), s.xseg.cpu().numpy(), s.k


def close_except_ties(a, b, tol=1e-5, frac=2e-3):
    """quantized messages enter x and lambda; a message level at a rounding
    tie moves one pixel of the neighbours' x by a level / |N[m]|"""
    bad = np.abs(a - b) > 1e-4 * (np.abs(b).max() + 1e-30)
    assert bad.mean() <= frac, bad.mean()
    assert rel_l2(a[~bad], b[~bad]) <= tol


@pytest.mark.parametrize("quant,graph,M", [("none", "ring", 4), ("none", "complete", 3), ("kmeans", "ring", 4),
                                          ("jpeg", "complete", 4), ("alternate", "ring", 6)])
def test_one_iteration_replayed_by_the_oracle(quant, graph, M):
    need_gpu()
    p = cons_problem(quant, graph, M, seed=M)
    eta = oracle_eta1(p)
    s = api.DADMM(p, eta)
    sino = torch.as_tensor(p["sino"]).cuda()
    s.step(sino, 3)
    u, lam, x, k = state(s)
    st = s.step(sino, 1)
    o = O.Consensus(p, eta)
    o.load_state(u, lam, x, k)
    ost = o.iterate(p["sino"])
    u1, lam1, x1, k1 = state(s)
    assert k1 == o.k
    assert rel_l2(u1, o.u) <= 1e-5  # Algorithm 2 reads x^k: no quantizer involved yet
    if quant == "none":
        assert rel_l2(x1, o.x) <= 1e-5 and rel_l2(lam1, o.lam) <= 1e-5
        assert st[0, 0, 4] == ost[0, 4]
    else:
        close_except_ties(x1, o.x)
        close_except_ties(lam1, o.lam, tol=1e-4)
        assert abs(st[0, 0, 4] - ost[0, 4]) <= 1e-3 * ost[0, 4]
    assert rel_l2(st[0, 0, :4], ost[0, :4]) <= 1e-3  # gap, change, norm, residual


def test_unquantized_trajectory_follows_the_oracle():
    need_gpu()
    p = cons_problem("none", "ring", 5, seed=3)
    eta = oracle_eta1(p)
    s = api.DADMM(p, eta)
    s.step(torch.as_tensor(p["sino"]).cuda(), 20)
    o = O.Consensus(p, eta)
    for _ in range(20):
        o.iterate(p["sino"])
    assert rel_l2(s.u.cpu().numpy(), o.u) <= 1e-4
    assert rel_l2(s.xseg.cpu().numpy(), o.x) <= 1e-4
    # the reconstruction is the mean of the nodes' x
    assert rel_l2(s.home_view().cpu().numpy(), o.x.mean(axis=1)) <= 1e-4


@pytest.mark.parametrize("quant", ["none", "alternate"])
def test_batched_and_plain_forms_are_bit_identical(quant):
    need_gpu()
    p = cons_problem(quant, "ring", 4, seed=9)
    eta = oracle_eta1(p)
    sino = torch.as_tensor(p["sino"]).cuda()
    a, b = api.DADMM(p, eta, mode="batched"), api.DADMM(p, eta, mode="plain")
    sa, sb = a.step(sino, 4), b.step(sino, 4)
    for name in ("u", "lam", "xseg", "hist"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
    assert np.array_equal(sa, sb)
