"""Lost messages on the GPU (dadmm_step_lossy) against the oracle: no losses
equal the lossless step bit for bit; random losses follow the oracle's
held-version rule over whole trajectories, mixed with lossless steps; a mask
that outlives the message ring is refused before anything runs."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import need_gpu, rel_l2
from paper_2410_06106_gb300 import api
from problems import oracle_eta1, small_problem
from test_gpu_dadmm import compare_states, gpu_state

pytestmark = pytest.mark.gpu


def masks(rng, n, M, p, max_run):
    """random losses, no pair lost more than max_run exchanges in a row"""
    d = (rng.random((n, M, M)) < p).astype(np.uint8)
    run = np.zeros((M, M), int)
    for i in range(n):
        run = np.where(d[i] > 0, run + 1, 0)
        d[i][run > max_run] = 0
        run[run > max_run] = 0
    return d


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_no_losses_equal_the_lossless_step(mode):
    need_gpu()
    p = dict(small_problem(N=40, A=40, B=59, M=5, graph="ring", quant="alternate", noise=0.02, seed=2),
             max_stale=2)
    eta = oracle_eta1(p)
    sino = torch.as_tensor(p["sino"]).cuda()
    a, b = api.DADMM(p, eta, mode=mode), api.DADMM(p, eta, mode=mode)
    sa = a.step(sino, 5)
    sb = b.step(sino, 5, drop=np.zeros((5, 5, 5), np.uint8))
    for name in ("u", "lam", "xseg", "hist", "iter"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
    assert np.array_equal(sa, sb)


@pytest.mark.parametrize("graph,M", [("ring", 6), ("complete", 4)])
def test_random_losses_follow_the_oracle(graph, M):
    """every iteration replayed by the oracle from the GPU's state (state
    injection, with the oracle's own held versions, which depend only on the
    masks): one-iteration parity at the protocol's 1e-5 through 12 lossy and
    lossless iterations; the free-running trajectories agree to 1e-3"""
    need_gpu()
    p = dict(small_problem(N=32, A=48, B=47, M=M, graph=graph, quant="none", noise=0.02, seed=5), max_stale=3)
    eta = oracle_eta1(p)
    d = masks(np.random.default_rng(M), 12, M, 0.35, 3)
    s = api.DADMM(p, eta)
    sino = torch.as_tensor(p["sino"]).cuda()
    inj = O.DADMM(p, eta)   # replays each GPU iteration
    free = O.DADMM(p, eta)  # runs on its own
    for i in range(12):
        lossy = not (5 <= i < 7)
        before = gpu_state(s)
        s.step(sino, 1, drop=d[i:i + 1] if lossy else None)
        inj.load_state(*before)
        inj.iterate(p["sino"], drop=d[i] if lossy else None)
        try:
            compare_states(gpu_state(s), inj, p)
        except AssertionError as e:
            raise AssertionError("iteration %d (%s): %s" % (i, "lossy" if lossy else "lossless", e)) from None
        free.iterate(p["sino"], drop=d[i] if lossy else None)
    assert rel_l2(s.u.cpu().numpy(), free.u) <= 1e-3


def test_quantized_messages_with_losses():
    need_gpu()
    M = 6
    p = dict(small_problem(N=48, A=48, B=71, M=M, graph="ring", quant="alternate", noise=0.02, seed=7,
                           km_k=16, jpeg_quality=60), max_stale=2)
    eta = oracle_eta1(p)
    d = masks(np.random.default_rng(1), 6, M, 0.3, 2)
    s = api.DADMM(p, eta)
    s.step(torch.as_tensor(p["sino"]).cuda(), 6, drop=d)
    o = O.DADMM(p, eta)
    for i in range(6):
        o.iterate(p["sino"], drop=d[i])
    assert rel_l2(s.u.cpu().numpy(), o.u) <= 1e-3  # quantized messages may differ at rounding ties


def test_a_mask_outliving_the_ring_is_refused():
    need_gpu()
    M = 4
    p = dict(small_problem(N=16, A=16, B=23, M=M, graph="ring"), max_stale=1)
    s = api.DADMM(p, oracle_eta1(p))
    sino = torch.as_tensor(p["sino"]).cuda()
    s.step(sino, 4)
    d = np.zeros((4, M, M), np.uint8)
    d[:, 2, 0] = 1  # node 0 loses segment 2 four times in a row
    before = s.u.clone()
    with pytest.raises(api.TomoError) as e:
        s.step(sino, 4, drop=d)
    assert e.value.code == -1 and s.k == 4 and torch.equal(s.u, before)
    s.step(sino, 1, drop=d[:1])  # one lost exchange fits
    assert s.k == 5
    p0 = dict(p, max_stale=0)
    with pytest.raises(api.TomoError):
        api.DADMM(p0, oracle_eta1(p0)).step(sino, 1, drop=d[:1])
