"""Pins of the oracle's neighbour-averaged consensus variant (the
decentralized analogue of the standard ADMM x-update, Eq. 9): on a complete
graph without quantization one iteration is Eq. 8-10 written out and the
iteration converges to the centralized least-squares solution (its fixed
point: u_m = x, sum of duals zero, sum of node gradients zero); the
noise-free truth is a fixed point on a ring with quantized messages; bytes
count every message sent to a neighbour."""
import numpy as np
import pytest

import oracle as O
from problems import oracle_eta1, small_problem


def dense(geo, N):
    """P as a dense matrix, column by column from the oracle's projector"""
    cols = []
    for i in range(N * N):
        e = np.zeros(N * N)
        e[i] = 1.0
        cols.append(geo.project(e.reshape(N, N)).ravel())
    return np.stack(cols, axis=1)


def test_complete_graph_iteration_is_the_standard_admm_x_update():
    N, M = 8, 3
    p = small_problem(N=N, M=M, graph="complete", quant="none", E1=3, rho=0.8)
    st = O.Consensus(p, oracle_eta1(p))
    rng = np.random.default_rng(1)
    u0, lam0, x0 = rng.random((1, M, N, N)), rng.standard_normal((1, M, N, N)), rng.random((1, M, N, N))
    st.load_state(u0, lam0, x0, 4)
    st.iterate(p["sino"])
    v = st.u + lam0 / 0.8  # u^{k+1} + lambda^k / rho
    want = v.mean(axis=1)  # Eq. 9
    for m in range(M):
        assert np.allclose(st.x[0, m], want[0], rtol=0, atol=1e-13)
        assert np.allclose(st.lam[0, m], lam0[0, m] + 0.8 * (st.u[0, m] - want[0]), rtol=0, atol=1e-12)


def test_complete_graph_converges_to_centralized_least_squares():
    N, B, A, M = 8, 13, 16, 3
    p = small_problem(N=N, A=A, B=B, M=M, graph="complete", quant="none", E1=20, noise=0.05, seed=2)
    geo = O.Geometry(N, B, p["geometry"]["theta"])
    P = dense(geo, N)
    x_ls = np.linalg.lstsq(P, p["sino"][0].astype(np.float64).ravel(), rcond=None)[0]
    st = O.Consensus(p, oracle_eta1(p))
    for _ in range(3000):  # linear convergence: ~1e-3 after 1000 iterations, ~1e-13 after 4000
        st.iterate(p["sino"])
    for m in range(M):
        assert np.linalg.norm(st.x[0, m].ravel() - x_ls) <= 1e-8 * np.linalg.norm(x_ls)
    assert np.abs(st.lam[0].sum(axis=0)).max() < 1e-8  # the duals cancel at the fixed point


@pytest.mark.parametrize("quant", ["none", "kmeans"])
def test_noise_free_truth_is_a_fixed_point_on_a_ring(quant):
    N, B, A, M = 8, 13, 16, 4
    p = small_problem(N=N, A=A, B=B, M=M, graph="ring", quant=quant, km_k=64)
    geo = O.Geometry(N, B, p["geometry"]["theta"])
    rng = np.random.default_rng(4)
    x_true = rng.integers(0, 4, (N, N)).astype(np.float64)  # few values: K-means and JPEG are exact
    sino = geo.project(x_true)[None]
    st = O.Consensus(p, oracle_eta1(p))
    st.load_state(np.broadcast_to(x_true, (1, M, N, N)), np.zeros((1, M, N, N)),
                  np.broadcast_to(x_true, (1, M, N, N)), 3)
    for _ in range(3):
        stats = st.iterate(sino)
    assert np.abs(st.u - x_true).max() < 1e-12
    assert np.abs(st.x - x_true).max() < 1e-12
    assert np.abs(st.lam).max() < 1e-12
    assert stats[0, 0] < 1e-24


def test_bytes_count_every_message_to_a_neighbour():
    N, M = 8, 4
    p = small_problem(N=N, M=M, graph="ring", quant="none")
    st = O.Consensus(p, oracle_eta1(p))
    stats = st.iterate(p["sino"])
    assert stats[0, 4] == 4.0 * N * N * 2 * M  # a ring has 2M directed edges


def test_bytes_of_quantized_messages():
    """alternating K-means / JPEG edges on a ring: every directed edge carries
    its owner's full-image message in the edge's quantizer"""
    N, M, k = 16, 4, 8
    p = small_problem(N=N, A=16, B=23, M=M, graph="ring", quant="alternate", km_k=k, jpeg_quality=50, noise=0.02)
    st = O.Consensus(p, oracle_eta1(p))
    stats = st.iterate(p["sino"])  # lambda^0 = 0: the messages are Q(u^1)
    want = 0.0
    for j in range(M):
        coefs, lohi, _, _ = O.jpeg(st.u[0, j].astype(np.float32), 50)
        jb = (len(O.jpeg_entropy(coefs)) if lohi[1] > lohi[0] else 0) + 8
        kb = 3 * N * N / 8 + 4 * k  # ceil(log2 8) = 3 bits per value + the centres
        for m in range(M):
            if m != j and p["adj"][j, m]:
                want += kb if p["edge_q"][j, m] == 1 else jb
    assert stats[0, 4] == want
