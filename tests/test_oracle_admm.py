"""Pins of the oracle's dADMM iteration (Algorithms 2-4, Eq. 15-18, 21-24)
against consequences of the mathematics: a single node reduces to
least squares (dense lstsq), exact noise-free data is a fixed point even with
relay delays, exactly solved sub-problems satisfy the optimality
conditions of Eq. 15-16 and zero the owner's dual (Eq. 18), the x-update has a closed form, the relay tables
of a 4-ring are known by hand, the view every node uses carries exactly
the hop delay and quantizer the graph dictates, and the FP64 statistics
(primal gap, change and norm of node 0's view, residual) equal their values
worked out by hand from the state."""
import numpy as np
import pytest

import oracle as O
from problems import oracle_eta1, small_problem


def dense_P(geo, N, sel=None):
    return np.stack([geo.project(e.reshape(N, N), sel).ravel() for e in np.eye(N * N)], axis=1)


def test_relay_tables_ring4_by_hand():
    adj = np.zeros((4, 4), np.int32)
    for m in range(4):
        adj[m, (m + 1) % 4] = adj[(m + 1) % 4, m] = 1
    dist, first = O.relay_tables(adj)
    assert np.array_equal(dist, [[0, 1, 2, 1], [1, 0, 1, 2], [2, 1, 0, 1], [1, 2, 1, 0]])
    # owner 0 reaches node 2 through its lowest-id parent (1), so via edge (0, 1)
    assert first[0, 2] == 1 and first[1, 3] == 0 and first[2, 0] == 1 and first[3, 1] == 0
    assert all(first[s, m] == m for s in range(4) for m in range(4) if dist[s, m] == 1)


def test_single_node_converges_to_min_norm_least_squares():
    """M = 1 and an exact x-step (E2 = 200): lambda vanishes after one
    iteration and the u-update is proximal-point GD on Eq. 5 from zero, whose
    limit is the minimum-norm least-squares solution"""
    N, B, A = 8, 13, 16
    p = small_problem(N=N, A=A, B=B, M=1, E1=10, E2=200, noise=0.05, seed=1)
    st = O.DADMM(p, oracle_eta1(p))
    geo = O.Geometry(N, B, p["geometry"]["theta"])
    P = dense_P(geo, N)
    x_ls = np.linalg.lstsq(P, p["sino"][0].astype(np.float64).ravel(), rcond=None)[0]
    for _ in range(3500):
        st.iterate(p["sino"])
    x = st.home_view()[0].ravel()
    assert np.linalg.norm(x - x_ls) <= 1e-7 * np.linalg.norm(x_ls)
    assert np.abs(st.lam).max() < 1e-12


@pytest.mark.parametrize("graph,M,quant", [("ring", 4, "none"), ("complete", 3, "none"),
                                          ("ring", 4, "kmeans")])
def test_noise_free_truth_is_a_fixed_point(graph, M, quant):
    """d = P x_true, u_m = x = x_true, lambda = 0: every update leaves the state
    unchanged, whatever the relay delays"""
    N, B, A = 8, 13, 16
    p = small_problem(N=N, A=A, B=B, M=M, graph=graph, quant=quant, km_k=64)
    geo = O.Geometry(N, B, p["geometry"]["theta"])
    rng = np.random.default_rng(4)
    # quantized runs: the image takes few values, so K-means reproduces it exactly
    x_true = rng.integers(0, 4, (N, N)).astype(np.float64) if quant != "none" else rng.random((N, N))
    sino = geo.project(x_true)[None].astype(np.float64)
    st = O.DADMM(p, oracle_eta1(p))
    u = np.broadcast_to(x_true, (1, M, N, N))
    hist = np.broadcast_to(x_true, (st.D, 3, 1, N, N))
    st.load_state(u, np.zeros((1, M, N, N)), x_true[None], hist, 7)
    for _ in range(3):
        stats = st.iterate(sino)
    assert np.abs(st.u - x_true).max() < 1e-12
    assert np.abs(st.lam).max() < 1e-12
    assert np.abs(st.xseg - x_true).max() < 1e-12
    assert stats[0, 0] < 1e-24 and stats[0, 1] < 1e-24


def test_exact_subproblem_solutions_satisfy_their_optimality_conditions():
    """With E1 and E2 large the GD loops solve Eq. 15 and 16 exactly:
    P_m^T (P_m u_m - d_m) + rho (u_m - x_m^k) + lambda_m^k = 0 at the new u_m,
    and x[m] = u_m + lambda_m^k / rho on segment m, which makes the dual
    update (Eq. 18) return lambda_m = 0 on the node's own segment."""
    N, B, A, M, rho = 8, 13, 16, 3, 2.0
    p = small_problem(N=N, A=A, B=B, M=M, graph="complete", E1=3000, E2=80, noise=0.05,
                      seed=3, rho=rho, eta2=0.5 / rho)
    st = O.DADMM(p, oracle_eta1(p))
    rng = np.random.default_rng(2)
    lam0 = rng.standard_normal((1, M, N, N))
    hist = np.broadcast_to(rng.random((N, N)), (st.D, 3, 1, N, N))
    st.load_state(rng.random((1, M, N, N)), lam0, rng.random((1, N, N)), hist, 4)
    x_k = hist[0, 0, 0]  # complete graph, unquantized: every view of x^k is this image
    st.iterate(p["sino"])
    geo = O.Geometry(N, B, p["geometry"]["theta"])
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    for m in range(M):
        sel = idx[ptr[m]:ptr[m + 1]]
        um = st.u[0, m]
        grad = (geo.backproject(geo.project(um, sel) - p["sino"][0][sel].astype(np.float64), sel)
                + rho * (um - x_k) + lam0[0, m])
        assert np.abs(grad).max() < 1e-9 * np.abs(lam0).max()
        r0, r1 = p["seg_row_ptr"][m], p["seg_row_ptr"][m + 1]
        assert np.abs(st.xseg[0, r0:r1] - (um + lam0[0, m] / rho)[r0:r1]).max() < 1e-12
        assert np.abs(st.lam[0, m, r0:r1]).max() < 1e-12


def test_x_update_closed_form():
    """E2 GD steps of Algorithm 3 from x0: v + (1 - eta2 rho)^E2 (x0 - v), v = u + lambda/rho"""
    N, M = 8, 2
    p = small_problem(N=N, M=M, E1=0, E2=7, rho=0.7, eta2=0.3)
    st = O.DADMM(p, np.ones(M))
    rng = np.random.default_rng(6)
    u, lam, x0 = rng.random((1, M, N, N)), rng.standard_normal((1, M, N, N)), rng.random((1, N, N))
    st.load_state(u, lam, x0, np.zeros((st.D, 3, 1, N, N)), 0)
    st.iterate(np.zeros((1, p["geometry"]["A"], p["geometry"]["B"]), np.float32))
    f = (1 - 0.3 * 0.7) ** 7
    for m in range(M):
        r0, r1 = p["seg_row_ptr"][m], p["seg_row_ptr"][m + 1]
        v = u[0, m, r0:r1] + lam[0, m, r0:r1] / 0.7
        assert np.allclose(st.xseg[0, r0:r1], v + f * (x0[0, r0:r1] - v), rtol=0, atol=1e-14)


@pytest.mark.parametrize("quant", ["none", "alternate"])
def test_views_follow_hop_delays_and_first_edge_quantizer(quant):
    """E1 = E2 = 0 and u = 0 turn the dual update into lambda_m = -rho x_m^{k+1},
    exposing every node's view: segment s reaches node m after
    max(dist - 1, 0) extra iterations through the plane of its first edge"""
    N, M, rho = 8, 4, 2.0
    p = small_problem(N=N, M=M, graph="ring", quant=quant, E1=0, E2=0, rho=rho)
    st = O.DADMM(p, np.ones(M))
    D, k = st.D, 5
    hist = np.zeros((D, 3, 1, N, N))
    seg = p["seg_row_ptr"]
    for j in range(D):
        for q in range(3):
            for s in range(M):
                hist[j, q, 0, seg[s]:seg[s + 1]] = 1000 * q + 100 * j + s
    xseg = np.zeros((1, N, N))
    for s in range(M):
        xseg[0, seg[s]:seg[s + 1]] = 7.0 + s  # constant segments: every quantizer is exact
    st.load_state(np.zeros((1, M, N, N)), np.zeros((1, M, N, N)), xseg, hist, k)
    st.iterate(np.zeros((1, 16, 13), np.float32))
    dist, first = O.relay_tables(p["adj"])
    for m in range(M):
        view = -st.lam[0, m] / rho
        for s in range(M):
            lag = 0 if s == m else dist[s, m] - 1
            kind = p["home_q"][m] if s == m else p["edge_q"][s, first[s, m]]
            want = 7.0 + s if lag == 0 else 1000 * kind + 100 * ((k + 1 - lag) % D) + s
            assert np.all(view[seg[s]:seg[s + 1]] == want), (m, s)


def test_bytes_follow_the_communication_model():
    """complete graph, no quantization: every owner sends its n/M segment to
    the M - 1 others, M (M-1) n / M values in total (Eq. 20 summed over nodes)"""
    N, M = 8, 4
    p = small_problem(N=N, M=M, graph="complete")
    st = O.DADMM(p, oracle_eta1(p))
    stats = st.iterate(p["sino"])
    assert stats[0, 4] == 4.0 * M * (M - 1) * (N * N // M)


def test_jpeg_bytes_are_the_entropy_coded_messages():
    """complete graph, JPEG messages: each owner's segment reaches the M - 1
    others as its baseline Huffman-coded blocks plus (lo, hi), 8 bytes"""
    N, M, quality = 32, 4, 60
    p = small_problem(N=N, A=24, B=47, M=M, graph="complete", quant="jpeg", jpeg_quality=quality, noise=0.02)
    st = O.DADMM(p, oracle_eta1(p))
    stats = st.iterate(p["sino"])
    seg = p["seg_row_ptr"]
    want = 0.0
    for m in range(M):
        x = st.xseg[0, seg[m]:seg[m + 1]].astype(np.float32)  # the owner's segment after Algorithm 3
        coefs, lohi, _, _ = O.jpeg(x, quality)
        eb = len(O.jpeg_entropy(coefs)) if lohi[1] > lohi[0] else 0
        want += (M - 1) * (eb + 8)
    assert stats[0, 4] == want


# ---------------------------------------------------------------------------
# the FP64 statistics of an iteration: [gap2, chg2, nrm2, resid2, bytes]
# (Sec. 3.2's stopping quantity and the residual, read as in the oracle's
# header), pinned against values that follow from the state by hand
# ---------------------------------------------------------------------------

def ring4_dist(s, m):
    d = abs(s - m)
    return min(d, 4 - d)


def test_residual_statistic_from_zero_is_the_data_norm():
    """From u = 0 with E1 = 1 the only inner step's residual is -d_m, so the
    statistic is sum_m ||d_m||^2 = ||d||^2 (the subsets partition the angles)"""
    p = small_problem(N=8, A=16, B=13, M=3, graph="complete", E1=1, noise=0.05, seed=5)
    st = O.DADMM(p, oracle_eta1(p))
    stats = st.iterate(p["sino"])
    d = p["sino"][0].astype(np.float64)
    assert abs(stats[0, 3] - np.sum(d * d)) <= 1e-13 * np.sum(d * d)


def test_residual_statistic_is_taken_at_the_last_inner_step():
    """E1 = 2 from zero: the first step gives u_m = eta1_m P_m^T d_m (x = lambda = 0),
    and the statistic is the second step's residual
    sum_m ||eta1_m P_m P_m^T d_m - d_m||^2, evaluated here with dense matrices"""
    N, B, A, M = 8, 13, 16, 2
    p = small_problem(N=N, A=A, B=B, M=M, graph="complete", E1=2, noise=0.05, seed=8)
    eta = oracle_eta1(p)
    st = O.DADMM(p, eta)
    stats = st.iterate(p["sino"])
    geo = O.Geometry(N, B, p["geometry"]["theta"])
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    want = 0.0
    for m in range(M):
        sel = idx[ptr[m]:ptr[m + 1]]
        P = dense_P(geo, N, sel)
        dm = p["sino"][0][sel].astype(np.float64).ravel()
        r = eta[m] * (P @ (P.T @ dm)) - dm
        want += float(r @ r)
    assert abs(stats[0, 3] - want) <= 1e-12 * want


@pytest.mark.parametrize("quant", ["none", "alternate"])
def test_change_norm_and_gap_statistics_follow_the_views(quant):
    """Ring of 4, E1 = 0, u = lambda = 0: the x-update gives x[m] = f X on
    every segment (f = (1 - eta2 rho)^E2, Algorithm 3 with v = 0), so every
    view is known by hand from the relay delays of the 4-ring (segment s
    reaches node m max(dist - 1, 0) iterations late). Then
      chg2 = ||x_0^{k+1} - x_0^k||^2 and nrm2 = ||x_0^k||^2 (node 0's views),
      gap2 = sum_m ||u_m - x_m^{k+1}||^2 = sum_m ||x_m^{k+1}||^2,
      resid2 = 0 (no inner step).
    Every stored version of every segment is a distinct constant, so a view
    read at the wrong iteration or from the wrong plane changes chg2 or nrm2.
    Constant segments pass every quantizer exactly (as their FP32 value)."""
    N, M, rho, eta2, E2, k = 8, 4, 0.7, 0.3, 3, 5
    p = small_problem(N=N, M=M, graph="ring", quant=quant, E1=0, E2=E2, rho=rho, eta2=eta2)
    st = O.DADMM(p, np.ones(M))
    D = st.D
    seg = p["seg_row_ptr"]
    hist = np.zeros((D, 3, 1, N, N))
    X = np.zeros((1, N, N))
    for s in range(M):
        X[0, seg[s]:seg[s + 1]] = 3.0 + s
        for j in range(D):
            for q in range(3):
                hist[j, q, 0, seg[s]:seg[s + 1]] = 1.0 + 0.5 * q + 0.25 * j + 0.01 * s
    st.load_state(np.zeros((1, M, N, N)), np.zeros((1, M, N, N)), X, hist, k)
    stats = st.iterate(np.zeros((1, 16, 13), np.float32))
    f = (1.0 - eta2 * rho) ** E2
    adj = p["adj"]

    def kind(s, m):
        if s == m:
            return p["home_q"][m]
        # first edge of the lowest-id-parent shortest path on the 4-ring: the
        # neighbour of s towards m (for the opposite node, the lower-id neighbour)
        nbrs = [t for t in range(M) if adj[s, t]]
        first = min(t for t in nbrs if ring4_dist(t, m) == ring4_dist(s, m) - 1)
        return p["edge_q"][s, first]

    def view(m, it):
        out = np.zeros((N, N))
        for s in range(M):
            lag = 0 if s == m else ring4_dist(s, m) - 1
            ver = it - lag
            if ver == k + 1:  # the fresh message; the quantizers code the FP32 segment
                v = f * (3.0 + s)
                out[seg[s]:seg[s + 1]] = v if kind(s, m) == 0 else float(np.float32(v))
            else:
                out[seg[s]:seg[s + 1]] = hist[ver % D, kind(s, m), 0, seg[s]:seg[s + 1]]
        return out

    v1, v0 = view(0, k + 1), view(0, k)
    assert np.isclose(stats[0, 1], np.sum((v1 - v0) ** 2), rtol=1e-13, atol=0)
    assert np.isclose(stats[0, 2], np.sum(v0 ** 2), rtol=1e-13, atol=0)
    gap = sum(np.sum(view(m, k + 1) ** 2) for m in range(M))
    assert np.isclose(stats[0, 0], gap, rtol=1e-13, atol=0)
    assert stats[0, 3] == 0.0


def test_change_statistic_over_the_first_two_iterations():
    """Complete graph, no quantizer: node 0's view is the owners'
    reconstruction. After iteration 1 from zero nrm2 = 0 and
    chg2 = ||x^1||^2; after iteration 2 nrm2 = ||x^1||^2 and
    chg2 = ||x^2 - x^1||^2"""
    p = small_problem(N=16, A=24, B=23, M=4, graph="complete", noise=0.02, seed=11)
    st = O.DADMM(p, oracle_eta1(p))
    s1 = st.iterate(p["sino"])
    x1 = st.home_view()
    s2 = st.iterate(p["sino"])
    x2 = st.home_view()
    assert s1[0, 2] == 0.0
    assert np.isclose(s1[0, 1], np.sum(x1 * x1), rtol=1e-13, atol=0)
    assert np.isclose(s2[0, 2], np.sum(x1 * x1), rtol=1e-13, atol=0)
    assert np.isclose(s2[0, 1], np.sum((x2 - x1) ** 2), rtol=1e-12, atol=0)


def test_single_node_algorithm2_solves_its_subproblem_and_matches_the_iteration():
    """orc_alg2_node (Algorithm 2 for one node, used to check single nodes of
    problems too large for the whole oracle iteration): with many steps it
    solves Eq. 15, P_m^T (P_m u - d_m) + rho (u - x_m) + lambda_m = 0; with
    E1 = 4 it reproduces node m's u of the full iteration bit for bit"""
    N, B, A, M, rho = 8, 13, 16, 3, 1.5
    p = small_problem(N=N, A=A, B=B, M=M, graph="complete", E1=4, noise=0.05, seed=7, rho=rho)
    eta = oracle_eta1(p)
    geo = O.Geometry(N, B, p["geometry"]["theta"])
    ptr, idx = p["node_ang_ptr"], p["node_ang"]
    rng = np.random.default_rng(12)
    u0, lam0 = rng.random((1, M, N, N)), rng.standard_normal((1, M, N, N))
    xk = rng.random((N, N))
    st = O.DADMM(p, eta)
    st.load_state(u0, lam0, rng.random((1, N, N)), np.broadcast_to(xk, (st.D, 3, 1, N, N)), 3)
    st.iterate(p["sino"])
    d = p["sino"][0].astype(np.float64)
    for m in range(M):
        sel = idx[ptr[m]:ptr[m + 1]]
        um, _ = geo.alg2_node(u0[0, m], xk, lam0[0, m], d, sel, rho, eta[m], 4)
        assert np.array_equal(um, st.u[0, m])
        us, _ = geo.alg2_node(u0[0, m], xk, lam0[0, m], d, sel, rho, eta[m], 3000)
        grad = geo.backproject(geo.project(us, sel) - d[sel], sel) + rho * (us - xk) + lam0[0, m]
        assert np.abs(grad).max() < 1e-9 * np.abs(lam0).max()


def test_supplied_messages_replace_the_quantizers_output():
    """orc_dadmm_iterate with msg_in: (a) supplying the messages the oracle's
    own quantizers produced leaves every state bit-identical; (b) supplied
    planes are what every node's view reads (E1 = E2 = 0, u = 0, so the dual
    update exposes the views: lambda_m = -rho x_m^{k+1}), through the plane of
    the path's first edge, for the segments that arrive fresh"""
    N, M, rho = 16, 4, 2.0
    p = small_problem(N=N, A=24, B=23, M=M, graph="ring", quant="alternate", noise=0.02, seed=4, km_k=8)
    eta = oracle_eta1(p, iters=30)
    a, b = O.DADMM(p, eta), O.DADMM(p, eta)
    for _ in range(4):
        a.iterate(p["sino"])
        slot = a.k % a.D
        b.iterate(p["sino"], msgs=a.hist[slot])
        for name in ("u", "lam", "xseg", "hist"):
            assert np.array_equal(getattr(a, name), getattr(b, name)), name
    q = small_problem(N=N, A=24, B=23, M=M, graph="ring", quant="alternate", E1=0, E2=0, rho=rho)
    c = O.DADMM(q, np.ones(M))
    k = 3
    c.load_state(np.zeros((1, M, N, N)), np.zeros((1, M, N, N)), np.ones((1, N, N)),
                 np.zeros((c.D, 3, 1, N, N)), k)
    msgs = np.zeros((3, 1, N, N))
    msgs[1], msgs[2] = 11.0, 22.0  # K-means and JPEG planes
    c.iterate(np.zeros((1, 24, 23), np.float32), msgs=msgs)
    dist, first = O.relay_tables(q["adj"])
    seg = q["seg_row_ptr"]
    for m in range(M):
        view = -c.lam[0, m] / rho
        for s in range(M):
            if s != m and dist[s, m] > 1:
                continue  # relayed: an older version from the ring (zero here)
            kind = q["home_q"][m] if s == m else q["edge_q"][s, first[s, m]]
            assert np.all(view[seg[s]:seg[s + 1]] == (1.0, 11.0, 22.0)[kind]), (m, s)


def test_ctr_first_step_and_limit():
    """Algorithm 1 (CTR, Eq. 5): one step from zero is eta P^T d (dense
    matrices); with eta < 2 / ||P||^2 the iteration from zero converges to the
    minimum-norm least-squares solution (dense lstsq)"""
    N, B, A = 8, 13, 16
    p = small_problem(N=N, A=A, B=B, M=1, noise=0.05, seed=3)
    geo = O.Geometry(N, B, p["geometry"]["theta"])
    P = dense_P(geo, N)
    d = p["sino"][0].astype(np.float64)
    L = np.linalg.norm(P, 2) ** 2
    eta = 1.0 / L
    u1 = geo.ctr(d, eta, 1)
    assert np.allclose(u1.ravel(), eta * (P.T @ d.ravel()), rtol=0, atol=1e-13 * np.abs(u1).max())
    x_ls = np.linalg.lstsq(P, d.ravel(), rcond=None)[0]
    u = geo.ctr(d, eta, 60000)  # condition number ~47: (1 - 1/47^2)^60000 ~ 1e-12
    assert np.linalg.norm(u.ravel() - x_ls) <= 1e-8 * np.linalg.norm(x_ls)
