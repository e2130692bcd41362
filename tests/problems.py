"""Small hand-built problems shared by the oracle pins and the GPU parity
tests. Inputs only: geometry, partitions, graphs and data come from the
seeded generators in paper_2410_06106_gb300.synth or from the oracle."""
import numpy as np

from paper_2410_06106_gb300 import synth


def small_problem(N=8, A=16, B=13, M=1, S=1, graph="complete", part="interleaved",
                  quant="none", seed=0, noise=0.0, E1=10, E2=10, rho=1.0, eta2=0.2,
                  km_k=4, km_iters=10, jpeg_quality=50, theta_offset=0.0, ellipses=3):
    theta = synth.angles(A) + theta_offset
    rng = np.random.default_rng(seed)
    if part == "interleaved":
        parts = synth.partition_interleaved(A, M)
    else:
        parts = synth.partition_even_blocks(A, M)
    ptr, idx = synth.csr(parts)
    adj = {"complete": synth.complete, "ring": synth.ring}[graph](M) if M > 1 else np.zeros((1, 1), np.int32)
    kinds = {"none": 0, "kmeans": 1, "jpeg": 2}
    if quant == "alternate":
        edge_q = synth.alternating_edge_kinds(adj)
        home_q = np.where(np.arange(M) % 2 == 0, 1, 2).astype(np.int32)
    else:
        edge_q = synth.uniform_edge_kinds(adj, kinds[quant])
        home_q = np.full(M, kinds[quant], np.int32)
    sino = np.empty((S, A, B), np.float32)
    ells = []
    for sl in range(S):
        ell = synth.random_ellipses(N, ellipses, rng)
        d = synth.ellipse_sinogram(ell, theta, B)
        sino[sl] = synth.add_noise(d, noise, rng).astype(np.float32)
        ells.append(ell)
    return dict(name="small", geometry=dict(N=N, A=A, B=B, theta=theta), M=M, S=S,
                node_ang_ptr=ptr, node_ang=idx, seg_row_ptr=synth.even_segments(N, M),
                adj=adj, edge_q=edge_q, home_q=home_q, km_k=km_k, jpeg_quality=jpeg_quality,
                seed=1234 + seed, iters=10, sino=sino, ellipses=ells, rho=rho, eta2=eta2,
                E1=E1, E2=E2, km_iters=km_iters)


def oracle_eta1(prob, iters=100):
    """eta1_m = 1 / (||P_m||^2 + rho) with the oracle's power iteration"""
    import oracle as O
    g = prob["geometry"]
    geo = O.Geometry(g["N"], g["B"], g["theta"])
    ptr, idx = prob["node_ang_ptr"], prob["node_ang"]
    L = np.array([geo.opnorm_sq(idx[ptr[m]:ptr[m + 1]], iters=iters) for m in range(prob["M"])])
    return 1.0 / (L + prob["rho"])
