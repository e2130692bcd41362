"""The seeded input generators: shapes, partitions, graphs, determinism."""
import numpy as np
import pytest

from paper_2410_06106_gb300 import synth


def test_uneven_counts_respect_bounds_and_sum():
    for seed in range(5):
        c = synth.uneven_counts(1800, 64, 8, 60, np.random.default_rng(seed))
        assert c.sum() == 1800 and c.min() >= 8 and c.max() <= 60
        c = synth.uneven_counts(720, 16, 10, 80, np.random.default_rng(seed))
        assert c.sum() == 720 and c.min() >= 10 and c.max() <= 80


def test_interleaved_partition_matches_the_papers_ten_node_split():
    parts = synth.partition_interleaved(804, 10)
    assert [len(p) for p in parts] == [81] * 4 + [80] * 6
    assert list(parts[0][:3]) == [0, 10, 20] and parts[0][-1] == 800 and parts[1][-1] == 801


@pytest.mark.parametrize("M,deg", [(16, 4), (64, 6)])
def test_random_geometric_graph_degree_and_connectivity(M, deg):
    adj = synth.random_geometric_graph(M, deg, 99)
    assert np.array_equal(adj, adj.T) and not adj.diagonal().any()
    assert adj.sum() == M * deg and synth.connected(adj)


def test_alternating_edge_kinds_cover_each_edge_once():
    adj = synth.random_geometric_graph(64, 6, 5)
    q = synth.alternating_edge_kinds(adj)
    assert np.array_equal(q >= 0, adj > 0) and np.array_equal(q, q.T)
    kinds = q[np.triu_indices(64, 1)]
    kinds = kinds[kinds >= 0]
    assert abs(int((kinds == 1).sum()) - int((kinds == 2).sum())) <= 1


def test_problem_is_deterministic_and_shaped():
    a = synth.make_problem("c1_tiny")
    b = synth.make_problem("c1_tiny")
    assert np.array_equal(a["sino"], b["sino"]) and a["sino"].shape == (1, 90, 91)
    assert a["sino"].dtype == np.float32
    assert list(np.diff(a["node_ang_ptr"])) == [23, 23, 22, 22]
    assert list(a["seg_row_ptr"]) == [0, 16, 32, 48, 64]
    c3 = synth.make_problem("c3_batch_jpeg")
    cnt = np.diff(c3["node_ang_ptr"])
    assert cnt.sum() == 720 and cnt.min() >= 10 and cnt.max() <= 80
    assert np.all(c3["edge_q"][c3["adj"] > 0] == synth.KIND_JPEG)


def test_noise_level_is_one_percent_of_the_peak():
    rng = np.random.default_rng(0)
    d = np.full((200, 300), 10.0)
    noisy = synth.add_noise(d, 0.01, rng)
    assert abs(np.std(noisy - d) - 0.1) < 0.005
