"""Pins of the oracle's message quantizers (Sec. 2.7): K-means (Algorithm 5)
against Lloyd's monotonicity, exact 1-D optimal clustering by dynamic
programming and lossless cases; the JPEG-style codec against the published
quantization table, scipy's orthonormal DCT-II, and exact closed forms."""
import itertools
import os

import numpy as np
import pytest
import scipy.fft

import oracle as O


def read_table(path):
    rows = [l for l in open(path) if l.strip() and not l.startswith("#")]
    return np.array([[int(x) for x in r.split()] for r in rows])


# ----------------------------- K-means ---------------------------------

def test_splitmix64_published_first_output(golden_dir):
    want = int([l for l in open(os.path.join(golden_dir, "splitmix64_seed0.txt"))
                if not l.startswith("#")][0], 16)
    assert O.mix64(0x9E3779B97F4A7C15) == want


@pytest.mark.parametrize("k,seed", [(2, 0), (4, 1), (16, 2), (32, 3)])
def test_kmeans_objective_never_increases(k, seed):
    rng = np.random.default_rng(seed)
    v = np.concatenate([rng.normal(m, 0.3, 500) for m in rng.uniform(-5, 5, 7)]).astype(np.float32)
    codes, cent, deq, obj = O.kmeans(v, k, 10, O.kmeans_key(7, 0, seed, 1))
    # exact arithmetic gives obj[t+1] <= obj[t]; the slack covers FP32 rounding
    # of centres and FP32 distance decisions
    assert np.all(np.diff(obj) <= 1e-9 * obj[:-1] + 1e-12)
    assert np.array_equal(deq, cent[codes])
    e = v.astype(np.float64) - deq
    assert abs(obj[-1] - e @ e) <= 1e-12 * obj[-1]
    # every value sits at its nearest centre
    d = np.abs(v[:, None] - cent[None, :])
    assert np.all(d[np.arange(v.size), codes] <= d.min(axis=1))


def test_kmeans_initial_centres_are_distinct_sorted_values():
    rng = np.random.default_rng(4)
    v = rng.integers(0, 50, 3000).astype(np.float32)
    codes, cent, deq, obj = O.kmeans(v, 16, 0, O.kmeans_key(3, 1, 2, 3))
    assert len(set(cent.tolist())) == 16
    assert np.all(np.diff(cent) > 0)
    assert set(cent.tolist()) <= set(v.tolist())


@pytest.mark.parametrize("kdist,k", [(3, 3), (5, 8), (16, 16)])
def test_kmeans_lossless_when_few_distinct_values(kdist, k):
    rng = np.random.default_rng(kdist)
    vals = rng.normal(0, 3, kdist).astype(np.float32)
    v = vals[rng.integers(0, kdist, 48)]
    v[:kdist] = vals  # every value present; n <= probe length covers them all
    codes, cent, deq, obj = O.kmeans(v, k, 10, O.kmeans_key(1, 0, 0, 1))
    assert np.array_equal(deq, v)
    assert obj[-1] == 0.0


def dp_optimum(x, k):
    """exact optimal 1-D k-clustering: clusters are contiguous in sorted order"""
    x = np.sort(x.astype(np.float64))
    n = len(x)

    def sse(i, j):
        seg = x[i:j]
        return float(((seg - seg.mean()) ** 2).sum())

    best = {(0, 0): 0.0}
    for c in range(1, k + 1):
        for j in range(1, n + 1):
            cands = [best[(c - 1, i)] + sse(i, j) for i in range(j) if (c - 1, i) in best]
            if cands:
                best[(c, j)] = min(cands)
    return min(best[(c, n)] for c in range(1, k + 1) if (c, n) in best)


@pytest.mark.parametrize("seed", range(6))
def test_kmeans_not_better_than_exact_optimum(seed):
    rng = np.random.default_rng(100 + seed)
    n, k = 12, 3
    v = rng.normal(0, 1, n).astype(np.float32)
    _, _, _, obj = O.kmeans(v, k, 10, O.kmeans_key(seed, 0, 0, 1))
    assert obj[-1] >= dp_optimum(v, k) * (1 - 1e-9)


def test_kmeans_finds_optimum_of_separated_clusters():
    rng = np.random.default_rng(9)
    v = np.concatenate([rng.normal(c, 0.01, 4) for c in (-10.0, 0.0, 10.0)]).astype(np.float32)
    _, _, _, obj = O.kmeans(v, 3, 10, O.kmeans_key(5, 0, 0, 1))
    assert abs(obj[-1] - dp_optimum(v, 3)) <= 1e-6 * dp_optimum(v, 3)


# ------------------------------ JPEG ------------------------------------

def test_quant_table_is_annex_k(golden_dir):
    k1 = read_table(os.path.join(golden_dir, "jpeg_luma_k1.txt"))
    assert np.array_equal(O.jpeg_qtable(50), k1)
    assert np.array_equal(O.jpeg_qtable(75), (k1 * 50 + 50) // 100)
    assert np.array_equal(O.jpeg_qtable(10), np.clip((k1 * 500 + 50) // 100, 1, 255))
    assert np.all(O.jpeg_qtable(100) == 1)


def test_dct_is_scipy_orthonormal_dct2():
    rng = np.random.default_rng(1)
    for _ in range(20):
        b = rng.uniform(-128, 127, (8, 8))
        assert np.allclose(O.dct8x8(b), scipy.fft.dctn(b, type=2, norm="ortho"), atol=1e-10)
        assert np.allclose(O.idct8x8(b), scipy.fft.idctn(b, type=2, norm="ortho"), atol=1e-10)
        assert np.allclose(O.idct8x8(O.dct8x8(b)), b, atol=1e-12)


def test_dct_of_basis_function_is_a_unit_coefficient():
    for p, q in itertools.product(range(8), repeat=2):
        e = np.zeros((8, 8))
        e[p, q] = 1.0
        assert np.allclose(O.dct8x8(O.idct8x8(e)), e, atol=1e-13)
        assert abs(np.sum(O.idct8x8(e) ** 2) - 1.0) < 1e-13  # orthonormal basis


@pytest.mark.parametrize("quality", [50, 75])
@pytest.mark.parametrize("c", [0, 7, 100, 128, 129, 200, 255])
def test_constant_block_closed_form(quality, c):
    """a block of constant sample c decodes to 128 + Qdc round(8 (c-128) / Qdc) / 8"""
    seg = np.zeros((8, 16), np.float32)
    seg[:, :8] = c
    seg[0, 8], seg[1, 8] = 0.0, 255.0  # lo = 0, hi = 255: samples equal the values
    coefs, lohi, deq, nnz = O.jpeg(seg, quality)
    qdc = O.jpeg_qtable(quality)[0, 0]
    q = np.sign(8.0 * (c - 128)) * np.floor(abs(8.0 * (c - 128) / qdc) + 0.5)  # half away
    want = np.clip(np.floor(128 + qdc * q / 8.0 + 0.5), 0, 255)
    assert coefs[0, 0] == q and np.all(coefs[0, 1:] == 0)
    assert np.all(deq[:, :8] == np.float32(want) if want < 255 else deq[:, :8] == 255.0)


def test_all_lo_all_hi_and_constant_segments_round_trip_exactly():
    rng = np.random.default_rng(2)
    lo, hi = np.float32(-0.3712), np.float32(2.9183)
    seg = np.where(rng.random((16, 24)) < 0.5, lo, hi).astype(np.float32)
    seg[:8, :8] = lo
    seg[8:, 16:] = hi
    _, lohi, deq, _ = O.jpeg(seg, 50)
    assert lohi[0] == lo and lohi[1] == hi
    assert np.array_equal(deq[:8, :8], seg[:8, :8])
    assert np.array_equal(deq[8:, 16:], seg[8:, 16:])
    const = np.full((8, 8), np.float32(0.123), np.float32)
    coefs, _, deq, nnz = O.jpeg(const, 75)
    assert np.array_equal(deq, const) and nnz == 0 and not coefs.any()


def test_jpeg_error_bounded_by_dequantization_step():
    """smooth content at quality 100 (all table entries 1) decodes within
    about one 8-bit level of the input"""
    y, x = np.mgrid[0:16, 0:32]
    seg = (np.sin(x / 7.0) + np.cos(y / 5.0)).astype(np.float32)
    coefs, lohi, deq, nnz = O.jpeg(seg, 100)
    step = (lohi[1] - lohi[0]) / 255.0
    assert np.max(np.abs(deq - seg)) <= 2.0 * step
    assert nnz == int(np.count_nonzero(coefs))


def test_rational_coefficient_ties_round_half_away():
    """rows alternating +3/-3 in the pattern of cos((2i+1) pi/4): the only
    non-zero coefficient is F[4][0] = (1/8) * 64 * 3 = 24 exactly; at quality
    55 its table entry is 16, so F / Q = 1.5 is an exact tie and must round
    away from zero to 2; the decoded rows are 128 +- 32/8"""
    sig = np.array([1, -1, -1, 1, 1, -1, -1, 1])
    seg = np.zeros((8, 16), np.float32)
    seg[:, :8] = (128 + 3 * sig)[:, None]
    seg[0, 8], seg[1, 8] = 0.0, 255.0  # lo = 0, hi = 255: samples equal the values
    assert O.jpeg_qtable(55)[4, 0] == 16
    F = O.dct8x8(seg[:, :8].astype(np.float64) - 128.0)
    assert F[4, 0] == 24.0 and np.all(np.abs(np.delete(F.ravel(), 32)) < 1e-12)
    coefs, _, deq, _ = O.jpeg(seg, 55)
    assert coefs[0, 32] == 2 and np.count_nonzero(coefs[0]) == 1
    assert np.array_equal(deq[:, :8], np.broadcast_to((128 + 4 * sig)[:, None], (8, 8)).astype(np.float32))
