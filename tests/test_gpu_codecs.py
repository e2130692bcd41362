"""GPU parity of the message quantizers (Sec. 2.7) against the oracle on the
same FP32 inputs. K-means (Algorithm 5): codes identical except at rounding
ties (<= 1e-4 of entries, each off by one level). JPEG: quantized
coefficients and 8-bit levels identical except at rounding ties (<= 1e-4 of
entries, each off by one)."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import cuda, need_gpu, rel_l2
from paper_2410_06106_gb300 import api

pytestmark = pytest.mark.gpu


def mixture(n, k, seed):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-3, 3, k)
    return (centres[rng.integers(0, k, n)] + rng.normal(0, 0.15, n)).astype(np.float32)


# The kernel adds member sums in 32-bit pieces below 2^21 - 128 values and in 64-bit slots
# above, with 16-byte access when the input allows it (n % 4 == 0, 16-byte aligned start):
# the cases cover both sums, both accesses and a ragged last trip.
@pytest.mark.parametrize("n,k,seed,offset", [(8192, 16, 0, 0), (65536, 32, 1, 0), (16384, 16, 2, 0),
                                             (1000, 3, 3, 0), (37, 8, 4, 0), (5, 4, 5, 0),
                                             (65536, 32, 8, 1), (2097152, 32, 6, 0), (2097155, 16, 7, 1)])
def test_kmeans_matches_oracle(n, k, seed, offset):
    need_gpu()
    v = mixture(n, max(k // 2, 2), seed)
    key = api.kmeans_key(99, 0, seed, 1)
    assert key == O.kmeans_key(99, 0, seed, 1)
    vin = cuda(np.concatenate([np.zeros(offset, np.float32), v]))[offset:]  # offset: start 4 bytes past 16
    codes, cent, deq, obj = api.quant_kmeans(vin, k, 10, key, objective=True)
    oc, ocent, odeq, oobj = O.kmeans(v, k, 10, key)
    codes = codes.cpu().numpy().astype(int)
    diff = codes != oc
    assert diff.mean() <= 1e-4 and np.all(np.abs(codes[diff] - oc[diff]) <= 1)
    assert rel_l2(cent.cpu().numpy(), ocent) <= 1e-6
    assert rel_l2(deq.cpu().numpy(), odeq) <= 1e-5
    o = obj.cpu().numpy()
    assert np.all(np.diff(o) <= 1e-9 * o[:-1] + 1e-12)
    assert rel_l2(o, oobj) <= 1e-5


def test_kmeans_constant_and_few_values_are_lossless():
    need_gpu()
    v = np.full(4096, 0.25, np.float32)
    _, _, deq, _ = api.quant_kmeans(cuda(v), 16, 10, 7)
    assert torch.equal(deq.cpu(), torch.as_tensor(v))
    vals = np.array([-1.5, 0.0, 2.25], np.float32)
    v = vals[np.arange(48) % 3]
    _, _, deq, _ = api.quant_kmeans(cuda(v), 3, 10, 11)
    assert torch.equal(deq.cpu(), torch.as_tensor(v))


def smooth_segment(rows, cols, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:rows, 0:cols]
    s = np.zeros((rows, cols))
    for _ in range(6):
        a, b, c = rng.uniform(0.01, 0.2, 3)
        s += rng.uniform(-1, 1) * np.sin(a * x + b * y + c * 7)
    return (s + 0.05 * rng.standard_normal((rows, cols))).astype(np.float32)


@pytest.mark.parametrize("rows,cols,q", [(32, 256, 50), (32, 512, 50), (32, 2048, 75), (8, 8, 75),
                                         (128, 1024, 10), (16, 64, 100)])
def test_jpeg_matches_oracle(rows, cols, q):
    need_gpu()
    v = smooth_segment(rows, cols, rows + cols + q)
    coefs, lohi, deq, nnz = api.quant_jpeg(cuda(v), q)
    oc, olohi, odeq, onnz = O.jpeg(v, q)
    c = coefs.cpu().numpy().astype(int)
    diff = c != oc
    assert diff.mean() <= 1e-4 and np.all(np.abs(c[diff] - oc[diff]) <= 1)
    assert np.array_equal(lohi.cpu().numpy(), olohi)
    assert abs(int(nnz.item()) - onnz) <= diff.sum()
    # decoded 8-bit levels: identical in every block whose codes agree, except
    # at rounding ties of the inverse transform
    step = (olohi[1] - olohi[0]) / 255.0
    d = deq.cpu().numpy()
    same = ~diff.any(axis=1)  # blocks with identical codes
    blocks = lambda a: a.reshape(rows // 8, 8, cols // 8, 8).transpose(0, 2, 1, 3).reshape(-1, 64)
    lev = np.abs(blocks(d) - blocks(odeq))[same]
    assert (lev > 0.5 * step).mean() <= 1e-4 and np.all(lev <= 1.01 * step)


def test_jpeg_exact_cases():
    need_gpu()
    lo, hi = np.float32(-0.3712), np.float32(2.9183)
    rng = np.random.default_rng(2)
    seg = np.where(rng.random((16, 24)) < 0.5, lo, hi).astype(np.float32)
    seg[:8, :8] = lo
    seg[8:, 16:] = hi
    _, _, deq, _ = api.quant_jpeg(cuda(seg), 50)
    d = deq.cpu().numpy()
    assert np.array_equal(d[:8, :8], seg[:8, :8]) and np.array_equal(d[8:, 16:], seg[8:, 16:])
    const = np.full((8, 16), np.float32(0.123), np.float32)
    coefs, _, deq, nnz = api.quant_jpeg(cuda(const), 75)
    assert torch.equal(deq.cpu(), torch.as_tensor(const)) and int(nnz.item()) == 0
    for c in (0, 7, 100, 129, 255):  # constant blocks decide DC ties exactly like the oracle
        seg = np.zeros((8, 16), np.float32)
        seg[:, :8] = c
        seg[0, 8], seg[1, 8] = 0.0, 255.0
        coefs, _, deq, _ = api.quant_jpeg(cuda(seg), 50)
        oc, _, odeq, _ = O.jpeg(seg, 50)
        assert np.array_equal(coefs.cpu().numpy()[0], oc[0])
        assert np.array_equal(deq.cpu().numpy()[:, :8], odeq[:, :8])


def test_jpeg_rational_coefficient_tie():
    """F[4][0] = 24, Q = 16 at quality 55: an exact tie, rounded away from zero
    on both sides"""
    need_gpu()
    sig = np.array([1, -1, -1, 1, 1, -1, -1, 1])
    seg = np.zeros((8, 16), np.float32)
    seg[:, :8] = (128 + 3 * sig)[:, None]
    seg[0, 8], seg[1, 8] = 0.0, 255.0
    coefs, _, deq, _ = api.quant_jpeg(cuda(seg), 55)
    oc, _, odeq, _ = O.jpeg(seg, 55)
    assert coefs.cpu().numpy()[0, 32] == 2
    assert np.array_equal(coefs.cpu().numpy(), oc) and np.array_equal(deq.cpu().numpy(), odeq)


def random_blocks(nblk, seed):
    """Laplacian-like sparse quantized blocks over the whole baseline range"""
    rng = np.random.default_rng(seed)
    zz = O.zigzag()
    c = np.zeros((nblk, 64), np.int16)
    for b in range(nblk):
        c[b, 0] = rng.integers(-1024, 1017)
        k = int(rng.integers(0, 64))
        pos = rng.choice(np.arange(1, 64), k, replace=False)
        c[b, zz[pos]] = np.clip(np.round(rng.laplace(0, [1, 20, 300][b % 3], k)), -1023, 1023)
    return c


@pytest.mark.parametrize("rows,cols,seed", [(8, 8, 0), (16, 800, 1), (64, 64, 2), (256, 512, 3), (8, 2056, 4)])
def test_entropy_coding_matches_oracle_bytewise(rows, cols, seed):
    """the stuffed baseline entropy-coded segment, byte for byte (several
    256-block batches in the larger cases)"""
    need_gpu()
    nblk = (rows // 8) * (cols // 8)
    c = random_blocks(nblk, seed)
    ref = O.jpeg_entropy(c)
    got = api.jpeg_entropy(torch.as_tensor(c).cuda(), rows, cols)
    assert got == ref
    assert api.jpeg_entropy(torch.as_tensor(c).cuda(), rows, cols, stream=False) == len(ref)


def test_entropy_coding_of_quantizer_output_and_stuffing():
    """coefficients from the JPEG quantizer at several qualities, and a block
    whose stream holds a stuffed 0xFF"""
    need_gpu()
    rng = np.random.default_rng(11)
    x = np.cumsum(rng.standard_normal((64, 512)), axis=1).astype(np.float32)
    for q in (10, 50, 75, 95):
        coefs, _, _, _ = api.quant_jpeg(cuda(x), q)
        assert api.jpeg_entropy(coefs, 64, 512) == O.jpeg_entropy(coefs.cpu().numpy())
    c = np.zeros((2, 64), np.int16)
    c[0, 0] = 1
    c[0, O.zigzag()[16]] = 1000
    data = api.jpeg_entropy(torch.as_tensor(c).cuda(), 8, 16)
    assert b"\xff\x00" in data and data == O.jpeg_entropy(c)


def test_entropy_coding_refuses_out_of_range_coefficients():
    need_gpu()
    c = np.zeros((1, 64), np.int16)
    c[0, 1] = 1024
    with pytest.raises(api.TomoError):
        api.jpeg_entropy(torch.as_tensor(c).cuda(), 8, 8)


@pytest.mark.parametrize("n,k,kind", [(65536, 8, "halves"), (65536, 32, "halves"), (65536, 32, "zeros"),
                                      (4099, 16, "halves"), (65536, 16, "magnitudes")])
def test_kmeans_duplicates_and_exact_ties_match_oracle(n, k, kind):
    """Inputs that stress the decision rule: few distinct values (multiples of 1/2 in
    [-3, 3], so that values fall exactly halfway between centres and, with k above
    the 13 distinct values, centres repeat); mostly zeros; magnitudes over seven
    decades. Codes, centres and dequantized values follow the oracle (Algorithm 5)."""
    need_gpu()
    rng = np.random.default_rng(n + k)
    if kind == "halves":
        v = (rng.integers(-6, 7, n) * 0.5).astype(np.float32)
    elif kind == "zeros":
        v = np.where(rng.random(n) < 0.7, 0.0, rng.normal(0, 1, n)).astype(np.float32)
    else:
        v = (rng.standard_normal(n) * 10.0 ** rng.integers(-3, 4, n)).astype(np.float32)
    key = api.kmeans_key(7, 1, k, 2)
    codes, cent, deq, _ = api.quant_kmeans(cuda(v), k, 10, key)
    oc, ocent, odeq, _ = O.kmeans(v, k, 10, key)
    codes = codes.cpu().numpy().astype(int)
    diff = codes != oc
    assert diff.mean() <= 1e-4 and np.all(np.abs(codes[diff] - oc[diff]) <= 1)
    assert rel_l2(cent.cpu().numpy(), ocent) <= 1e-6
    assert rel_l2(deq.cpu().numpy(), odeq) <= 1e-5
