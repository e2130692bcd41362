"""Pins of the oracle's baseline JPEG entropy coder (ITU-T T.81 Annex F.1.2,
luminance tables K.3 / K.5): the code tables against the standard's code
words and the structure every Huffman table must have, the zig-zag order,
a stream worked by hand, byte stuffing, and decode(encode(c)) == c."""
import numpy as np
import pytest

import oracle as O

# (symbol, code word) pairs printed in Tables K.3 and K.5
DC_WORDS = {0: "00", 1: "010", 2: "011", 3: "100", 4: "101", 5: "110", 6: "1110", 7: "11110",
            8: "111110", 9: "1111110", 10: "11111110", 11: "111111110"}
AC_WORDS = {0x00: "1010", 0x01: "00", 0x02: "01", 0x03: "100", 0x04: "1011", 0x05: "11010",
            0x11: "1100", 0x12: "11011", 0x21: "11100", 0x31: "111010", 0xF0: "11111111001",
            0x82: "111111111000000", 0x09: "1111111110000010", 0xFA: "1111111111111110"}


def word(ac, sym):
    code, ln = O.huff_code(ac, sym)
    return format(code, "0%db" % ln) if ln else ""


def test_code_words_of_the_standard_tables():
    for s, w in DC_WORDS.items():
        assert word(False, s) == w
    for s, w in AC_WORDS.items():
        assert word(True, s) == w


def test_tables_are_complete_prefix_codes_over_the_baseline_symbols():
    ac_syms = [0x00, 0xF0] + [(r << 4) | s for r in range(16) for s in range(1, 11)]
    for ac, syms in ((False, range(12)), (True, ac_syms)):
        words = [word(ac, s) for s in syms]
        assert all(words) and len(set(words)) == len(words)
        for a in words:  # prefix-free
            assert not any(b != a and b.startswith(a) for b in words)
        kraft = sum(2.0 ** -len(w) for w in words)
        assert kraft < 1.0 and kraft > 0.99  # no all-ones code word (Annex C)
    assert all(word(True, s) == "" for s in range(256) if s not in ac_syms)


def test_zigzag_order():
    zz = O.zigzag()
    assert sorted(zz.tolist()) == list(range(64))
    assert zz[:10].tolist() == [0, 1, 8, 16, 9, 2, 3, 10, 17, 24] and zz[-1] == 63
    for a, b in zip(zz[:-1], zz[1:]):  # every step moves to a neighbouring cell
        assert max(abs(a // 8 - b // 8), abs(a % 8 - b % 8)) == 1


def test_hand_worked_stream():
    """DC 5 (category 3: 100 + 101), AC -3 at zig-zag 1 (symbol 0x02: 01 +
    extra 00), EOB 1010: 14 bits 10010101 001010, padded with 11"""
    c = np.zeros((1, 64), np.int16)
    c[0, 0], c[0, 1] = 5, -3
    assert O.jpeg_entropy(c) == bytes([0x95, 0x2B])
    # a second block with the same DC codes a zero difference (00) and EOB
    c2 = np.concatenate([c, np.array([[5] + [0] * 63], np.int16)])
    # 10010101 00101000 1010 + 1111 -> 0x95 0x28 0xAF
    assert O.jpeg_entropy(c2) == bytes([0x95, 0x28, 0xAF])


def test_byte_stuffing():
    """DC 1 (010 1) then 15 zeros and 1000 at zig-zag 16 (symbol 0xFA, 16
    bits 1111111111111110): bits 8..15 are eight ones, so 0xFF 0x00 follow
    the first byte"""
    c = np.zeros((1, 64), np.int16)
    c[0, 0] = 1
    c[0, O.zigzag()[16]] = 1000
    data = O.jpeg_entropy(c)
    assert data[1:3] == b"\xff\x00"
    assert np.array_equal(O.jpeg_entropy_decode(data, 1), c)
    # length = whole bytes of the bit count + one stuffed zero per 0xFF
    bits = 3 + 1 + 16 + 10 + 4  # DC code + extra, AC code + extra, EOB
    assert len(data) == (bits + 7) // 8 + 1


@pytest.mark.parametrize("seed", range(6))
def test_round_trip_and_bit_count(seed):
    rng = np.random.default_rng(seed)
    nblk = int(rng.integers(1, 300))
    c = np.zeros((nblk, 64), np.int16)
    zz = O.zigzag()
    for b in range(nblk):  # Laplacian-like sparse blocks, long zero runs, full range
        c[b, 0] = rng.integers(-1024, 1017)
        k = int(rng.integers(0, 64))
        pos = rng.choice(np.arange(1, 64), k, replace=False)
        c[b, zz[pos]] = np.clip(np.round(rng.laplace(0, [1, 20, 300][b % 3], k)), -1023, 1023)
    data = O.jpeg_entropy(c)
    assert np.array_equal(O.jpeg_entropy_decode(data, nblk), c)
    # independent bit count from the code lengths
    bits, pred = 0, 0
    for b in range(nblk):
        d = int(c[b, 0]) - pred
        pred = int(c[b, 0])
        s = abs(d).bit_length()
        bits += O.huff_code(False, s)[1] + s
        run = 0
        for k in range(1, 64):
            v = int(c[b, zz[k]])
            if v == 0:
                run += 1
                continue
            while run > 15:
                bits += O.huff_code(True, 0xF0)[1]
                run -= 16
            s = abs(v).bit_length()
            bits += O.huff_code(True, (run << 4) | s)[1] + s
            run = 0
        if run:
            bits += O.huff_code(True, 0)[1]
    n_ff = 0
    i = 0
    while i < len(data):  # count stuffed pairs
        if data[i] == 0xFF:
            assert data[i + 1] == 0
            n_ff += 1
            i += 2
        else:
            i += 1
    assert len(data) == (bits + 7) // 8 + n_ff


def test_out_of_range_coefficient_is_refused():
    c = np.zeros((1, 64), np.int16)
    c[0, 1] = 1024  # category 11 is not a baseline AC size
    with pytest.raises(ValueError):
        O.jpeg_entropy(c)
