"""CPU checks of the integer identities the fused kernel's packed count
relies on (the kernel itself is checked bit-exactly against the oracle by the
GPU parity tests).

The dense passes sum the 0/1 results of the fp16 closed-neighbour test as
32-bit integers: each result is the fp16 bit pattern 0x0000 or 0x3C00 in the
low (pixel 2j) or high (pixel 2j + 1) half of a word.  After K_lo and K_hi
closed neighbours the word, times 47 modulo 2^32, must have byte 1 equal to
4 K_lo and byte 3 equal to 4 K_hi + (0..2), so that "at most one closed
neighbour" is "byte & 0xF8 == 0"; and the SWAR test that marks the bytes
with bit 7 must agree.  Both are checked for every K_lo, K_hi <= 48 (beta
<= 3 has at most 48 neighbours)."""
import itertools


def packed_count(k_lo, k_hi):
    return (k_lo * 0x3C00 + k_hi * 0x3C00 * 65536) % 2**32


def test_decode_bytes_exhaustive():
    for k_lo, k_hi in itertools.product(range(49), repeat=2):
        z = packed_count(k_lo, k_hi) * 47 % 2**32
        b1, b3 = (z >> 8) & 0xFF, (z >> 24) & 0xFF
        assert b1 == 4 * k_lo, (k_lo, k_hi)
        assert 4 * k_hi <= b3 <= 4 * k_hi + 2, (k_lo, k_hi)
        assert ((b1 & 0xF8) == 0) == (k_lo <= 1)
        assert ((b3 & 0xF8) == 0) == (k_hi <= 1)


def test_swar_byte_test_exhaustive():
    """((q & 0x78787878) + 0x7F7F7F7F | q) & 0x80808080 sets bit 7 of exactly
    the bytes of q with (byte & 0xF8) != 0, for every byte value."""
    for v in range(256):
        for pos in range(4):
            q = v << (8 * pos)
            nz = (((q & 0x78787878) + 0x7F7F7F7F) | q) & 0x80808080
            expect = (0x80 << (8 * pos)) if (v & 0xF8) else 0
            assert nz == expect, (v, pos)
    # four bytes at once (every combination of the four states that matter)
    for bytes_ in itertools.product((0, 5, 7, 8, 0x80, 0xFF), repeat=4):
        q = sum(b << (8 * i) for i, b in enumerate(bytes_))
        nz = (((q & 0x78787878) + 0x7F7F7F7F) | q) & 0x80808080
        assert nz == sum((0x80 << (8 * i)) for i, b in enumerate(bytes_) if b & 0xF8)


def test_gather_of_bytes_1_and_3():
    """The byte permute 0x7531 of (a, b) gathers bytes 1 and 3 of a, then of
    b: pixels 0-3 of the 8-pixel segment from the words of pairs 0 and 1."""
    def prmt(a, b, sel):
        src = a | (b << 32)
        out = 0
        for i in range(4):
            idx = (sel >> (4 * i)) & 0x7
            out |= ((src >> (8 * idx)) & 0xFF) << (8 * i)
        return out
    a, b = 0x44332211, 0x88776655
    assert prmt(a, b, 0x7531) == 0x88664422


def test_two_stage_decision_table():
    """beta 3's two-stage count: stage one keeps a pixel when its inner-ring
    count K_in is 0 or 1 (flag bits: not settled, K_in == 1); stage two has
    byte b = 4 K_out (+ 0..2) of its outer-ring count and calls it a
    candidate when b < (4 if K_in == 1 else 8).  That must be K_in + K_out
    <= 1 for every K_in <= 8 and K_out <= 40 (the 8 inner and 40 outer
    neighbours of a 7 x 7 window)."""
    for k_in in range(9):
        unsettled = k_in <= 1
        for k_out in range(41):
            for k_other in range(41):  # the pair's other pixel only moves the carry
                acc = (k_out * 0x3C00 + k_other * 0x3C00 * 65536) % 2**32
                z = acc * 47 % 2**32
                b_lo = (z >> 8) & 0xFF
                cand = unsettled and b_lo < (4 if k_in == 1 else 8)
                assert cand == (k_in + k_out <= 1), (k_in, k_out, k_other)
                acc2 = (k_other * 0x3C00 + k_out * 0x3C00 * 65536) % 2**32
                b_hi = (acc2 * 47 % 2**32) >> 24
                cand_hi = unsettled and b_hi < (4 if k_in == 1 else 8)
                assert cand_hi == (k_in + k_out <= 1), (k_in, k_out, k_other, "hi")


def test_symmetric_pair_test_fp16_exhaustive():
    """The symmetric count (beta 1 and 2) tests each unordered pixel pair once
    with sat(2 alpha - 1 - 2 |v_n - v_p|) in fp16x2: an fp16 subtraction of
    the two values, then one fused multiply-add with saturation.  For every
    pair of 8-bit values and every alpha it must be exactly 1.0 when
    |v_n - v_p| < alpha (Algorithm 1's test) and +0 otherwise, with the
    roundings of fp16 arithmetic; and that test must imply Algorithm 2's
    closed test (v_p - alpha < v_n <= v_p + alpha), so that a pixel with at
    most one closed neighbour has at most one neighbour passing it."""
    import numpy as np
    v = np.arange(256, dtype=np.float16)
    vp, vn = np.meshgrid(v, v, indexing="ij")
    e = (vn - vp).astype(np.float16)              # exact: integers within +-255
    assert np.array_equal(e.astype(np.int32), vn.astype(np.int32) - vp.astype(np.int32))
    ip, inn = vp.astype(np.int32), vn.astype(np.int32)
    for alpha in range(256):
        lim = np.float16(2 * alpha - 1)
        # fma rounds once: |e| * -2 + lim is an integer of magnitude below 2048, exact in fp16
        f = np.clip((np.abs(e).astype(np.float64) * -2.0 + float(lim)).astype(np.float16), 0, 1)
        strict = np.abs(inn - ip) < alpha
        assert np.array_equal(f == 1, strict) and np.all((f == 0) | (f == 1)), alpha
        closed = (inn > ip - alpha) & (inn <= ip + alpha)
        assert not np.any(strict & ~closed), alpha
