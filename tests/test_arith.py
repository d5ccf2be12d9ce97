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


def test_reciprocal_division_exhaustive():
    """The kernels' floor(sum / flag) is the high word of sum * ceil(2^32 /
    flag).  For every window of beta 1..7 a replaced pixel has flag in {P - 2,
    P - 1, P} (P = (2 beta + 1)^2, Algorithm 2's test flag > pix_count - 3)
    and 0 <= sum <= flag * 255^2: every such sum must give the exact
    quotient."""
    import numpy as np
    for beta in range(1, 8):
        p = (2 * beta + 1) ** 2
        for flag in (p - 2, p - 1, p):
            m = np.uint64((2**32 + flag - 1) // flag)
            top = flag * 255 * 255
            for lo in range(0, top + 1, 1 << 22):
                s = np.arange(lo, min(lo + (1 << 22), top + 1), dtype=np.uint64)
                assert np.array_equal((s * m) >> np.uint64(32), s // np.uint64(flag)), (beta, flag, lo)


def test_reciprocal_division_every_flag_at_the_quotient_edges():
    """hgrms_rms uses the same division for every flag 2..225: the largest
    remainder of each quotient is where the high word would first exceed it."""
    import numpy as np
    q = np.arange(0, 255 * 255 + 1, dtype=np.uint64)
    for flag in range(2, 226):
        m = np.uint64((2**32 + flag - 1) // flag)
        for r in (0, flag - 1):
            s = q * np.uint64(flag) + np.uint64(r)
            s = s[s <= flag * 255 * 255]
            assert np.array_equal((s * m) >> np.uint64(32), s // np.uint64(flag)), (flag, r)


def test_isqrt_rounding_with_rsqrt_error_bound():
    """The kernels' integer square root of q <= 255^2: q as a float from its
    bit pattern (2^23 + q minus 2^23), times rsqrtf(q), rounded to the
    nearest integer by adding 1.5 * 2^23, less one when its square exceeds
    q.  With rsqrtf anywhere within its 2 ulp error bound the result must be
    floor(sqrt(q)) for every q (float32 arithmetic, round to nearest even)."""
    import math
    import numpy as np
    q = np.arange(0, 255 * 255 + 1, dtype=np.int64)
    qf = (np.array(0x4B000000 | q, dtype=np.uint32).view(np.float32) - np.float32(8388608.0)).astype(np.float32)
    assert np.array_equal(qf.astype(np.int64), q)
    exact = np.array([math.isqrt(int(v)) for v in q], dtype=np.int64)
    base = (1.0 / np.sqrt(np.maximum(qf, 1).astype(np.float64))).astype(np.float32)
    for ulps in range(-2, 3):
        rs = base
        for _ in range(abs(ulps)):
            rs = np.nextafter(rs, np.float32(np.inf if ulps > 0 else 0)).astype(np.float32)
        s = (qf * rs).astype(np.float32)
        t = (s + np.float32(12582912.0)).astype(np.float32)
        r = t.view(np.int32).astype(np.int64) - 0x4B400000
        r -= (r * r > q).astype(np.int64)
        assert np.array_equal(r, exact), ulps


def _bytes_in_range(v, lo, hi):
    """Python form of the list-pass kernel's bytes_in_range (uint64 arrays
    holding 32-bit words): 0xFF in every byte of v with lo <= byte <= hi."""
    import numpy as np
    m32 = np.uint64(0xFFFFFFFF)
    kl = (np.uint64(0x01000100) - lo.astype(np.uint64) * np.uint64(0x00010001)) & m32
    kh = (np.uint64(0x01000100) - (hi.astype(np.uint64) + np.uint64(1)) * np.uint64(0x00010001)) & m32
    e = v & np.uint64(0x00FF00FF)
    o = ((v >> np.uint64(8)) & np.uint64(0xFF)) | (((v >> np.uint64(24)) & np.uint64(0xFF)) << np.uint64(16))
    ce = ((e + kl) & m32) & (~((e + kh) & m32) & m32)
    co = ((o + kl) & m32) & (~((o + kh) & m32) & m32)
    m = ((ce >> np.uint64(8)) & np.uint64(0x00010001)) | (co & np.uint64(0x01000100))
    return (m * np.uint64(0xFF)) & m32


def test_swar_closed_test_exhaustive():
    """The list passes test four window values at once: a byte v is closed
    for the centre value ip when ip - alpha < v <= ip + alpha (Algorithm 2),
    i.e. lo <= v <= hi with lo = max(ip - alpha + 1, 0), hi = min(ip + alpha,
    255).  Every (ip, alpha, v) with v in each byte position, the other
    bytes random (no carry may leak between bytes)."""
    import numpy as np
    rng = np.random.default_rng(5)
    ip = np.repeat(np.arange(256), 256).astype(np.int64)
    v = np.tile(np.arange(256), 256).astype(np.int64)
    for alpha in range(256):
        lo = np.maximum(ip - alpha + 1, 0)
        hi = np.minimum(ip + alpha, 255)
        expect = (v > ip - alpha) & (v <= ip + alpha)
        for pos in range(4):
            other = rng.integers(0, 2**32, size=v.size, dtype=np.uint64) & ~np.uint64(0xFF << (8 * pos))
            word = other | (v.astype(np.uint64) << np.uint64(8 * pos))
            got = (_bytes_in_range(word, lo, hi) >> np.uint64(8 * pos)) & np.uint64(0xFF)
            assert np.array_equal(got == 0xFF, expect) and np.all((got == 0) | (got == 0xFF)), (alpha, pos)


def test_swar_window_evaluation_matches_definition():
    """The list passes' whole evaluation of Algorithm 2 from byte words (rows
    of 2 beta + 1 values, four per word; beta 2 gathers the fifth value of
    rows 0-3 into one word): the sum of the open values' squares (4-way dot
    products) and their count (a second dot product with 0x01010101: 255
    per open value), against the definition,
    on random windows of beta 1, 2 and 3 with values near the centre."""
    import numpy as np
    rng = np.random.default_rng(11)
    for beta in (1, 2, 3):
        w = 2 * beta + 1
        for trial in range(4000):
            alpha = int(rng.integers(0, 40))
            ip = int(rng.integers(0, 256))
            win = np.clip(ip + rng.integers(-2 * alpha - 3, 2 * alpha + 4, size=(w, w)), 0, 255)
            if trial % 3 == 0:
                win = rng.integers(0, 256, size=(w, w))
            win[beta, beta] = ip
            nw = (w + 3) // 4
            rowwords = []
            for r in range(w):
                vals = list(win[r]) + [int(rng.integers(0, 256)) for _ in range(4 * nw - w)]
                rowwords.append([sum(int(vals[4 * k + j]) << (8 * j) for j in range(4)) for k in range(nw)])
            words, oks = [], []
            if beta == 2:
                for r in range(w):
                    words.append(rowwords[r][0]); oks.append(0xFFFFFFFF)
                packed = sum((rowwords[r][1] & 0xFF) << (8 * r) for r in range(4))
                words += [packed, rowwords[4][1]]; oks += [0xFFFFFFFF, 0xFF]
            else:
                last = w - 4 * (nw - 1)
                for r in range(w):
                    for k in range(nw):
                        words.append(rowwords[r][k])
                        oks.append(0xFFFFFFFF if (k < nw - 1 or last == 4) else (1 << (8 * last)) - 1)
            words = np.array(words, dtype=np.uint64)
            lo = np.full(words.shape, max(ip - alpha + 1, 0)); hi = np.full(words.shape, min(ip + alpha, 255))
            closed = _bytes_in_range(words, lo, hi)
            s, open255 = 0, 0
            for word, c, ok in zip(words.tolist(), closed.tolist(), oks):
                open_ = ~c & ok & 0xFFFFFFFF
                for j in range(4):
                    ob = (open_ >> (8 * j)) & 0xFF
                    b = (word >> (8 * j)) & 0xFF
                    s += (b & ob) * b     # dp4a(v & open, v)
                    open255 += ob * 1     # dp4a(open, 0x01010101)
            op = ~((win > ip - alpha) & (win <= ip + alpha))
            assert open255 == 255 * int(op.sum()), (beta, trial)
            assert s == int((win.astype(np.int64) ** 2 * op).sum()), (beta, trial)


def test_three_stage_decision_table():
    """beta 3's staged count: after the inner ring (K_in <= 1 for a pixel
    still in the work list), stage two adds the ring at distance 2 (K_mid <=
    16) and keeps the pixel when its byte b = 4 K_mid (+ 0..2) is below 4
    (K_in = 1) or 8 (K_in = 0), recording K_in + K_mid as 1 when K_in = 1 or
    b >= 4; stage three then applies the two-stage rule with that count.
    Every combination of the counts, the pair's other pixel only moving the
    carry: kept exactly when K_in + K_mid <= 1, with the right count."""
    for k_in in range(2):
        for k_mid in range(17):
            for k_other in range(17):
                for hi in (False, True):
                    lo_val = (k_other if hi else k_mid) * 0x3C00
                    hi_val = (k_mid if hi else k_other) * 0x3C00
                    z = ((lo_val + (hi_val << 16)) % 2**32) * 47 % 2**32
                    b = (z >> 24) if hi else ((z >> 8) & 0xFF)
                    kept = b < (4 if k_in == 1 else 8)
                    assert kept == (k_in + k_mid <= 1), (k_in, k_mid, k_other, hi)
                    if kept:
                        assert (1 if (k_in == 1 or b >= 4) else 0) == k_in + k_mid
