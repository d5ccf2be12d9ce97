"""Pins of the CPU oracle to facts that do not come from the oracle itself.

* hand-derived worked examples (tests/golden/*.txt, each citing the passage
  of Algorithms 1-2 / Section 2 it exercises);
* the literal transcription of Algorithm 1 (scattered increments into the
  neighbour's count) and Algorithm 2 with an explicit temporary image and
  copy-back, against the gather-form oracle - exhaustively on 3x3 images
  over small palettes and on random images of every beta;
* the integer square root against Python's math.isqrt over the whole range
  the method can produce;
* mathematical invariants: border band of width beta never changes, a
  converged image is a fixed point, k <= max_k with the documented stop
  rule, passes are deterministic, PSNR closed forms.
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_1306_5390_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(path):
    """Parse a golden file: key/value lines and image blocks."""
    d = {}
    lines = [ln.rstrip("\n") for ln in open(path) if not ln.startswith("#") and ln.strip()]
    i = 0
    rows = cols = None
    while i < len(lines):
        parts = lines[i].split()
        key = parts[0]
        if key == "input":
            rows, cols = int(parts[1]), int(parts[2])
            d["input"] = np.array([[int(v) for v in lines[i + 1 + r].split()] for r in range(rows)],
                                  dtype=np.uint8)
            i += 1 + rows
        elif key in ("pass1", "output"):
            d[key] = np.array([[int(v) for v in lines[i + 1 + r].split()] for r in range(rows)],
                              dtype=np.uint8)
            i += 1 + rows
        else:
            d[key] = int(parts[1])
            i += 1
    assert d["input"].shape == (rows, cols)
    return d


GOLDEN_FILES = sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))


@pytest.mark.parametrize("name", GOLDEN_FILES)
def test_golden_worked_examples(oracle_mod, name):
    g = load_golden(os.path.join(GOLDEN, name))
    a, b, mk = g["alpha"], g["beta"], g["max_k"]
    out, k, conv = oracle_mod.denoise(g["input"], a, b, mk)
    assert k == g["k"], name
    assert conv == bool(g["converged"]), name
    np.testing.assert_array_equal(out, g["output"], err_msg=name)
    lout, lk, lconv = oracle_mod.literal_denoise(g["input"], a, b, mk)
    assert (lk, lconv) == (k, conv)
    np.testing.assert_array_equal(lout, g["output"])
    if "pass1" in g:
        p1, _ = oracle_mod.one_pass(g["input"], a, b)
        np.testing.assert_array_equal(p1, g["pass1"], err_msg=name)


def test_golden_files_cite_the_paper():
    for name in GOLDEN_FILES:
        text = open(os.path.join(GOLDEN, name)).read()
        assert "# cite:" in text and ("Algorithm" in text or "Section" in text), name


def test_isqrt_exhaustive(oracle_mod):
    # The method only takes square roots of floor(sum/flag) <= 255^2; check a
    # wider range plus the 32-bit extremes.
    for x in range(0, 70000):
        assert oracle_mod.isqrt(x) == math.isqrt(x)
    for x in (2**24 - 1, 2**24, 2**31, 2**32 - 1):
        assert oracle_mod.isqrt(x) == math.isqrt(x)


@pytest.mark.parametrize("beta", [1, 2, 3])
@pytest.mark.parametrize("alpha", [0, 1, 5, 10, 255])
def test_scatter_card_equals_gather_card(oracle_mod, alpha, beta):
    for seed in range(12):
        rows, cols = 1 + seed % 9, 1 + (seed * 7) % 12
        img = synth.random_image(rows, cols, 1000 + seed, levels=[0, 3, 9, 10, 11, 20, 250, 255])
        np.testing.assert_array_equal(oracle_mod.literal_card(img, alpha, beta),
                                      oracle_mod.card(img, alpha, beta))


def test_exhaustive_3x3_literal_vs_gather(oracle_mod):
    """All 3^9 images over three palettes; one pass of the literal form
    (scatter + Algorithm 2 + copy-back) equals one gather pass."""
    palettes = [(0, 100, 255), (100, 110, 90), (0, 5, 10)]
    for pal, alpha in itertools.product(palettes, (0, 1, 10, 100)):
        imgs = np.array(list(itertools.product(pal, repeat=9)), dtype=np.uint8).reshape(-1, 3, 3)
        for img in imgs[:: 1 if alpha == 10 else 7]:
            c = oracle_mod.literal_card(img, alpha, 1)
            lit, lch = oracle_mod.literal_remove_noise(img, c, alpha, 1)
            out, ch = oracle_mod.one_pass(img, alpha, 1)
            assert lch == ch
            assert np.array_equal(lit, out)


def _direct_pass_4x4(imgs, alpha):
    """One pass of Algorithms 1-2 (beta 1) on a stack of 4 x 4 images, by
    the definitions: the four interior pixels each read their 3 x 3 window
    of the previous image (Section 2's temporary image and copy-back);
    card counts |I_n - I_p| < alpha, and for card <= 2 a window value is
    open unless I_p - alpha < I_n <= I_p + alpha; flag > 9 - 3 replaces the
    pixel by floor(sqrt(floor(sum / flag)))."""
    old = imgs.astype(np.int64)
    out = old.copy()
    for y in (1, 2):
        for x in (1, 2):
            p = old[:, y, x][:, None]
            win = old[:, y - 1:y + 2, x - 1:x + 2].reshape(len(old), 9)
            card = ((win > p - alpha) & (win < p + alpha)).sum(axis=1)
            opn = ~((win > p - alpha) & (win <= p + alpha))
            flag = opn.sum(axis=1)
            ssum = (win * win * opn).sum(axis=1)
            q = ssum // np.maximum(flag, 1)
            r = np.floor(np.sqrt(q.astype(np.float64))).astype(np.int64)
            r -= (r * r > q)
            r += ((r + 1) * (r + 1) <= q)
            rep = (card <= 2) & (flag > 6)
            out[:, y, x] = np.where(rep, r, old[:, y, x])
    return out.astype(np.uint8)


def test_sampled_4x4_against_the_direct_definition(oracle_mod):
    """4 x 4 images (the smallest whose interior windows overlap, so a pass
    that updated pixels in place would differ), 8,000 per palette and alpha
    drawn from 3^16: the oracle's iteration (bytes, k, converged; max_k 4)
    equals iterating the direct definition with the stop rule of Section 2
    (k = passes that changed a pixel, stopping after the first that changes
    none)."""
    rng = np.random.Generator(np.random.PCG64(4416))
    palettes = [(0, 100, 255), (100, 110, 90), (0, 5, 10)]
    max_k = 4
    for pal, alpha in itertools.product(palettes, (0, 1, 10, 100)):
        imgs = np.asarray(pal, dtype=np.uint8)[rng.integers(0, 3, size=(8000, 4, 4))]
        cur = imgs.copy()
        k = np.zeros(len(imgs), dtype=np.int64)
        done = np.zeros(len(imgs), dtype=bool)
        for _ in range(max_k):
            nxt = _direct_pass_4x4(cur, alpha)
            changed = (nxt != cur).reshape(len(cur), -1).any(axis=1)
            done |= ~changed
            k += changed & ~done
            cur = np.where(done[:, None, None], cur, nxt)
        for i in range(len(imgs)):
            out, k_o, conv = oracle_mod.denoise(imgs[i], alpha, 1, max_k)
            assert (k_o, conv) == (int(k[i]), bool(done[i])), (pal, alpha, imgs[i].tolist())
            assert np.array_equal(out, cur[i]), (pal, alpha, imgs[i].tolist())


@pytest.mark.parametrize("beta", [1, 2, 3, 4, 7])
def test_literal_loop_equals_gather_loop_random(oracle_mod, beta):
    for seed in range(6):
        rows, cols = 3 + seed * 5, 4 + seed * 7
        img = synth.random_image(rows, cols, 50 + seed, levels=[0, 40, 45, 50, 55, 255])
        for alpha in (0, 6, 10, 30):
            a = oracle_mod.denoise(img, alpha, beta, 9)
            b = oracle_mod.literal_denoise(img, alpha, beta, 9)
            assert a[1:] == b[1:]
            np.testing.assert_array_equal(a[0], b[0])


@pytest.mark.parametrize("beta", [1, 2, 3])
def test_literal_loop_equals_gather_loop_synthetic(oracle_mod, beta):
    clean, noisy = synth.noisy_image(48, 61, 0.3, synth.seed_for(9, beta))
    for alpha in (5, 10, 20):
        a = oracle_mod.denoise(noisy, alpha, beta, 32)
        b = oracle_mod.literal_denoise(noisy, alpha, beta, 32)
        assert a[1:] == b[1:]
        np.testing.assert_array_equal(a[0], b[0])


@pytest.mark.parametrize("beta", [1, 2, 3, 5])
def test_border_band_never_changes(oracle_mod, beta):
    for seed in range(4):
        img = synth.random_image(20 + seed, 23 + 2 * seed, 300 + seed)
        for alpha in (0, 1, 10, 64):
            out, k, _ = oracle_mod.denoise(img, alpha, beta, 20)
            band = np.ones(img.shape, dtype=bool)
            band[beta:-beta, beta:-beta] = False
            np.testing.assert_array_equal(out[band], img[band])


def test_small_images_unchanged(oracle_mod):
    for beta in (1, 2, 3):
        n = 2 * beta  # one short of 2*beta + 1
        for shape in ((n, 40), (40, n), (1, 1), (n, n)):
            img = synth.random_image(*shape, seed=77)
            out, k, conv = oracle_mod.denoise(img, 10, beta, 32)
            assert k == 0 and conv
            np.testing.assert_array_equal(out, img)


def test_fixed_point_and_stop_rule(oracle_mod):
    clean, noisy = synth.noisy_image(64, 64, 0.2, synth.seed_for(9, 1))
    out, k, conv, changes = oracle_mod.denoise(noisy, 10, 1, 50, return_changes=True)
    assert conv and 0 < k < 50
    assert all(c > 0 for c in changes[:k]) and changes[k] == 0
    again, ch = oracle_mod.one_pass(out, 10, 1)
    assert ch == 0
    np.testing.assert_array_equal(again, out)
    # max_k caps the number of changing passes: m passes of one_pass.
    for m in (0, 1, 2, 3):
        o, km, cm = oracle_mod.denoise(noisy, 10, 1, m)
        ref = noisy
        for _ in range(m):
            ref, _ = oracle_mod.one_pass(ref, 10, 1)
        assert km == m and not cm
        np.testing.assert_array_equal(o, ref)


def test_smooth_noise_free_image_unchanged(oracle_mod):
    clean = synth.clean_image(128, 160, synth.seed_for(9, 2))
    out, k, conv = oracle_mod.denoise(clean, 10, 1, 32)
    assert k == 0 and conv
    np.testing.assert_array_equal(out, clean)


def test_denoising_restores_quality(oracle_mod):
    """PSNR falls as impulse density rises and denoising raises it
    (the trend of the paper's Table 2, on synthetic images)."""
    vals = []
    for d in (0.05, 0.10, 0.15, 0.20):
        clean, noisy = synth.noisy_image(96, 96, d, synth.seed_for(9, 3))
        out, k, _ = oracle_mod.denoise(noisy, 10, 1, 32)
        p_out = oracle_mod.psnr(clean, out)
        assert p_out > oracle_mod.psnr(clean, noisy) + 5
        vals.append(p_out)
    assert vals == sorted(vals, reverse=True)


def test_psnr_closed_forms(oracle_mod):
    a = np.full((10, 10), 7, dtype=np.uint8)
    assert oracle_mod.psnr(a, a) == float("inf")
    b = a.copy()
    b[3, 4] += 1  # MSE = 1/100
    assert oracle_mod.psnr(a, b) == pytest.approx(10 * math.log10(255**2 * 100), abs=1e-9)
    c = np.zeros((4, 4), np.uint8)
    d = np.full((4, 4), 255, np.uint8)  # MSE = 255^2 -> 0 dB
    assert oracle_mod.psnr(c, d) == pytest.approx(0.0, abs=1e-12)


def test_planted_mistakes_are_caught(oracle_mod, tmp_path):
    """Each plausible slip in the oracle's C (a flipped comparison, a dropped
    pix_count position, rounding instead of truncation) is caught by one of
    the pins above.  The slips are planted in copies of the oracle source
    compiled here on the CPU."""
    import ctypes
    import subprocess

    src = open(os.path.join(os.path.dirname(oracle_mod.__file__), "hgrms_oracle.c")).read()
    slips = {
        "strict_flag": ("if (flag > pix_count - 3) {\n                out", "if (flag >= pix_count - 3) {\n                out"),
        "open_upper": ("int closed = (v < ip + alpha + 1) && (v > ip - alpha);",
                       "int closed = (v < ip + alpha) && (v > ip - alpha);"),
        "pix_count_inimage": ("++pix_count; /* off-image positions are counted too */\n                    if (!in_image(i, j, rows, cols)) continue;",
                              "if (!in_image(i, j, rows, cols)) continue;\n                    ++pix_count;"),
        # (card <= 3 instead of <= 2 would change nothing: for alpha >= 1,
        # flag > pix_count - 3 already forces card <= 2.)
        "card_le_alpha": ("if (d < alpha && d > -alpha) ++card;",
                          "if (d <= alpha && d >= -alpha) ++card;"),
        "round_rms": ("out[r * cols + c] = (uint8_t)hgo_isqrt((uint32_t)(sum / flag));",
                      "out[r * cols + c] = (uint8_t)(sqrt((double)sum / flag) + 0.5);"),
    }
    goldens = [load_golden(os.path.join(GOLDEN, n)) for n in GOLDEN_FILES]
    for name, (old, new) in slips.items():
        assert old in src, name
        cfile = tmp_path / f"{name}.c"
        cfile.write_text(src.replace(old, new))
        so = tmp_path / f"{name}.so"
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", str(so), str(cfile), "-lm"])
        lib = ctypes.CDLL(str(so))
        caught = False
        for g in goldens:
            img = g["input"].copy()
            conv = ctypes.c_int(0)
            k = lib.hgo_denoise(img.ctypes.data_as(ctypes.c_void_p), img.shape[0], img.shape[1],
                                g["alpha"], g["beta"], g["max_k"], ctypes.byref(conv), None)
            if k != g["k"] or not np.array_equal(img, g["output"]):
                caught = True
                break
        assert caught, f"planted slip {name} not caught by the golden examples"
