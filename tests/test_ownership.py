"""CPU check of the ownership rule the list passes use to evaluate every
pixel that can change exactly once, restated with the same bit masks as the
(changed pixel, window row) tasks of the list-pass loop.

A pixel q can change in a pass only if some pixel of its window changed in
the previous pass (locality of change, from Algorithm 2).  Task (p, dy), for
a changed pixel p, handles the pixels q = p + (dy, dx), |dx| <= beta; it
owns q when no changed pixel of q's window precedes p in raster order.  With
bits[r] = the changes in row qy - beta + r, columns px - 2 beta ..
px + 2 beta (bit j: column px - 2 beta + j), q's window columns are bits
dx + beta .. dx + 3 beta; its rows above p's must hold none of them and p's
own row none left of p (bits below 2 beta).  Brute force over random change
sets: every interior pixel with a change in its window has exactly one
owner, and no other pixel has one."""
import numpy as np
import pytest


def row_bits(bm, gy, start, nbits):
    """Bits [start, start + nbits) of bitmap row gy (0 outside the image)."""
    cols = bm.shape[1]
    out = 0
    for j in range(nbits):
        c = start + j
        if 0 <= c < cols and bm[gy, c]:
            out |= 1 << j
    return out


def owned(bm, B, py, px, dy):
    """The dx (as a set) whose pixel q = (py + dy, px + dx) task (p, dy) owns."""
    rows, cols = bm.shape
    W = 2 * B + 1
    qy = py + dy
    if not (B <= qy < rows - B):
        return set()
    before = 0
    for r in range(2 * B + 1):
        gy = qy - B + r
        if gy < py:
            before |= row_bits(bm, gy, px - 2 * B, 4 * B + 1)
        elif gy == py:
            before |= row_bits(bm, gy, px - 2 * B, 4 * B + 1) & ((1 << (2 * B)) - 1)
    out = set()
    for dx in range(-B, B + 1):
        qx = px + dx
        wm = ((1 << W) - 1) << (dx + B)
        if B <= qx < cols - B and (before & wm) == 0:
            out.add(dx)
    return out


@pytest.mark.parametrize("beta", [1, 2, 3, 7])
def test_every_candidate_pixel_has_one_owner(beta):
    rng = np.random.default_rng(1306 + beta)
    for trial in range(30):
        rows = int(rng.integers(2 * beta + 1, 2 * beta + 25))
        cols = int(rng.integers(2 * beta + 1, 2 * beta + 25))
        bm = rng.random((rows, cols)) < rng.choice([0.02, 0.1, 0.3, 0.7])
        count = np.zeros((rows, cols), dtype=int)
        for py, px in zip(*np.nonzero(bm)):
            for dy in range(-beta, beta + 1):
                for dx in owned(bm, beta, int(py), int(px), dy):
                    count[py + dy, px + dx] += 1
        for y in range(rows):
            for x in range(cols):
                interior = beta <= y < rows - beta and beta <= x < cols - beta
                near = bm[max(0, y - beta):y + beta + 1, max(0, x - beta):x + beta + 1].any()
                assert count[y, x] == (1 if interior and near else 0), (beta, trial, y, x)


def owned_beta1(bm, py, px):
    """beta 1, one task per changed pixel p: the (dy, dx) of p's 3 x 3 window
    that p owns, with the kernel's masks.  rb[r] = the changes of row
    py - 2 + r (r = 0, 1, 2: the rows up to p's), columns px - 2 .. (bit j:
    column px - 2 + j); q = p + (dy, dx) has window rows r = dy + 1 .. dy + 3
    and window columns bits dx + 1 .. dx + 3: rows above p's (r < 2) must
    hold none of them, p's row (r = 2) none left of p (bits dx + 1 .. 1)."""
    rows, cols = bm.shape
    rb = [row_bits(bm, py - 2 + r, px - 2, 32) if py - 2 + r >= 0 else 0 for r in range(3)]
    out = set()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            qy, qx = py + dy, px + dx
            if not (1 <= qy < rows - 1 and 1 <= qx < cols - 1):
                continue
            owner = True
            for r in range(dy + 1, dy + 4):
                if r < 2 and rb[r] & (7 << (dx + 1)):
                    owner = False
                if r == 2 and rb[2] & 3 & ~((1 << (dx + 1)) - 1):
                    owner = False
            if owner:
                out.add((dy, dx))
    return out


def test_beta1_per_changed_pixel_tasks_one_owner():
    rng = np.random.default_rng(2013)
    for trial in range(60):
        rows = int(rng.integers(3, 30))
        cols = int(rng.integers(3, 30))
        bm = rng.random((rows, cols)) < rng.choice([0.02, 0.1, 0.3, 0.7, 1.0])
        count = np.zeros((rows, cols), dtype=int)
        for py, px in zip(*np.nonzero(bm)):
            for dy, dx in owned_beta1(bm, int(py), int(px)):
                count[py + dy, px + dx] += 1
        for y in range(rows):
            for x in range(cols):
                interior = 1 <= y < rows - 1 and 1 <= x < cols - 1
                near = bm[max(0, y - 1):y + 2, max(0, x - 1):x + 2].any()
                assert count[y, x] == (1 if interior and near else 0), (trial, y, x)
