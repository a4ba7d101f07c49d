"""Pins for the oracle's directional detector, an option beside Eq. 3a/3b.

Fig. 1 (its image is missing) compares the centre of a 3x3 window with its
two neighbours along each direction; Sec. 3 rests on the gray level of a
signal pixel varying monotonically over an object's surface. The reading
pinned here: p(x, y) is a signal pixel iff along at least one of the four
lines through it (horizontal, vertical, the two diagonals) g(x, y) lies
strictly between its two neighbours at distance one; a noisy pixel takes the
median of its k x k window (Sec. 3.4). What fixes it, besides the oracle:

* hand-worked fixtures in tests/golden/dir_*.txt;
* two-valued frames: no value lies strictly between two values of the frame,
  so every pixel is noisy and the result is scipy's median filter, for each
  border reading;
* bilinear ramps g = c + a y + b x (a, b > 0): every pixel lies strictly
  between its neighbours along a line, except the frame's minimum and maximum
  corners, so exactly those two are noisy;
* a pixel equal to its 3 x 3 minimum or maximum (Eq. 3 with k = 3) lies
  strictly between no two of its neighbours, so it is noisy here too; noisy
  pixels take scipy's k x k median and the others keep their value;
* symmetries: transpose and flips map the four lines onto each other, and
  strictly increasing maps and v -> MAXV - v keep "strictly between".
Each pin set is then run against wrong variants of the detector (diagonal
ends paired wrongly, betweenness not strict, a line left out, noisy when any
line breaks instead of all, neighbours at distance r, a 3 x 3 median for
every k) to show that every such mistake fails one.
"""
import numpy as np
import pytest
import scipy.ndimage as nd

from _golden import all_fixtures
from paper_1201_3972_gb300 import synth

SCIPY_MODE = {"replicate": "nearest", "mirror": "mirror", "zero": "constant"}

# one end of each line through the centre; the other end is the opposite offset
LINES = (((0, -1), (0, 1)), ((-1, 0), (1, 0)), ((-1, -1), (1, 1)), ((-1, 1), (1, -1)))


def slow_directional(a, k, border="replicate", pair_swap=False, nonstrict=False, three_lines=False,
                     any_line=False, far=False, small_window=False):
    """Slow Python form of the reading, with switches that plant one mistake each."""
    H, W = a.shape
    r = (k - 1) // 2
    src = a.astype(np.int64)

    def idx(i, n):
        if 0 <= i < n:
            return i
        if border == "zero":
            return None
        if border == "mirror":
            if n == 1:
                return 0
            period = 2 * (n - 1)
            j = i % period
            return j if j < n else period - j
        return min(max(i, 0), n - 1)

    def px(y, x):
        yy, xx = idx(y, H), idx(x, W)
        return 0 if yy is None or xx is None else int(src[yy, xx])

    lines = LINES
    if pair_swap:
        lines = (LINES[0], LINES[1], ((-1, -1), (-1, 1)), ((1, 1), (1, -1)))
    if three_lines:
        lines = LINES[:3]
    dist = r if far else 1
    wr = 1 if small_window else r
    out = src.copy()
    flagged = 0
    for y in range(H):
        for x in range(W):
            g = int(src[y, x])
            mono = []
            for (u, v) in lines:
                p = px(y + u[0] * dist, x + u[1] * dist)
                q = px(y + v[0] * dist, x + v[1] * dist)
                lo, hi = min(p, q), max(p, q)
                mono.append(lo <= g <= hi if nonstrict else lo < g < hi)
            noisy = (not all(mono)) if any_line else (not any(mono))
            if noisy:
                w = sorted(px(y + dy, x + dx) for dy in range(-wr, wr + 1) for dx in range(-wr, wr + 1))
                out[y, x] = w[(len(w) - 1) // 2]
                flagged += 1
    return out.astype(a.dtype), flagged


def two_valued(rng, H, W, lo, hi, npdt):
    return np.where(rng.random((H, W)) < 0.5, lo, hi).astype(npdt)


def ramp(H, W, a, b, c=7):
    return (c + a * np.arange(H)[:, None] + b * np.arange(W)[None, :]).astype(np.uint16)


def check_two_valued(impl, rng, k, border, H, W, npdt=np.uint8):
    lo = 0 if border == "zero" else 3   # with a zero border, outside pixels read as one of the two values
    a = two_valued(rng, H, W, lo, 200, npdt)
    out, f = impl(a, k, border)
    want = nd.median_filter(a, size=k, mode=SCIPY_MODE[border], cval=0)
    return np.array_equal(out, want) and f == a.size


def check_ramp(impl, H, W, a, b, k):
    g = ramp(H, W, a, b)
    out, f = impl(g, k, "replicate")
    med = nd.median_filter(g, size=k, mode="nearest")
    want = g.copy()
    for (y, x) in ((0, 0), (H - 1, W - 1)):
        want[y, x] = med[y, x]
    return f == 2 and np.array_equal(out, want)


def check_against_eq3(impl, a, k):
    """Eq. 3's k = 3 extremes are noisy here too; outputs are the pixel or its k x k median."""
    out, f = impl(a, k, "replicate")
    ext = (a == nd.minimum_filter(a, size=3, mode="nearest")) | (a == nd.maximum_filter(a, size=3, mode="nearest"))
    med = nd.median_filter(a, size=k, mode="nearest")
    changed = out != a
    return (np.array_equal(out[ext], med[ext]) and np.array_equal(out[changed], med[changed])
            and int(ext.sum()) <= f <= a.size)


def check_symmetries(impl, a, k):
    out, f = impl(a, k, "replicate")
    for op in (np.transpose, np.fliplr, np.flipud):
        o2, f2 = impl(np.ascontiguousarray(op(a)), k, "replicate")
        if f2 != f or not np.array_equal(o2, op(out)):
            return False
    maxv = 255 if a.dtype == np.uint8 else 65535
    o3, f3 = impl((maxv - a.astype(np.int64)).astype(a.dtype), k, "replicate")
    if f3 != f or not np.array_equal(o3, (maxv - out.astype(np.int64)).astype(a.dtype)):
        return False
    if a.dtype == np.uint8:
        o4, f4 = impl(a.astype(np.uint16) * 2 + 3, k, "replicate")
        if f4 != f or not np.array_equal(o4, out.astype(np.uint16) * 2 + 3):
            return False
    return True


def _few_valued(rng, H, W):
    return rng.choice(np.array([0, 40, 41, 120, 255], np.uint8), size=(H, W))


def _dir_pins_pass(impl):
    """Every pin on small cases; False at the first failure."""
    for fx in all_fixtures("directional"):
        o, f = impl(fx["input"], fx["k"], "replicate")
        if not np.array_equal(o, fx["output"]) or f != fx["flagged"]:
            return False
    rng = np.random.default_rng(5)
    for border in ("replicate", "mirror", "zero"):
        for k in (3, 5):
            if not check_two_valued(impl, rng, k, border, 7, 9):
                return False
    for (H, W, a, b) in ((5, 7, 3, 5), (6, 4, 4, 4), (4, 6, 7, 1)):
        for k in (3, 5):
            if not check_ramp(impl, H, W, a, b, k):
                return False
    for (H, W, k) in ((8, 9, 3), (7, 6, 5)):
        f = _few_valued(rng, H, W)
        u = rng.integers(0, 256, (H, W)).astype(np.uint8)
        for a in (f, u):
            if not check_against_eq3(impl, a, k) or not check_symmetries(impl, a, k):
                return False
    return True


@pytest.fixture(scope="module")
def dir_impl(oracle_mod):
    return lambda a, k, border: oracle_mod.fnr_directional(a, k, border)


def test_oracle_passes_every_pin(dir_impl):
    assert _dir_pins_pass(dir_impl)


def test_slow_form_passes_every_pin():
    assert _dir_pins_pass(slow_directional)


@pytest.mark.parametrize("mutation", [
    dict(pair_swap=True), dict(nonstrict=True), dict(three_lines=True), dict(any_line=True), dict(far=True),
    dict(small_window=True)], ids=str)
def test_pins_catch_mutation(mutation):
    assert not _dir_pins_pass(lambda a, k, border: slow_directional(a, k, border, **mutation))


# the oracle over wider ranges than the mutation harness needs
@pytest.mark.parametrize("border", ["replicate", "mirror", "zero"])
@pytest.mark.parametrize("k", [3, 5, 7, 9, 15, 21])
def test_two_valued_frames_are_the_median_filter(dir_impl, border, k):
    rng = np.random.default_rng(k)
    for (H, W) in ((1, 1), (1, 13), (11, 1), (17, 23)):
        for npdt in (np.uint8, np.uint16):
            assert check_two_valued(dir_impl, rng, k, border, H, W, npdt)


@pytest.mark.parametrize("k", [3, 5, 9, 21])
def test_ramps_flag_only_the_frame_extremes(dir_impl, k):
    for (H, W) in ((2, 2), (2, 9), (9, 2), (13, 17)):
        for (a, b) in ((1, 1), (3, 5), (50, 1)):
            assert check_ramp(dir_impl, H, W, a, b, k)


@pytest.mark.parametrize("k", [3, 5, 7, 9, 15, 21])
def test_eq3_extremes_are_noisy_and_symmetries_hold(dir_impl, k):
    rng = np.random.default_rng(100 + k)
    frames = [_few_valued(rng, 19, 23), rng.integers(0, 256, (21, 18)).astype(np.uint8),
              synth.make_frame(24, 40, synth.U14, 3, 8.0, 0.2)]
    for a in frames:
        assert check_against_eq3(dir_impl, a, k)
        assert check_symmetries(dir_impl, a, k)


def test_directional_matches_slow_form_on_synthetic_frames(dir_impl):
    """The C oracle and the slow form agree on noisy synthetic frames, each border."""
    for border in ("replicate", "mirror", "zero"):
        for k in (3, 5):
            a = synth.make_frame(14, 19, synth.U14, 11 + k, 8.0, 0.2)
            o1, f1 = dir_impl(a, k, border)
            o2, f2 = slow_directional(a, k, border)
            assert f1 == f2 and np.array_equal(o1, o2)
