"""Pins for the CPU oracle, checked against things other than the oracle itself.

* hand-worked fixtures in tests/golden/ (derived from Sec. 3.3-3.4 by hand);
* library routines the method reduces to: numpy's sort for the introsort
  (Sec. 3.4, Eq. 4), and scipy.ndimage's textbook minimum, maximum and median
  filters (replicate border) for the window extremes (Eq. 3a/3b) and the
  median g_m of S_xy;
* brute force over every binary 4x4 and every ternary 3x4 frame;
* invariants that hold for any frame: unflagged pixels untouched, output
  inside [g_min, g_max], constant frames fixed, isolated impulses restored,
  salt-and-pepper always detected, commuting with monotone maps, with
  transpose and flips, and the flagged count.
Finally each pin set is run against deliberately wrong variants of the
method (zero border, strict ties, centre left out, wrong rank, recursive
raster pass, transposed clamp) to show that every such mistake fails one.
"""
import itertools

import numpy as np
import pytest
import scipy.ndimage as nd

from _golden import all_fixtures
from paper_1201_3972_gb300 import synth

KS = (3, 5, 7, 9, 11, 13, 15, 17, 19, 21)


def library_fnr(a, k):
    """FNR expressed through scipy's textbook filters: flagged pixels are those
    equal to the k x k min or max filter; they take the k x k median filter;
    the rest keep their value. Replicate border is scipy's mode='nearest'."""
    mn = nd.minimum_filter(a, size=k, mode="nearest")
    mx = nd.maximum_filter(a, size=k, mode="nearest")
    md = nd.median_filter(a, size=k, mode="nearest")
    flag = (a == mn) | (a == mx)
    return np.where(flag, md, a).astype(a.dtype), int(flag.sum())


def rand_frame(rng, H, W, dtype, style):
    maxv = synth.MAXV[dtype]
    npdt = synth.NP_DTYPE[dtype]
    if style == "uniform":
        return rng.integers(0, maxv + 1, size=(H, W)).astype(npdt)
    if style == "few":       # heavy ties
        vals = rng.choice([0, 1, maxv // 2, maxv], size=(H, W))
        return vals.astype(npdt)
    if style == "smooth_sp":
        base = (np.add.outer(np.arange(H), np.arange(W)) * 3 + 40) % (maxv + 1)
        f = base.astype(npdt)
        return synth.add_impulses(rng, f, 0.2, maxv, "sp")
    raise ValueError(style)


# ---------------------------------------------------------------------------
# introsort
# ---------------------------------------------------------------------------
def _sort_cases(rng):
    yield np.zeros(0, np.uint32)
    yield np.array([7], np.uint32)
    for n in (2, 3, 5, 9, 16, 17, 25, 49, 81, 100, 225, 441, 700):
        yield rng.integers(0, 2 ** 16, n).astype(np.uint32)
        yield rng.integers(0, 3, n).astype(np.uint32)                 # duplicates
        yield np.arange(n, dtype=np.uint32)                            # sorted
        yield np.arange(n, dtype=np.uint32)[::-1].copy()               # reversed
        yield np.full(n, 5, np.uint32)                                 # constant
        h = np.arange(n // 2 + 1, dtype=np.uint32)
        yield np.concatenate([h, h[::-1]])[:n].copy()                  # organ pipe


@pytest.mark.parametrize("depth", [-1, 0, 1, 3, 1000])
def test_introsort_matches_numpy_sort(oracle_mod, depth):
    rng = np.random.default_rng(1)
    for a in _sort_cases(rng):
        got = oracle_mod.introsort(a, depth)
        np.testing.assert_array_equal(got, np.sort(a, kind="stable"))


def test_median_rank_matches_numpy_partition(oracle_mod):
    rng = np.random.default_rng(2)
    for k in KS:
        n = k * k
        for _ in range(20):
            w = rng.integers(0, 300, n)
            assert oracle_mod.median(w) == int(np.partition(w, (n - 1) // 2)[(n - 1) // 2])


# ---------------------------------------------------------------------------
# hand-worked fixtures
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fx", all_fixtures(), ids=lambda f: f["name"])
def test_golden_fixture(oracle_mod, fx):
    if fx["detector"] == "directional":
        out, flagged = oracle_mod.fnr_directional(fx["input"], fx["k"])
    else:
        out, flagged = oracle_mod.fnr(fx["input"], fx["k"])
    np.testing.assert_array_equal(out, fx["output"])
    assert flagged == fx["flagged"]


def test_golden_fixtures_present():
    assert len(all_fixtures("extreme")) >= 6
    assert len(all_fixtures("directional")) >= 3


# ---------------------------------------------------------------------------
# library filters
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [synth.U8, synth.U16, synth.U14])
@pytest.mark.parametrize("style", ["uniform", "few", "smooth_sp"])
def test_matches_library_filters(oracle_mod, dtype, style):
    rng = np.random.default_rng(100 + dtype * 10 + len(style))
    shapes = [(1, 1), (1, 7), (7, 1), (2, 3), (5, 5), (9, 16), (16, 9), (13, 17), (23, 20)]
    for H, W in shapes:
        for k in KS:
            a = rand_frame(rng, H, W, dtype, style)
            want, wf = library_fnr(a, k)
            got, gf = oracle_mod.fnr(a, k)
            np.testing.assert_array_equal(got, want, err_msg=f"{H}x{W} k={k}")
            assert gf == wf


def test_matches_library_filters_on_synthetic_frames(oracle_mod):
    specs = [s for s in synth.workload_sweep_u14()[:3]] + synth.workload_single_u8()
    for s in specs:
        f = s.make()[:48, :64].copy()
        for k in (3, 5, 7, 9, 15):
            want, wf = library_fnr(f, k)
            got, gf = oracle_mod.fnr(f, k)
            np.testing.assert_array_equal(got, want)
            assert gf == wf


@pytest.mark.parametrize("dtype", [synth.U8, synth.U16])
def test_median_filter_matches_library(oracle_mod, dtype):
    """The MF baseline (every pixel takes its window median) equals scipy's
    median filter with a replicated border."""
    rng = np.random.default_rng(11 + dtype)
    for H, W in ((1, 1), (3, 9), (13, 17), (20, 23)):
        for k in (3, 5, 7, 9, 15, 21):
            for style in ("uniform", "few"):
                a = rand_frame(rng, H, W, dtype, style)
                got, n = oracle_mod.median_filter(a, k)
                np.testing.assert_array_equal(got, nd.median_filter(a, size=k, mode="nearest"))
                assert n == a.size


def test_iterative_passes_are_compositions(oracle_mod):
    """Two and three passes equal the library-filter definition applied
    repeatedly, with the flagged count of each pass."""
    rng = np.random.default_rng(12)
    a = rand_frame(rng, 30, 41, synth.U8, "smooth_sp")
    for k in (3, 5):
        cur, want_counts = a, []
        for _ in range(3):
            cur, c = library_fnr(cur, k)
            want_counts.append(c)
        got, counts = oracle_mod.fnr_passes(a, k, 3)
        np.testing.assert_array_equal(got, cur)
        assert counts == want_counts
        got2, counts2 = oracle_mod.fnr_passes(a, k, 3, threads=4)
        np.testing.assert_array_equal(got2, cur)
        assert counts2 == counts


@pytest.mark.parametrize("border,mode", [("replicate", "nearest"), ("mirror", "mirror"), ("zero", "constant")])
def test_border_readings_match_library(oracle_mod, border, mode):
    """Each border reading equals scipy's filters with the same extension:
    nearest (replicate), mirror (d c b | a b c d | c b a) and constant 0,
    including windows wider than the frame."""
    rng = np.random.default_rng(21)
    for H, W in ((1, 1), (1, 6), (2, 3), (4, 9), (11, 7), (16, 23)):
        for k in (3, 5, 7, 9, 21):
            for style in ("uniform", "few"):
                a = rand_frame(rng, H, W, synth.U8, style)
                mn = nd.minimum_filter(a, size=k, mode=mode, cval=0)
                mx = nd.maximum_filter(a, size=k, mode=mode, cval=0)
                md = nd.median_filter(a, size=k, mode=mode, cval=0)
                flag = (a == mn) | (a == mx)
                got, f = oracle_mod.fnr_border(a, k, border)
                np.testing.assert_array_equal(got, np.where(flag, md, a).astype(a.dtype), err_msg=f"{H}x{W} k{k}")
                assert f == int(flag.sum())


def test_pitched_input(oracle_mod):
    rng = np.random.default_rng(5)
    a = rng.integers(0, 65536, (11, 13)).astype(np.uint16)
    buf, view = synth.pitched_copy(a, 21, 3)
    got, gf = oracle_mod.fnr(view, 5)
    want, wf = library_fnr(a, 5)
    np.testing.assert_array_equal(got, want)
    assert gf == wf


# ---------------------------------------------------------------------------
# exhaustive small frames
# ---------------------------------------------------------------------------
def _all_frames(values, H, W):
    vals = np.array(values)
    idx = np.array(list(itertools.product(range(len(values)), repeat=H * W)), dtype=np.int64)
    return vals[idx].reshape(-1, H, W)


def _stack_library_fnr(frames, k):
    size = (1, k, k)
    mn = nd.minimum_filter(frames, size=size, mode="nearest")
    mx = nd.maximum_filter(frames, size=size, mode="nearest")
    md = nd.median_filter(frames, size=size, mode="nearest")
    flag = (frames == mn) | (frames == mx)
    return np.where(flag, md, frames).astype(frames.dtype), int(flag.sum())


@pytest.mark.parametrize("values", [(0, 1), (3, 200)])
def test_exhaustive_binary_4x4_k3(oracle_mod, values):
    frames = _all_frames(values, 4, 4).astype(np.uint8)
    assert frames.shape[0] == 2 ** 16
    got, gf = oracle_mod.fnr_stack(frames, 3)
    want, wf = _stack_library_fnr(frames, 3)
    np.testing.assert_array_equal(got, want)
    assert gf == wf


def test_exhaustive_ternary_3x4_k3(oracle_mod):
    frames = _all_frames((0, 9, 65535), 3, 4).astype(np.uint16)
    assert frames.shape[0] == 3 ** 12
    got, gf = oracle_mod.fnr_stack(frames, 3)
    want, wf = _stack_library_fnr(frames, 3)
    np.testing.assert_array_equal(got, want)
    assert gf == wf


@pytest.mark.parametrize("k", [5, 7, 21])
def test_exhaustive_ternary_2x3_large_window(oracle_mod, k):
    frames = _all_frames((1, 2, 3), 2, 3).astype(np.uint8)
    got, gf = oracle_mod.fnr_stack(frames, k)
    want, wf = _stack_library_fnr(frames, k)
    np.testing.assert_array_equal(got, want)
    assert gf == wf


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def _frames_for_invariants():
    rng = np.random.default_rng(9)
    out = []
    for s in (synth.workload_single_u8()[0], synth.workload_sweep_u14()[7],
              synth.workload_large_k()[0]):
        out.append(s.make()[:40, :56].copy())
    out.append(rand_frame(rng, 31, 29, synth.U16, "uniform"))
    out.append(rand_frame(rng, 17, 33, synth.U8, "few"))
    return out


@pytest.mark.parametrize("k", [3, 5, 7, 9, 15, 21])
def test_invariants(oracle_mod, k):
    for a in _frames_for_invariants():
        out, flagged = oracle_mod.fnr(a, k)
        mn = nd.minimum_filter(a, size=k, mode="nearest")
        mx = nd.maximum_filter(a, size=k, mode="nearest")
        noisy = (a == mn) | (a == mx)
        # 1. signal pixels are bit-identical
        np.testing.assert_array_equal(out[~noisy], a[~noisy])
        # 2. every output lies within its window's extremes
        assert np.all(out >= mn) and np.all(out <= mx)
        # 8. flagged count = pixels equal to a window extreme
        assert flagged == int(noisy.sum())
        # 6. strictly increasing maps commute
        if a.dtype == np.uint8:
            up = a.astype(np.uint16) * 2 + 3
            o2, f2 = oracle_mod.fnr(up, k)
            np.testing.assert_array_equal(o2, out.astype(np.uint16) * 2 + 3)
            assert f2 == flagged
        maxv = 255 if a.dtype == np.uint8 else 65535
        inv = (maxv - a.astype(np.int64)).astype(a.dtype)
        o3, f3 = oracle_mod.fnr(inv, k)
        np.testing.assert_array_equal(o3, (maxv - out.astype(np.int64)).astype(a.dtype))
        assert f3 == flagged
        # 7. transpose and flips commute
        for op in (np.transpose, np.fliplr, np.flipud):
            o4, f4 = oracle_mod.fnr(np.ascontiguousarray(op(a)), k)
            np.testing.assert_array_equal(o4, op(out))
            assert f4 == flagged


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("dtype", [synth.U8, synth.U14])
def test_constant_frame_is_fixed_point(oracle_mod, k, dtype):
    maxv = synth.MAXV[dtype]
    for c in (0, 1, maxv // 3, maxv):
        a = np.full((19, 23), c, dtype=synth.NP_DTYPE[dtype])
        out, flagged = oracle_mod.fnr(a, k)
        np.testing.assert_array_equal(out, a)
        assert flagged == a.size          # every pixel ties with both extremes


@pytest.mark.parametrize("k", [3, 5, 7, 9, 15, 21])
def test_sparse_salt_and_pepper_fully_restored(oracle_mod, k):
    """Isolated impulses on a constant background c: every window holds at most
    m zeros and m MAXV values, so each median is c and the frame is restored."""
    rng = np.random.default_rng(k)
    for dtype in (synth.U8, synth.U14):
        maxv = synth.MAXV[dtype]
        c = maxv // 2 + 1
        H, W = 3 * k + 5, 4 * k + 3
        a = np.full((H, W), c, dtype=synth.NP_DTYPE[dtype])
        ys = np.arange(0, H, k + 1)
        xs = np.arange(0, W, k + 1)
        for y in ys:
            for x in xs:
                a[y, x] = 0 if rng.random() < 0.5 else maxv
        out, flagged = oracle_mod.fnr(a, k)
        np.testing.assert_array_equal(out, np.full_like(a, c))
        assert flagged >= len(ys) * len(xs)


@pytest.mark.parametrize("k", [3, 5, 7, 9])
def test_salt_and_pepper_recall_is_total(oracle_mod, k):
    """A 0 or MAXV impulse is always an extreme of its window, so it is always
    flagged: the count is at least the number of extreme-valued pixels and the
    output at those pixels is the window median."""
    for s in synth.workload_sweep_u14()[::3]:
        a = s.make()[:64, :64].copy()
        maxv = synth.MAXV[s.dtype]
        imp = (a == 0) | (a == maxv)
        out, flagged = oracle_mod.fnr(a, k)
        md = nd.median_filter(a, size=k, mode="nearest")
        np.testing.assert_array_equal(out[imp], md[imp])
        assert flagged >= int(imp.sum())


@pytest.mark.parametrize("k", [3, 7, 15])
def test_multithreaded_equals_single(oracle_mod, k):
    a = synth.workload_sweep_u14()[4].make()
    o1, f1 = oracle_mod.fnr(a[:100], k)
    for t in (1, 2, 3, 8):
        o2, f2 = oracle_mod.fnr_mt(a[:100], k, t)
        np.testing.assert_array_equal(o1, o2)
        assert f1 == f2


def test_bad_arguments_rejected(oracle_mod):
    a = np.zeros((4, 4), np.uint8)
    for k in (0, 2, 4, -1):
        with pytest.raises(ValueError):
            oracle_mod.fnr(a, k)


# ---------------------------------------------------------------------------
# the pins catch plausible mistakes
# ---------------------------------------------------------------------------
def slow_fnr(a, k, border="nearest", strict=False, exclude_centre=False, rank_shift=0,
             recursive=False, swap_clamp=False):
    """Slow Python FNR with switches that introduce one mistake each."""
    H, W = a.shape
    r = (k - 1) // 2
    src = a.astype(np.int64)
    out = src.copy()
    flagged = 0
    for y in range(H):
        for x in range(W):
            base = out if recursive else src
            w = []
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    yy, xx = y + dy, x + dx
                    if border == "zero" and not (0 <= yy < H and 0 <= xx < W):
                        w.append(0)
                        continue
                    if swap_clamp:            # clamps rows by W and columns by H
                        yy = min(max(yy, 0), W - 1)
                        xx = min(max(xx, 0), H - 1)
                    yy = min(max(yy, 0), H - 1)
                    xx = min(max(xx, 0), W - 1)
                    w.append(int(base[yy, xx]))
            c = int(src[y, x])
            lo, hi = min(w), max(w)
            if strict:
                noisy = (c == lo and w.count(lo) == 1) or (c == hi and w.count(hi) == 1)
            else:
                noisy = c == lo or c == hi
            if noisy:
                ww = list(w)
                if exclude_centre:
                    ww.pop(len(ww) // 2)
                ww.sort()
                out[y, x] = ww[min(len(ww) - 1, (len(ww) - 1) // 2 + rank_shift)]
                flagged += 1
    return out.astype(a.dtype), flagged


def _pins_pass(impl):
    """Run the golden and library pins against ``impl``; False at first failure."""
    for fx in all_fixtures("extreme"):
        o, f = impl(fx["input"], fx["k"])
        if not np.array_equal(o, fx["output"]) or f != fx["flagged"]:
            return False
    rng = np.random.default_rng(77)
    for H, W, k in ((6, 9, 3), (9, 5, 5), (7, 7, 3)):
        a = rand_frame(rng, H, W, synth.U8, "few")
        o, f = impl(a, k)
        w, wf = library_fnr(a, k)
        if not np.array_equal(o, w) or f != wf:
            return False
    return True


def test_pin_harness_accepts_correct_method():
    assert _pins_pass(slow_fnr)


@pytest.mark.parametrize("mutation", [
    dict(border="zero"), dict(strict=True), dict(exclude_centre=True), dict(rank_shift=1),
    dict(recursive=True), dict(swap_clamp=True)], ids=str)
def test_pins_catch_mutation(mutation):
    assert not _pins_pass(lambda a, k: slow_fnr(a, k, **mutation))


def test_detail_retention_metric_on_oracle_outputs(oracle_mod):
    """The retention metric: the unfiltered pre-impulse frame keeps every
    structure pixel; the oracle's FNR and median filter give fractions in
    [0, 1]; the structure mask covers the inserted lines and targets."""
    from paper_1201_3972_gb300 import quality, synth
    noisy, pre, mask = synth.make_frame_parts(96, 128, synth.U14, 77, 8.0, 0.10, "sp", True)
    assert 96 * 2 + 96 + 96 <= mask.sum() <= 128 * 2 + 96 * 2 + 16 * 4
    assert np.array_equal(noisy, synth.make_frame(96, 128, synth.U14, 77, 8.0, 0.10, "sp", True))
    full = quality.retention(pre, pre, noisy, mask, 16383)
    assert full["kept"] == 1.0 and full["psnr"] == float("inf") and full["pixels"] > 0
    for out in (oracle_mod.fnr(noisy, 3)[0], oracle_mod.median_filter(noisy, 3)[0]):
        r = quality.retention(out, pre, noisy, mask, 16383)
        assert 0.0 <= r["kept"] <= 1.0
