"""The separable median networks of the dense strategy (k = 5, 7), checked on
the CPU before any kernel runs them.

* the vertical stage (one word column: the k-1 shared rows sorted, the row
  above merged in for row y, the row below for row y+1) on every 0-1 input;
* the horizontal stage (sorted columns -> g_m, g_min, g_max of eight output
  columns) on every 0-1 input whose columns are sorted, window by window:
  thresholding a sorted column gives a sorted 0-1 column, so by the 0-1
  principle this covers every input with sorted columns, which is what the
  vertical stage hands over;
* the whole lane item (vertical, transpose, horizontal, on packed pairs of
  16-bit lanes) against numpy's sort on random and tie-heavy values;
* the sliding form the 7x7 kernel runs (a carry of shared sorted columns and
  merged blocks handed from item to item) the same way, over four items;
* the generated header is the generator's current output.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_1201_3972_gb300", "csrc"))
import gen_separable as gs  # noqa: E402

KS = (5, 7)


def test_generated_header_is_current():
    with open(gs.HEADER) as fh:
        assert fh.read() == gs.emit()


@pytest.mark.parametrize("k", KS)
def test_vertical_zero_one(k):
    p, top, bot = gs.vertical_program(k)
    ops = gs.live_ops(p, [(0, *top, *bot)])
    n = k + 1
    idx = np.arange(1 << n)
    inputs = {}
    for d, kind, args in p.ops:
        if kind == "in":
            inputs[d] = ((idx >> args[0][1]) & 1).astype(bool)
    v = gs.evaluate(ops, inputs, np.logical_and, np.logical_or)
    bits = np.array([[(i >> r) & 1 for r in range(n)] for i in idx])
    want_top = np.sort(bits[:, :k], axis=1)
    want_bot = np.sort(bits[:, 1:], axis=1)
    for i in range(k):
        assert np.array_equal(v[top[i]], want_top[:, i].astype(bool)), ("top", i)
        assert np.array_equal(v[bot[i]], want_bot[:, i].astype(bool)), ("bot", i)


def _sorted_column_patterns(ncols, k):
    """Every assignment of sorted 0-1 columns (z zeros then ones, z = 0..k)
    to ncols columns, as packed bitsets: per (column, rank) a uint64 array."""
    total = (k + 1) ** ncols
    idx = np.arange(total)
    words = (total + 63) // 64
    out = {}
    for c in range(ncols):
        z = (idx // (k + 1) ** c) % (k + 1)
        for i in range(k):
            bits = np.zeros(words * 64, dtype=bool)
            bits[:total] = i >= z
            out[(c, i)] = np.packbits(bits, bitorder="little").view(np.uint64)
    return out, total


@pytest.mark.parametrize("k", KS)
def test_horizontal_zero_one_sorted_columns(k):
    R = (k - 1) // 2
    m = (k * k - 1) // 2
    p, outs = gs.horizontal_program(k)
    ins = [(d, args[0]) for d, kind, args in p.ops if kind == "in"]
    for o, med, gmn, gmx in outs:
        window = list(range(o - R, o + R + 1))
        ops = gs.live_ops(p, [(o, med, gmn, gmx)])
        # the outputs of column o read only the columns of its window
        used = {args[0][1] for d, kind, args in ops if kind == "in"}
        assert used <= set(window), (o, used)
        pats, total = _sorted_column_patterns(k, k)
        inputs = {}
        for d, (_, c, i) in ins:
            if c in window:
                inputs[d] = pats[(window.index(c), i)]
        v = gs.evaluate(ops, inputs, np.bitwise_and, np.bitwise_or)
        # count of ones in the window per pattern: sum over columns of (k - zeros)
        idx = np.arange(total)
        ones = np.zeros(total, dtype=np.int64)
        for c in range(k):
            ones += k - (idx // (k + 1) ** c) % (k + 1)

        def unpack(a):
            return np.unpackbits(a.view(np.uint8), bitorder="little")[:total].astype(bool)
        n = k * k
        assert np.array_equal(unpack(v[med]), (n - ones) <= m), ("median", o)
        assert np.array_equal(unpack(v[gmn]), ones == n), ("min", o)
        assert np.array_equal(unpack(v[gmx]), ones > 0), ("max", o)


@pytest.mark.parametrize("k", KS)
def test_item_random_values(k):
    """The whole item on 16-bit lanes packed in pairs, like the kernel."""
    p, outs = gs.item_program(k)
    ops = gs.live_ops(p, outs)
    R = (k - 1) // 2
    w0 = gs.first_word_col(k)
    nw = gs.words_per_row(k)
    rng = np.random.default_rng(k)
    trials = 64
    mask = np.uint32(0xFFFF)

    def lane_min(a, b):
        return np.minimum(a & mask, b & mask) | (np.minimum(a >> 16, b >> 16) << 16)

    def lane_max(a, b):
        return np.maximum(a & mask, b & mask) | (np.maximum(a >> 16, b >> 16) << 16)

    def lo(a, b):
        return (a & mask) | ((b & mask) << 16)

    def hi(a, b):
        return (a >> 16) | ((b >> 16) << 16)
    imgs = []
    for t in range(trials):
        top = [2, 6, 300, 65536][t % 4]
        imgs.append(rng.integers(0, top, size=(k + 1, 2 * nw)).astype(np.uint32))
    imgs = np.stack(imgs)                      # trial, row, column (from w0)
    inputs = {}
    for d, kind, args in p.ops:
        if kind == "in":
            r, w = args[0]
            inputs[d] = imgs[:, r, 2 * w] | (imgs[:, r, 2 * w + 1] << 16)
    v = gs.evaluate(ops, inputs, lane_min, lane_max, lo, hi)
    for o, med, gmn, gmx in outs:
        c0 = o - R - w0
        for half in (0, 1):
            win = imgs[:, half:half + k, c0:c0 + k].reshape(trials, -1)
            srt = np.sort(win, axis=1)
            assert np.array_equal((v[med] >> (16 * half)) & mask, srt[:, (k * k - 1) // 2]), (o, half)
            assert np.array_equal((v[gmn] >> (16 * half)) & mask, srt[:, 0])
            assert np.array_equal((v[gmx] >> (16 * half)) & mask, srt[:, -1])


@pytest.mark.parametrize("k", KS)
def test_span_random_values(k):
    """The sliding form (pre, then body item after item with the carry handed
    on) against numpy's sort for every window of four items. The kernel runs
    it for the windows gs.SLIDING names; the others are checked too."""
    p, pre, body, carry_in, carry_out, outs = gs.span_program(k)
    assert len(carry_in) == len(carry_out)
    R = (k - 1) // 2
    n = gs.NOUT[k]
    w0 = gs.first_word_col(k)
    nw = gs.words_per_row(k)
    items = 4
    rng = np.random.default_rng(100 + k)
    trials = 64
    mask = np.uint32(0xFFFF)

    def lane_min(a, b):
        return np.minimum(a & mask, b & mask) | (np.minimum(a >> 16, b >> 16) << 16)

    def lane_max(a, b):
        return np.maximum(a & mask, b & mask) | (np.maximum(a >> 16, b >> 16) << 16)

    def lo(a, b):
        return (a & mask) | ((b & mask) << 16)

    def hi(a, b):
        return (a >> 16) | ((b >> 16) << 16)
    width = n * (items - 1) + 2 * (nw + gs.LOOKAHEAD[k])  # image column 0 = x0 + w0 of the first item
    imgs = np.stack([rng.integers(0, [2, 6, 300, 65536][t % 4], size=(k + 1, width)).astype(np.uint32)
                     for t in range(trials)])

    def words(ops, x):
        got = {}
        for d, kind, args in ops:
            if kind == "in":
                r, w = args[0]
                c = x + 2 * w
                got[d] = imgs[:, r, c] | (imgs[:, r, c + 1] << 16)
        return got
    v = gs.evaluate(pre, words(pre, 0), lane_min, lane_max, lo, hi)
    carry = [v[d] for d in carry_in]
    for it in range(items):
        inputs = words(body, it * n)
        inputs.update(zip(carry_in, carry))
        v = gs.evaluate(body, inputs, lane_min, lane_max, lo, hi)
        carry = [v[d] for d in carry_out]
        for o, med, gmn, gmx, *centre in outs:
            c0 = it * n + o - R - w0                 # first window column in the image
            for half in (0, 1):
                win = imgs[:, half:half + k, c0:c0 + k].reshape(trials, -1)
                srt = np.sort(win, axis=1)
                assert np.array_equal((v[med] >> (16 * half)) & mask, srt[:, (k * k - 1) // 2]), (it, o, half)
                assert np.array_equal((v[gmn] >> (16 * half)) & mask, srt[:, 0]), (it, o, half)
                assert np.array_equal((v[gmx] >> (16 * half)) & mask, srt[:, -1]), (it, o, half)
            # the words handed to the flag test hold the centre pixel (column o of rows y, y + 1)
            # in the half the emitter picks for o's parity
            for word, row in zip(centre, (R, R + 1)):
                assert np.array_equal((v[word] >> (16 * (o & 1))) & mask, imgs[:, row, c0 + R]), (it, o, row)


def test_span_op_counts_recorded():
    """Per sliding item of 16 pixels: 456 (5x5) and 964 (7x7) min/max
    operations, against 534 and 1240 for an item computed on its own."""
    for k, want in ((5, 456), (7, 964)):
        _, _, body, _, _, _ = gs.span_program(k)
        c = gs.op_counts(body)
        assert c["min"] + c["max"] == want


def test_header_forms_match_kernel_choice():
    """The header holds the sliding form exactly for the windows the kernel's
    dense_sliding() names (k = 7), the single-item form for the others."""
    with open(gs.HEADER) as fh:
        text = fh.read()
    for k in KS:
        block = text[text.index(f"struct SepNet<{k}>"):]
        block = block[:block.index("};")]
        assert (f"kSliding = {'true' if gs.SLIDING[k] else 'false'}") in block
        assert ("static void body(" in block) == gs.SLIDING[k]
        assert ("static void run(" in block) == (not gs.SLIDING[k])
    params = open(os.path.join(ROOT, "paper_1201_3972_gb300", "csrc", "fnr_params.h")).read()
    assert "constexpr bool dense_sliding(int k) { return k == 7; }" in params
    assert [k for k in KS if gs.SLIDING[k]] == [7]


def test_op_counts_recorded():
    """Per 16-pixel item: the 5x5 network stays at 534 min/max operations and
    the 7x7 one at 1240 (the figures the design's cost model uses)."""
    for k, want in ((5, 534), (7, 1240)):
        p, outs = gs.item_program(k)
        c = gs.op_counts(gs.live_ops(p, outs))
        assert c["min"] + c["max"] == want
