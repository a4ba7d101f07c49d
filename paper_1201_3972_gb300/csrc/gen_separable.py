#!/usr/bin/env python3
"""Generate the separable median networks of the dense strategy (k = 5, 7).

The dense strategy takes the window median g_m (Sec. 3.4) of EVERY pixel and
keeps it only where the detector flags the pixel, so that the work of
overlapping windows can be shared. Any exact selection gives the same g_m;
this one is a fixed min/max network, so it is branch-free and integer-exact.

One lane item is a pair of output rows (y, y+1) times NOUT[k] output columns
x0 .. x0+NOUT[k]-1. The network reads the item's k+1 stage rows as 32-bit words of two
16-bit pixels (columns c, c+1: "x-packed") and works in three stages:

1. Vertical (per x-packed word column): the k-1 rows that the windows of
   rows y and y+1 share are sorted once (an optimal small sorting network),
   then the row above is merged in for row y and the row below for row y+1
   (Batcher's odd-even merge). Each word holds two columns, so one network
   sorts both.
2. Transpose: byte permutes turn the two sorted columns of a word, for rows y
   and y+1, into two words that each hold one column for both rows
   ("row-packed"): from here on every operation serves the two output rows
   at once, and neighbouring columns are separate words, so windows that
   overlap horizontally can share work column by column.
3. Horizontal: sorted columns are merged (Batcher's odd-even merge, pruned to
   the ranks used and with comparisons that the sortedness of the inputs
   decides removed) into blocks shared by neighbouring windows. The windows
   of outputs x and x+1 share k-1 columns; the ranks m-k .. m of that shared
   union S (m = (k*k-1)/2) are computed once, and each output adds its one
   remaining sorted column C:
       g_m = min(S[m], max(S[m-1], C[0]), ..., max(S[m-k], C[k-1]))
   (the element of rank m of S u C). k = 5: S = M2 u M2', M2 the merge of two
   neighbouring columns, each M2 shared by two pairs. k = 7: S is a 4-column
   block B4 (shared by two pairs) merged with one M2; only the ranks 17..24
   of S are needed, hence only the ranks 3..24 of B4.
   g_min and g_max of every window (Eq. 3a/3b) come out of the same merges.
The construction follows the idea of separable sorting networks (A. Adams,
"Fast median filters using separable sorting networks", ACM TOG 40(4),
2021): sort columns once, share merges between overlapping windows.

A value that is never read is not computed (dead-code pruning); a min/max
pair of the same operands is emitted as a compare-exchange so that part of
the maxima can go to the FMA pipe (PackedOp::cmax).

Sliding form (the 7x7, SLIDING[k]): neighbouring items of a row pair share
sorted columns and merged blocks, so a lane filters a span of items and
hands these on in registers. span_program() builds the program of two
neighbouring items, takes the values of the left one that the right one
reads as the carry (after moving transpositions whose inputs the left item
holds to the left item when that shrinks it), pairs each carried value with
its counterpart one item further right by structure (the same function of
the same relative words), and returns `pre` (the carry of a span's first
item) and `body` (one item from its carry, leaving the next item's carry).
Each output of the sliding form also names the input words of its centre
pixels, so the flag test needs no second read of the stage.

Run this file to rewrite ``fnr_separable.cuh``; the tests import it to check
the vertical network exhaustively, the horizontal network over every 0-1
input with sorted columns (which by the 0-1 principle covers every input),
the whole item and the sliding form (pre, then bodies with the carry handed
on) on random values, and that the header is current.
"""
from __future__ import annotations

import os
from typing import Dict, List, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "fnr_separable.cuh")
KS = (5, 7)
NOUT = {5: 8, 7: 8}   # output columns per lane item
# word columns an item of the sliding form sorts beyond its own windows, for
# the next item: they put each item's new word columns on an 8-byte boundary
# of the stage (two words per shared load)
LOOKAHEAD = {5: 1, 7: 0}
# windows whose kernel runs the sliding form (a lane filters a span of items
# and hands the shared columns and blocks on); the others run items on their
# own (the 5x5 sliding form measured slower: its carry spills at the
# 96-register cap of two CTAs per SM)
SLIDING = {5: False, 7: True}
NEG, POS = "-inf", "+inf"

# optimal-size sorting networks for small n (D. Knuth, TAOCP 5.3.4)
SORTS = {
    2: [(0, 1)],
    3: [(0, 1), (1, 2), (0, 1)],
    4: [(0, 1), (2, 3), (0, 2), (1, 3), (1, 2)],
    6: [(1, 2), (4, 5), (0, 2), (3, 5), (0, 1), (3, 4), (2, 5), (0, 3), (1, 4), (2, 4), (1, 3), (2, 3)],
    8: [(0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7), (0, 1), (2, 3), (4, 5), (6, 7),
        (2, 4), (3, 5), (1, 4), (3, 6), (1, 2), (3, 4), (5, 6)],
}


# ---------------------------------------------------------------------------
# programs: a list of (dst, kind, args); kinds in / min / max / lo / hi
# (lo, hi: the low or high 16-bit halves of two words, packed)
# ---------------------------------------------------------------------------
class Prog:
    """Straight-line program; an operation identical to an earlier one (min and
    max taken as commutative) returns the earlier value instead."""

    def __init__(self):
        self.ops: List[Tuple[int, str, tuple]] = []
        self.seen: Dict[tuple, int] = {}

    def _new(self, kind, *args) -> int:
        key = (kind, tuple(sorted(args)) if kind in ("min", "max") else args)
        if kind != "in" and key in self.seen:
            return self.seen[key]
        d = len(self.ops)
        self.ops.append((d, kind, args))
        self.seen[key] = d
        return d

    def inp(self, name) -> int:
        return self._new("in", name)

    def mn(self, a, b) -> int:
        return self._new("min", a, b)

    def mx(self, a, b) -> int:
        return self._new("max", a, b)

    def lo(self, a, b) -> int:
        return self._new("lo", a, b)

    def hi(self, a, b) -> int:
        return self._new("hi", a, b)


def oe_merge(ces: list, A: Sequence[int], B: Sequence[int]) -> List[int]:
    """Batcher's odd-even merge of the sorted wire lists A and B (any lengths):
    appends its compare-exchanges (min to the first wire) to `ces` and returns
    the wires of the merged sequence in order."""
    if not A:
        return list(B)
    if not B:
        return list(A)
    if len(A) == 1 and len(B) == 1:
        ces.append((A[0], B[0]))
        return [A[0], B[0]]
    v = oe_merge(ces, A[0::2], B[0::2])
    w = oe_merge(ces, A[1::2], B[1::2])
    out = [v[0]]
    for i in range(max(len(w), len(v) - 1)):
        if i < len(w) and i + 1 < len(v):
            ces.append((w[i], v[i + 1]))
            out += [w[i], v[i + 1]]
        elif i < len(w):
            out.append(w[i])
        else:
            out.append(v[i + 1])
    return out


def _zero_one(lists: Sequence[Sequence[int]]):
    """Every 0-1 assignment that keeps each list sorted, as bool arrays per wire."""
    import numpy as np
    sizes = [len(L) + 1 for L in lists]
    total = 1
    for s in sizes:
        total *= s
    idx = np.arange(total)
    sim = {}
    for L, s in zip(lists, sizes):
        a = idx % s
        idx = idx // s
        for j, w in enumerate(L):
            sim[w] = j >= a
    return sim, total


def merge(p: Prog, A: Sequence, B: Sequence, ranks) -> Dict[int, int]:
    """Ranks `ranks` of the union of the sorted value lists A and B. NEG / POS
    entries stand for values known to lie below / above every wanted rank.
    Exchanges that sorted inputs never swap are dropped, those that always
    swap become relabels, and only what the wanted ranks read is emitted."""
    import numpy as np
    ces: list = []
    wa = list(range(len(A)))
    wb = list(range(len(A), len(A) + len(B)))
    out = oe_merge(ces, wa, wb)
    vals = dict(zip(wa + wb, list(A) + list(B)))
    sim, total = _zero_one([[w for w in wa if vals[w] not in (NEG, POS)],
                            [w for w in wb if vals[w] not in (NEG, POS)]])
    for w in wa + wb:
        if vals[w] == NEG:
            sim[w] = np.zeros(total, bool)
        elif vals[w] == POS:
            sim[w] = np.ones(total, bool)
    steps = []
    for a, b in ces:
        x, y = sim[a], sim[b]
        if not np.any(x & ~y):
            continue
        steps.append(("swap" if (np.all(x) or not np.any(y)) else "ce", a, b))
        sim[a], sim[b] = x & y, x | y
    live = {out[r] for r in ranks}
    kept = []
    for kind, a, b in reversed(steps):
        if a in live or b in live:
            kept.append((kind, a, b, a in live, b in live))
            live |= {a, b}
    v = dict(vals)
    for kind, a, b, ka, kb in reversed(kept):
        x, y = v[a], v[b]
        if kind == "swap":
            v[a], v[b] = y, x
            continue
        assert x not in (NEG, POS) and y not in (NEG, POS)
        if ka:
            v[a] = p.mn(x, y)
        if kb:
            v[b] = p.mx(x, y)
    res = {r: v[out[r]] for r in ranks}
    assert all(x not in (NEG, POS) for x in res.values())
    return res


def sort_values(p: Prog, X: Sequence[int]) -> List[int]:
    v = list(X)
    for a, b in SORTS[len(X)]:
        v[a], v[b] = p.mn(v[a], v[b]), p.mx(v[a], v[b])
    return v


def vertical(p: Prog, rows: Sequence[int], k: int) -> Tuple[List[int], List[int]]:
    """rows: the k+1 words of rows y-R .. y+R+1 of one word column. Returns the
    sorted windows of rows y (top) and y+1 (bot)."""
    core = sort_values(p, rows[1:k])
    top = merge(p, [rows[0]], core, range(k))
    bot = merge(p, core, [rows[k]], range(k))
    return [top[i] for i in range(k)], [bot[i] for i in range(k)]


def select(p: Prog, S: Dict[int, int], C: Sequence[int], m: int) -> int:
    """Rank m of S u C, S given by its ranks m-len(C) .. m, C sorted."""
    r = S[m]
    for i in range(1, len(C) + 1):
        r = p.mn(r, p.mx(S[m - i], C[i - 1]))
    return r


def first_word_col(k: int) -> int:
    """Column (relative to x0) of the low half of the item's first word."""
    R = (k - 1) // 2
    return -R if R % 2 == 0 else -R - 1


def words_per_row(k: int) -> int:
    R = (k - 1) // 2
    return (NOUT[k] - 1 + R - first_word_col(k)) // 2 + 1


def horizontal(p: Prog, col, k: int, x0: int = 0):
    """col(c) -> the sorted column c (k row-packed values). Returns, per output
    column j of the item whose first output column is x0, (j, median, window
    min, window max)."""
    m = (k * k - 1) // 2
    M2: Dict[int, List[int]] = {}

    def m2(j):
        if j not in M2:
            d = merge(p, col(j), col(j + 1), range(2 * k))
            M2[j] = [d[i] for i in range(2 * k)]
        return M2[j]

    outs = []
    if k == 5:
        for x in range(x0, x0 + NOUT[k], 2):
            A, B = m2(x - 1), m2(x + 1)             # columns x-1 .. x+2, shared by x and x+1
            S = merge(p, A, B, range(m - k, m + 1))
            smin, smax = p.mn(A[0], B[0]), p.mx(A[-1], B[-1])
            for o, C in ((x, col(x - 2)), (x + 1, col(x + 3))):
                outs.append((o, select(p, S, C, m), p.mn(smin, C[0]), p.mx(smax, C[-1])))
    elif k == 7:
        B4: Dict[int, tuple] = {}

        def b4(j):                                   # columns j .. j+3
            if j not in B4:
                A, B = m2(j), m2(j + 2)
                B4[j] = (merge(p, A, B, range(3, 25)), p.mn(A[0], B[0]), p.mx(A[-1], B[-1]))
            return B4[j]

        for x in range(x0, x0 + NOUT[k], 2):         # columns x-2 .. x+3, shared by x and x+1
            if x % 4 == 0:
                (Bd, bmin, bmax), A = b4(x), m2(x - 2)
            else:
                (Bd, bmin, bmax), A = b4(x - 2), m2(x + 2)
            Bl = [Bd[i] if i in Bd else (NEG if i < 3 else POS) for i in range(28)]
            S = merge(p, A, Bl, range(m - k, m + 1))
            smin, smax = p.mn(A[0], bmin), p.mx(A[-1], bmax)
            for o, C in ((x, col(x - 3)), (x + 1, col(x + 4))):
                outs.append((o, select(p, S, C, m), p.mn(smin, C[0]), p.mx(smax, C[-1])))
    else:
        raise ValueError(k)
    return outs


def _columns(p: Prog, k: int, w_first: int, w_end: int):
    """col(c) for the word columns w_first .. w_end-1 (word w: columns
    first_word_col(k) + 2w and the next), built on first use: the rows of a
    word column are loaded, sorted vertically and transposed."""
    w0 = first_word_col(k)
    cols: Dict[int, List[int]] = {}
    loaded: Dict[int, List[int]] = {}

    def rows_of(w):
        if w not in loaded:
            loaded[w] = [p.inp((r, w)) for r in range(k + 1)]
        return loaded[w]

    def col(c):
        if c not in cols:
            # a word column's rows are read one word column ahead of their
            # use: few inputs are live at a time, and the loads' latency
            # overlaps the previous column's work
            w = (c - w0) // 2
            assert w_first <= w < w_end, (c, w)
            rows = rows_of(w)
            if w + 1 < w_end:
                rows_of(w + 1)
            top, bot = vertical(p, rows, k)
            cols[w0 + 2 * w] = [p.lo(top[i], bot[i]) for i in range(k)]
            cols[w0 + 2 * w + 1] = [p.hi(top[i], bot[i]) for i in range(k)]
        return cols[c]

    col.rows = rows_of  # the input words of a word column, rows 0 .. k
    return col


def item_program(k: int):
    """The whole lane item: inputs r[row][word] (x-packed), outputs per column."""
    p = Prog()
    outs = horizontal(p, _columns(p, k, 0, words_per_row(k)), k)
    return p, outs


def _ancestors(p: Prog, roots) -> set:
    seen = set(roots)
    for d, kind, args in reversed(p.ops):
        if d in seen and kind != "in":
            seen |= {a for a in args if isinstance(a, int)}
    return seen


def span_program(k: int):
    """The sliding form of the item, for a lane that filters several items of
    one row pair side by side. Neighbouring items (x0 - NOUT, x0) share sorted
    columns and merged blocks: the program of both is built, the values of the
    left item that the right one reads are its carry, and
      pre  computes the carry of the item at x0 (what the item at x0 - NOUT
           would hand over) from the words they share,
      body computes the item at x0 from its carry and its new word columns and
           leaves the carry of the item at x0 + NOUT (the same values NOUT
           columns further right, matched by their structure).
    Returns (p, pre ops, body ops, carry in, carry out, outputs of x0)."""
    n = NOUT[k]
    shift = n // 2                                  # words per item
    nw = words_per_row(k)
    w0 = first_word_col(k)
    p = Prog()
    col = _columns(p, k, -shift, nw + LOOKAHEAD[k])
    outs_a = horizontal(p, col, k, -n)
    ahead_a = [v for j in range(LOOKAHEAD[k]) for h in (0, 1) for v in col(w0 + 2 * (nw + j - shift) + h)]
    outs_b = horizontal(p, col, k, 0)
    # each output also carries the x-packed words of its centre pixels (rows
    # y and y + 1 are the item's stage rows R and R + 1): the flag test takes
    # them from the words the network loaded, not from shared memory again
    R = (k - 1) // 2
    outs_b = [(o, *rest, col.rows((o - w0) // 2)[R], col.rows((o - w0) // 2)[R + 1]) for o, *rest in outs_b]
    ahead_b = [v for j in range(LOOKAHEAD[k]) for h in (0, 1) for v in col(w0 + 2 * (nw + j) + h)]
    da = _ancestors(p, [v for o in outs_a for v in o[1:]] + ahead_a)
    db = _ancestors(p, [v for o in outs_b for v in o[1:]] + ahead_b)
    out_b = {v for o in outs_b for v in o[1:]}

    def cut(left, roots):
        """Body ops and carry when the values in `left` come from the left item."""
        ops = [op for op in p.ops if op[0] in roots and op[0] not in left]
        need = {a for _, kind, args in ops if kind != "in" for a in args if a in left} | (out_b & left)
        return ops, sorted(need)
    left = set(da)
    body, carry_in = cut(left, db)
    # structural keys: equal keys compute the same function of the same words
    intern: Dict[tuple, int] = {}
    key: Dict[int, int] = {}
    for d, kind, args in p.ops:
        if kind == "in":
            t = ("in", *args[0])
        else:
            ka = [key[a] for a in args]
            t = (kind, *(sorted(ka) if kind in ("min", "max") else ka))
        key[d] = intern.setdefault(t, len(intern))
    moved: Dict[int, object] = {}                    # key of the same structure `shift` words right
    for d, kind, args in p.ops:
        if kind == "in":
            row, w = args[0]
            tm = ("in", row, w + shift)
        else:
            km = [moved[a] for a in args]
            tm = None if None in km else (kind, *(sorted(km) if kind in ("min", "max") else km))
        moved[d] = intern.get(tm) if tm is not None else None
    by_key = {key[d]: d for d in key}
    # A transposition whose inputs the left item holds is moved to the left
    # item (whose own word columns' transpositions then compute it one item
    # earlier) when that shrinks the carry: one transposed value instead of
    # the two sorted words it reads.
    for d, kind, args in list(body):
        if kind in ("lo", "hi") and all(a in left for a in args) and moved[d] in by_key:
            twin = by_key[moved[d]]
            trial = left | {d}
            db_t = db | _ancestors(p, [twin])
            ops_t, need_t = cut(trial, db_t)
            if len(need_t) < len(carry_in):
                left, db = trial, db_t
                body, carry_in = ops_t, need_t
    carry_out = []
    for c in carry_in:
        assert moved[c] is not None and moved[c] in by_key, ("carry without a counterpart", c)
        d = by_key[moved[c]]
        assert d in db and d not in left, ("carry counterpart outside the item", c, d)
        carry_out.append(d)
    pre_set = _ancestors(p, carry_in)
    pre = [op for op in p.ops if op[0] in pre_set]
    return p, pre, body, carry_in, carry_out, outs_b


def horizontal_program(k: int):
    """The horizontal stage alone: inputs ("col", c, i) are rank i of the
    sorted column c (row-packed), for the tests."""
    p = Prog()
    cols: Dict[int, List[int]] = {}

    def col(c):
        if c not in cols:
            cols[c] = [p.inp(("col", c, i)) for i in range(k)]
        return cols[c]

    return p, horizontal(p, col, k)


def vertical_program(k: int):
    """The vertical stage of one word column: inputs ("row", r), outputs the
    sorted windows of the item's two output rows, for the tests."""
    p = Prog()
    rows = [p.inp(("row", r)) for r in range(k + 1)]
    top, bot = vertical(p, rows, k)
    return p, top, bot


def live_ops(p: Prog, outs) -> List[Tuple[int, str, tuple]]:
    live = set()
    for o in outs:
        live |= set(o[1:])
    for d, kind, args in reversed(p.ops):
        if d in live and kind != "in":
            live |= {a for a in args if isinstance(a, int)}
    return [op for op in p.ops if op[0] in live]


def op_counts(ops) -> Dict[str, int]:
    c: Dict[str, int] = {}
    for _, kind, _ in ops:
        c[kind] = c.get(kind, 0) + 1
    return c


# ---------------------------------------------------------------------------
# emission
# ---------------------------------------------------------------------------
def _emit_ops(k: int, ops, outs, lines: List[str], indent: str = "    ", pairs: bool = True) -> None:
    """Emit a straight-line op list; a min and max of the same operands form a
    compare-exchange whose max may take the FMA-pipe form (op.cmax<J>)."""
    pair_of = {}
    mins = {}
    for d, kind, args in ops:
        if kind == "min":
            mins[tuple(sorted(args))] = d
        elif kind == "max" and tuple(sorted(args)) in mins:
            pair_of[d] = mins[tuple(sorted(args))]
    defined = {d for d, _, _ in ops}
    done_at: Dict[int, list] = {}
    for o in outs:
        done_at.setdefault(max(v for v in o[1:] if v in defined) if any(v in defined for v in o[1:]) else -1,
                           []).append(o)
    def put(o):
        return f"{indent}emit.template put<{o[0]}>(" + ", ".join(f"v{v}" for v in o[1:]) + ");"
    for o in sorted(done_at.pop(-1, []), key=lambda o: o[0]):
        lines.append(put(o))
    # words (w, w + 1) of a row that start on an 8-byte boundary of the stage
    # (w of parity `par`) are read by one shared load where both are read
    par = (-first_word_col(k) // 2) % 2
    word_at = {args[0]: d for d, kind, args in ops if kind == "in"}
    loaded = set()
    j = 0
    for d, kind, args in ops:
        if kind == "in":
            if d in loaded:
                continue
            row, word = args[0]
            base = word if word % 2 == par else word - 1
            mate = word_at.get((row, base + 1 if word == base else base)) if pairs else None
            if mate is None:
                lines.append(f"{indent}const uint32_t v{d} = ld.template get<{row}, {word}>();")
            else:
                lo_v, hi_v = (d, mate) if word == base else (mate, d)
                lines.append(f"{indent}uint32_t v{lo_v}, v{hi_v};")
                lines.append(f"{indent}ld.template get2<{row}, {base}>(v{lo_v}, v{hi_v});")
                loaded.add(mate)
        elif kind == "min":
            lines.append(f"{indent}const uint32_t v{d} = op.mn(v{args[0]}, v{args[1]});")
        elif kind == "max":
            if d in pair_of:
                lines.append(f"{indent}const uint32_t v{d} = op.template cmax<{j}>(v{args[0]}, v{args[1]}, "
                             f"v{pair_of[d]});")
                j += 1
            else:
                lines.append(f"{indent}const uint32_t v{d} = op.mx(v{args[0]}, v{args[1]});")
        elif kind == "lo":
            lines.append(f"{indent}const uint32_t v{d} = __byte_perm(v{args[0]}, v{args[1]}, 0x5410);")
        elif kind == "hi":
            lines.append(f"{indent}const uint32_t v{d} = __byte_perm(v{args[0]}, v{args[1]}, 0x7632);")
        for o in sorted(done_at.get(d, []), key=lambda o: o[0]):
            lines.append(put(o))


def _shape(k: int, sliding: bool) -> List[str]:
    return [f"template <> struct SepNet<{k}> {{",
            f"  static constexpr bool kSliding = {'true' if sliding else 'false'};",
            f"  static constexpr int kOut = {NOUT[k]};",
            f"  static constexpr int kRows = {k + 1};",
            f"  static constexpr int kWords = {words_per_row(k)};",
            f"  static constexpr int kFirstCol = {first_word_col(k)};"]


def emit_item(k: int) -> List[str]:
    p, outs = item_program(k)
    ops = live_ops(p, outs)
    c = op_counts(ops)
    lines = [f"// k={k}: {c.get('min', 0)} min, {c.get('max', 0)} max, {c.get('lo', 0) + c.get('hi', 0)} permutes"
             f" per item of {2 * NOUT[k]} pixels"] + _shape(k, False) + [
             "  // ld.get<row, word>(): x-packed word `word` (columns x0 + kFirstCol + 2 word and the next)",
             "  // of stage row `row` of the item (0 .. k); emit.put<j>(g_m, g_min, g_max) gets the",
             "  // row-packed results of output column x0 + j (low half row y, high half row y + 1)",
             "  template <class Op, class Load, class Emit>",
             "  __device__ __forceinline__ static void run(const Op op, Load &&ld, Emit &&emit) {"]
    _emit_ops(k, ops, outs, lines, pairs=False)
    lines += ["  }", "};", ""]
    return lines


def emit_sliding(k: int) -> List[str]:
    p, pre, body, carry_in, carry_out, outs = span_program(k)
    c = op_counts(body)
    cp = op_counts(pre)
    nc = len(carry_in)
    lines = [f"// k={k}, sliding items of {2 * NOUT[k]} pixels: per item {c.get('min', 0)} min, {c.get('max', 0)} max,"
             f" {c.get('lo', 0) + c.get('hi', 0)} permutes and {c.get('in', 0)} word loads, {nc} values"
             f" carried; before a lane's first item {cp.get('min', 0) + cp.get('max', 0)} min/max,"
             f" {cp.get('lo', 0) + cp.get('hi', 0)} permutes"] + _shape(k, True) + [
             f"  static constexpr int kCarry = {nc};",
             "  // ld.get<row, word>(): x-packed word `word` (columns x0 + kFirstCol + 2 word and the next)",
             "  // of stage row `row` of the item at x0 (0 .. k); ld.get2<row, word>(a, b): words `word` and",
             "  // `word` + 1 by one 8-byte aligned read; emit.put<j>(g_m, g_min, g_max, a, b) gets the",
             "  // row-packed results of output column x0 + j (low half row y, high half row y + 1) and the",
             "  // x-packed words a, b of rows y and y + 1 that hold the centre pixels of column x0 + j",
             "  // pre: the carry of the item at x0, from its first word columns",
             "  template <class Op, class Load>",
             f"  __device__ __forceinline__ static void pre(const Op op, Load &&ld, uint32_t (&c)[{nc}]) {{"]
    _emit_ops(k, pre, [], lines)
    for i, d in enumerate(carry_in):
        lines.append(f"    c[{i}] = v{d};")
    lines += ["  }",
              "  // body: the item at x0 from its carry c; leaves in c the carry of the item at x0 + kOut",
              "  template <class Op, class Load, class Emit>",
              f"  __device__ __forceinline__ static void body(const Op op, Load &&ld, Emit &&emit, "
              f"uint32_t (&c)[{nc}]) {{"]
    for i, d in enumerate(carry_in):
        lines.append(f"    const uint32_t v{d} = c[{i}];")
    _emit_ops(k, body, outs, lines)
    for i, d in enumerate(carry_out):
        lines.append(f"    c[{i}] = v{d};")
    lines += ["  }", "};", ""]
    return lines


def emit() -> str:
    lines = [
        "// Generated by gen_separable.py: separable median networks of the dense strategy.",
        "// Do not edit by hand; rerun the generator.",
        "#pragma once",
        "#include <cstdint>",
        "",
        "namespace fnr {",
        "",
        "template <int K> struct SepNet;",
        "",
    ]
    for k in KS:
        lines += emit_sliding(k) if SLIDING[k] else emit_item(k)
    lines += ["}  // namespace fnr", ""]
    return "\n".join(lines)


# ---------------------------------------------------------------------------
# evaluation (tests)
# ---------------------------------------------------------------------------
def evaluate(ops, inputs: Dict[int, object], mn, mx, lo=None, hi=None) -> Dict[int, object]:
    """Evaluate a program given values for its inputs (by op id) and the
    elementwise operations to use (for the tests: numpy arrays, or 0-1
    bitsets with AND for min and OR for max)."""
    v = dict(inputs)
    for d, kind, args in ops:
        if kind == "in":
            continue
        if kind == "min":
            v[d] = mn(v[args[0]], v[args[1]])
        elif kind == "max":
            v[d] = mx(v[args[0]], v[args[1]])
        elif kind == "lo":
            v[d] = lo(v[args[0]], v[args[1]])
        else:
            v[d] = hi(v[args[0]], v[args[1]])
    return v


def main() -> None:
    with open(HEADER, "w") as fh:
        fh.write(emit())
    for k in KS:
        if SLIDING[k]:
            _, pre, body, carry_in, _, _ = span_program(k)
            c = op_counts(body)
            what = f"per sliding item, {len(carry_in)} values carried"
        else:
            p, outs = item_program(k)
            c = op_counts(live_ops(p, outs))
            what = "per item"
        mm = c.get("min", 0) + c.get("max", 0)
        print(f"k={k}: {mm} min/max {what} ({mm / (2 * NOUT[k]):.2f} per pixel), "
              f"{c.get('lo', 0) + c.get('hi', 0)} permutes")


if __name__ == "__main__":
    main()
