#!/usr/bin/env python3
"""Generate the rank-m selection networks used by the per-pixel median stage.

For a flagged pixel the kernel gathers its n = k*k window values into
registers and runs a fixed compare-exchange network whose wire ``out``
ends up holding the element of rank m = (n-1)/2 (the median g_m of S_xy,
Sec. 3.4). Any exact selection gives the same g_m; a network is used on the
GPU because it is branch-free and lives in registers.

Construction:
* k = 3: sort the three columns, sort the three rows, then the median is the
  median of the anti-diagonal (a standard result for 3x3 matrices with sorted
  rows and columns); expressed as compare-exchanges and pruned.
* k >= 5: Parberry's pairwise sorting network (I. Parberry, "The pairwise
  sorting network", Parallel Processing Letters 2(2-3), 1992) on N = 2^t >= n
  wires, with the n window values on wires 1..n and the other wires standing
  for -inf (wire 0) and +inf (wires n+1..N-1): a compare-exchange that touches
  one of those is a no-op and is dropped, and rank m of the window is wire
  m + 1. Pruned to the median wire it needs 182 / 512 / 1090 min-max
  operations for k = 5 / 7 / 9, against 202 / 578 / 1242 for Knuth's
  merge-exchange network (TAOCP 5.3.4, Algorithm M) pruned the same way
  (``merge_exchange`` below, kept for comparison). One -inf wire gave the
  fewest operations of all splits of the padding.
Pruning walks the network backwards keeping only compare-exchanges whose
min or max output is still live; a half that is never read is not emitted.

A compare-exchange whose two outputs are both live is emitted as
``op.cx<j>(a, b)`` with j its index among such exchanges, so that the
operation type can spread them over different execution units; one with a
single live output is a lone ``op.mn`` or ``op.mx``.

Run this file to rewrite ``fnr_networks.cuh``; the tests import it to check
each network with the 0-1 principle and that the header is up to date.
"""
from __future__ import annotations

import os
from typing import List, Tuple

CE = Tuple[int, int, bool, bool]   # (a, b, keep_min_on_a, keep_max_on_b)

KS = (3, 5, 7, 9)
HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "fnr_networks.cuh")


def merge_exchange(n: int) -> List[Tuple[int, int]]:
    """Knuth's merge exchange: a sorting network for any n >= 1."""
    if n < 2:
        return []
    ces = []
    t = (n - 1).bit_length()
    p = 1 << (t - 1)
    while p > 0:
        q, r, d = 1 << (t - 1), 0, p
        while True:
            for i in range(n - d):
                if (i & p) == r:
                    ces.append((i, i + d))
            if q == p:
                break
            d, q, r = q - p, q >> 1, p
        p >>= 1
    return ces


def pairwise(N: int) -> List[Tuple[int, int]]:
    """Parberry's pairwise sorting network on N = 2^t wires: compare-exchanges
    (i, j), i < j, min to i. First the pairing phase (adjacent blocks of size
    a = 1, 2, 4, ... compared element by element), then the merging phase
    (for a = N/4 .. 1, distances d*a for d = 2^s - 1 .. 1)."""
    assert N >= 2 and N & (N - 1) == 0
    ces = []
    a = 1
    while a < N:
        b, c = a, 0
        while b < N:
            ces.append((b - a, b))
            b += 1
            c = (c + 1) % a
            if c == 0:
                b += a
        a *= 2
    a //= 4
    e = 1
    while a > 0:
        d = e
        while d > 0:
            b, c = (d + 1) * a, 0
            while b < N:
                ces.append((b - d * a, b))
                b += 1
                c = (c + 1) % a
                if c == 0:
                    b += a
            d //= 2
        a //= 2
        e = e * 2 + 1
    return ces


def pairwise_padded(n: int, low: int = 1) -> List[Tuple[int, int]]:
    """Pairwise network for n values on wires low..low+n-1 of the next power of
    two, renumbered to 0..n-1; exchanges with a padding wire (-inf below,
    +inf above) are dropped, since they never move a value."""
    N = 1
    while N < n + low:
        N *= 2
    return [(a - low, b - low) for a, b in pairwise(N) if a >= low and b < low + n]


def prune(ces: List[Tuple[int, int]], out: int) -> List[CE]:
    live = {out}
    kept: List[CE] = []
    for a, b in reversed(ces):
        if a in live or b in live:
            kept.append((a, b, a in live, b in live))
            live |= {a, b}
    kept.reverse()
    return kept


def median_network(k: int) -> Tuple[List[CE], int]:
    """(pruned network, output wire) selecting rank (k*k-1)/2 of k*k wires.
    Wire i*k+j holds window row i, column j."""
    n = k * k
    m = (n - 1) // 2
    if k == 3:
        idx = lambda i, j: 3 * i + j
        s3 = [(0, 1), (1, 2), (0, 1)]
        ces = []
        for j in range(3):
            ces += [(idx(a, j), idx(b, j)) for a, b in s3]
        for i in range(3):
            ces += [(idx(i, a), idx(i, b)) for a, b in s3]
        diag = [idx(0, 2), idx(1, 1), idx(2, 0)]
        ces += [(diag[a], diag[b]) for a, b in s3]
        return prune(ces, diag[1]), diag[1]
    return prune(pairwise_padded(n), m), m


def op_count(net: List[CE]) -> int:
    return sum(int(a) + int(b) for _, _, a, b in net)


def apply(net: List[CE], values):
    w = list(values)
    for a, b, _, _ in net:
        x, y = w[a], w[b]
        w[a], w[b] = min(x, y), max(x, y)
    return w


def emit() -> str:
    lines = [
        "// Generated by gen_networks.py: rank-(k*k-1)/2 selection networks.",
        "// Do not edit by hand; rerun the generator.",
        "#pragma once",
        "#include <cstdint>",
        "",
        "namespace fnr {",
        "",
        "template <int K> struct MedianNet;",
        "",
    ]
    for k in KS:
        net, out = median_network(k)
        n = k * k
        lines.append(f"// k={k}: {len(net)} compare-exchanges, {op_count(net)} min/max ops")
        lines.append(f"template <> struct MedianNet<{k}> {{")
        lines.append(f"  static constexpr int kOps = {op_count(net)};")
        lines.append(f"  template <class Op> __device__ __forceinline__ static uint32_t run(uint32_t (&v)[{n}], Op op) {{")
        j = 0
        for a, b, ka, kb in net:
            if ka and kb:
                lines.append(f"    op.template cx<{j}>(v[{a}], v[{b}]);")
                j += 1
            elif ka:
                lines.append(f"    v[{a}] = op.mn(v[{a}], v[{b}]);")
            else:
                lines.append(f"    v[{b}] = op.mx(v[{a}], v[{b}]);")
        lines.append(f"    return v[{out}];")
        lines.append("  }")
        lines.append("};")
        lines.append("")
    lines.append("}  // namespace fnr")
    lines.append("")
    return "\n".join(lines)


def main() -> None:
    with open(HEADER, "w") as fh:
        fh.write(emit())
    for k in KS:
        net, _ = median_network(k)
        print(f"k={k}: {len(net)} CEs, {op_count(net)} ops")


if __name__ == "__main__":
    main()
