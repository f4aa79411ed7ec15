"""The padded shared-memory layout of the one-sweep tile paint (TSC and PCS
on 16^3 tiles, Sec. 3.3.1 painting with the windows of Sec. 3.3.2),
modelled on the CPU from the constants in the kernel source (no GPU):

* every window that reaches the tile along z is kept (its first node lies in
  [BzMin, BzMax]) and all its deposits stay inside their row's words;
* a kept window that does not reach the tile deposits into the halo only;
* the rows of the tile's 16 x 16 (x, y) positions are disjoint and inside the
  mesh's words, which are a multiple of four (16-byte zeroing);
* the row starts fall on all 32 shared-memory banks (odd strides: lanes whose
  candidates share z offsets but sit in different rows spread over the
  banks instead of piling onto a few).

The GPU tests check the painted meshes themselves against the oracle."""
import math
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(__file__), os.pardir, "paper_1712_05834_gb300", "csrc", "pk_kernels.cu")
T = 16


def _cexpr(expr, P):
    """Value of a C expression made of integers, P, ==, ?: and parentheses."""
    toks = re.findall(r"\d+|==|[?:()]|[-+*]|P", expr)
    pos = 0

    def peek():
        return toks[pos] if pos < len(toks) else None

    def take():
        nonlocal pos
        pos += 1
        return toks[pos - 1]

    def atom():
        t = take()
        if t == "(":
            v = ternary()
            assert take() == ")"
            return v
        if t == "P":
            return P
        return int(t)

    def arith():
        v = atom()
        while peek() in ("+", "-", "*"):
            op, r = take(), atom()
            v = v + r if op == "+" else (v - r if op == "-" else v * r)
        return v

    def comparison():
        v = arith()
        if peek() == "==":
            take()
            v = int(v == arith())
        return v

    def ternary():
        c = comparison()
        if peek() == "?":
            take()
            a = ternary()
            assert take() == ":"
            b = ternary()
            return a if c else b
        return c

    v = ternary()
    assert pos == len(toks), expr
    return v


def layout(P):
    src = open(SRC).read()
    body = src[src.index("struct SweepLayout {"):]
    body = body[:body.index("};")]
    get = lambda name: _cexpr(re.search(r"static constexpr int %s = ([^;]+);" % name, body).group(1), P)
    assert get("T") == T
    zlo, ys, xs = get("Zlo"), get("YS"), get("XS")
    return zlo, ys, xs, T * xs


def first_node(P, u):
    """First node of the window at tile-frame coordinate u (the kernel's spline bases)."""
    return math.floor(u - 0.5) if P == 3 else math.floor(u) - 1


@pytest.mark.parametrize("P", [3, 4])
def test_windows_that_reach_the_tile_stay_in_their_row(P):
    zlo, ys, xs, words = layout(P)
    bz_min, bz_max = -zlo, ys - zlo - P
    for k in range(-8 * 64, 26 * 64):
        u = k / 64.0 + 1.0 / 128.0
        b = first_node(P, u)
        reaches = b + P - 1 >= 0 and b <= T - 1
        kept = bz_min <= b <= bz_max
        if reaches:
            assert kept, (P, u, b)
        if kept:
            offs = [b + zlo + c for c in range(P)]
            assert all(0 <= o < ys for o in offs), (P, u, offs)
            if not reaches:
                assert all(not (zlo <= o < zlo + T) for o in offs), (P, u, offs)


@pytest.mark.parametrize("P", [3, 4])
def test_rows_are_disjoint_inside_the_mesh_and_cover_every_bank(P):
    zlo, ys, xs, words = layout(P)
    assert words % 4 == 0
    starts = sorted(x * xs + y * ys for x in range(T) for y in range(T))
    assert starts[0] == 0 and starts[-1] + ys <= words
    assert all(b - a >= ys for a, b in zip(starts, starts[1:]))
    assert len({s % 32 for s in starts}) == 32
    # the flush reads the cell pairs (z, z + 1), z even, of every row
    assert zlo + T <= ys
