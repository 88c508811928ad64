"""Host check of the GPU bulge chase's schedule (Eq. 6b, Sec. 2.2.1): stage
i+1 may run sweep j' once stage i has finished sweeps 0 .. j'+2.

Each sweep's touched band entries are enumerated from the reduction's
definition (generation column, left, diagonal block and right updates). The
test checks that sweep j' of stage i+1 shares no entry with any sweep
j >= j'+3 of stage i, or of any earlier stage at j >= j'+3, so those may run
concurrently, and that a lag of two sweeps would not be safe."""

import itertools

import pytest


def sweeps(n, b, cplx):
    last = n - 2 if cplx else n - 3
    for i in range(0, last + 1):
        ns = (n - i - 2 + b - 1) // b if i <= n - 3 else 1
        for j in range(ns):
            yield i, j


def touched(n, b, i, j):
    r = i + 1 + j * b
    L = min(b, n - r)
    c = i if j == 0 else r - b
    cells = set()
    for t in range(L):
        cells.add((r + t, c))                      # the reflector's column
        for col in range(c + 1, r):                # left
            cells.add((r + t, col))
        for s in range(t + 1):                     # diagonal block (lower)
            cells.add((r + t, r + s))
    for row in range(r + L, min(r + L + b, n)):    # right
        for t in range(L):
            cells.add((row, r + t))
    return cells


@pytest.mark.parametrize("n,b,cplx", [(12, 1, False), (20, 2, True), (33, 3, False), (40, 4, True), (57, 5, False),
                                      (64, 8, False), (50, 7, True)])
def test_lag_three_is_safe_and_two_is_not(n, b, cplx):
    sw = list(sweeps(n, b, cplx))
    cells = {s: touched(n, b, *s) for s in sw}
    conflicts_lag2 = 0
    for (i1, j1), (i0, j0) in itertools.product(sw, sw):
        if i0 >= i1:
            continue
        shared = cells[(i1, j1)] & cells[(i0, j0)]
        if j0 >= j1 + 3 * (i1 - i0):
            # a sweep of an earlier stage that may still run stays clear of sweep j1 of stage i1
            assert not shared, ((i1, j1), (i0, j0), sorted(shared)[:3])
        if i0 == i1 - 1 and j0 == j1 + 2 and shared:
            conflicts_lag2 += 1
    if b >= 2 and n >= 4 * b:
        assert conflicts_lag2 > 0  # a lag of two sweeps would race


def right_block(n, b, i, j):
    """The entries the right update of sweep j of stage i writes (empty for j < 0)."""
    if j < 0:
        return set()
    r = i + 1 + j * b
    L = min(b, n - r)
    return {(row, r + t) for row in range(r + L, min(r + L + b, n)) for t in range(L)}


@pytest.mark.parametrize("n,b,cplx", [(12, 1, False), (20, 2, True), (33, 3, False), (40, 4, True), (57, 5, False),
                                      (64, 8, False), (50, 7, True)])
def test_lag_three_is_safe_with_the_right_block_kept_on_chip(n, b, cplx):
    # The kernel keeps the right-update block of sweep j in shared memory and
    # writes it back to L2 during sweep j+1 (after that sweep's reflector and
    # left update have consumed it), before progress j+2 is released. So the
    # L2 entries that sweep j may hold stale or write are its own entries and
    # those of the right block of sweep j-1; sweeps that may run at the same
    # time must still share none.
    sw = list(sweeps(n, b, cplx))
    cells = {(i, j): touched(n, b, i, j) | right_block(n, b, i, j - 1) for (i, j) in sw}
    for (i1, j1), (i0, j0) in itertools.product(sw, sw):
        if i0 >= i1 or j0 < j1 + 3 * (i1 - i0):
            continue
        shared = cells[(i1, j1)] & cells[(i0, j0)]
        assert not shared, ((i1, j1), (i0, j0), sorted(shared)[:3])
    # the next sweep's reflector column and left-update columns are exactly
    # the right block of the sweep before it (what stays on chip)
    for (i, j) in sw:
        if j == 0:
            continue
        r = i + 1 + j * b
        L = min(b, n - r)
        consumed = {(r + t, col) for t in range(L) for col in range(r - b, r)}
        assert consumed == right_block(n, b, i, j - 1), (i, j)
    # a stage's last sweep may leave a right block (when n - i - 2 is a
    # multiple of b: the fill lands inside the band); no sweep of the stage
    # consumes it, so the kernel writes that one straight to L2
    last = {}
    for (i, j) in sw:
        last[i] = max(last.get(i, -1), j)
    assert any(right_block(n, b, i, j) for i, j in last.items()) == any(
        (n - i - 2) % b == 0 and j >= 0 for i, j in last.items() if i <= n - 3)
