"""The split band -> full form's work layout, checked on the host (no GPU):
the library walks the layout its launcher would use, as the apply and
preparation kernels walk it, for many sizes and SM counts. Every row of
every 32-reflector block must belong to exactly one (slot, batch, part) row,
each (strip, slot) to one CTA, and each block's W counter must wait for
exactly the slots that publish."""

import ctypes

import pytest

from paper_2002_10991_gb300 import _native


@pytest.fixture(scope="module")
def L():
    _native.build()
    return _native.load()


SHAPES = [(2, 1, 2), (5, 2, 3), (33, 1, 33), (64, 63, 9), (65, 64, 65), (96, 64, 96), (100, 8, 37),
          (129, 96, 129), (200, 128, 50), (257, 32, 100), (300, 16, 70), (300, 64, 300), (400, 32, 40),
          (513, 64, 200), (600, 64, 300), (700, 5, 613), (1000, 64, 500), (1000, 64, 1000), (2100, 64, 1000),
          (3000, 48, 2999), (4096, 64, 2048)]


@pytest.mark.parametrize("sms", [152, 148, 132, 17, 8, 3, 1])
def test_layout_covers_every_row_once(L, sms):
    sk = ctypes.c_int32()
    items = ctypes.c_int64()
    for n, b, nev in SHAPES:
        rc = L.tbbt_b2f_split_layout_check(n, b, nev, sms, ctypes.byref(sk), ctypes.byref(items))
        assert rc == 0, (n, b, nev, sms, rc)
        if n > b:
            assert 1 <= sk.value <= min(8, sms) and items.value >= 1


def test_slots_per_strip_follow_the_strip_count(L):
    # 32 strips on 152 SMs: 4 slots each (128 CTAs); 77 strips: 7 slots, the
    # fewest rounds of strips per CTA group (see the launcher)
    sk = ctypes.c_int32()
    for nev, want in [(4096, 4), (9830, 7), (128, 8), (19456, 1)]:
        n = max(nev, 8192)
        assert L.tbbt_b2f_split_layout_check(n, 64, nev, 152, ctypes.byref(sk), None) == 0
        assert sk.value == want, (nev, sk.value)


def test_layout_check_rejects_bad_arguments(L):
    assert L.tbbt_b2f_split_layout_check(0, 1, 1, 152, None, None) == -1
    assert L.tbbt_b2f_split_layout_check(10, 0, 1, 152, None, None) == -1
    assert L.tbbt_b2f_split_layout_check(10, 2, 11, 152, None, None) == -1
    assert L.tbbt_b2f_split_layout_check(10, 2, 5, 0, None, None) == -1
    assert L.tbbt_b2f_split_layout_check(10, 12, 5, 152, None, None) == 0  # nbw >= n: nothing to do
