"""The C ABI without a GPU: the library builds and loads, exports every
symbol include/tbbt.h declares, and its host-side logic (store geometry,
argument checks, the block schedule) is right. No kernel is launched."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2002_10991_gb300 import _native

HEADER = os.path.join(_native.INCLUDE, "tbbt.h")


@pytest.fixture(scope="module")
def L():
    _native.build()
    return _native.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tbbt_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("tbbt_trans_ev_tridi_to_band_d", "tbbt_trans_ev_tridi_to_band_z", "tbbt_plan_create",
                 "tbbt_plan_set_reflectors", "tbbt_plan_execute", "tbbt_plan_destroy", "tbbt_stream_check",
                 "tbbt_status_string", "tbbt_num_reflectors"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_num_reflectors_matches_oracle(L):
    for n in (0, 1, 2, 3, 4, 17, 64, 100, 513):
        for b in (1, 2, 3, 4, 31, 32, 64, 128, 1000):
            for c in (0, 1):
                assert L.tbbt_num_reflectors(n, b, c) == oracle.num_reflectors(n, b, bool(c))
    assert L.tbbt_num_reflectors(-1, 4, 0) == -1
    assert L.tbbt_num_reflectors(10, 0, 0) == -1


def test_status_strings(L):
    for s in range(6):
        assert len(L.tbbt_status_string(s)) > 0


def test_schedule_is_sound_for_many_shapes(L):
    # every reflector applied once, dependencies respected, warps disjoint,
    # rows resident when touched; the ring size formula covers the live rows
    for n in list(range(0, 36)) + [63, 64, 65, 129, 257, 600]:
        for b in (1, 2, 3, 4, 5, 8, 31, 32, 33, 64, 128):
            for c in (0, 1):
                for G, NB in ((1, 1), (2, 3), (3, 8), (4, 8), (8, 8), (16, 2)):
                    m = L.tbbt_schedule_max_live_rows(n, b, c, G, NB)
                    assert m >= 0, (n, b, c, G, NB)
                    assert m <= G * b + (G + 2) * NB + 8, (n, b, c, G, NB, m)


def test_argument_checks_fail_before_any_device_work(L):
    p = ctypes.c_void_p(16)
    EINVAL = 1
    f = L.tbbt_trans_ev_tridi_to_band_d
    assert f(p, p, 10, 0, 5, p, 10, None) == EINVAL  # nbw < 1
    assert f(p, p, 10, 129, 5, p, 10, None) == EINVAL  # nbw > 128
    assert f(p, p, 10, 4, 11, p, 10, None) == EINVAL  # nev > n
    assert f(p, p, 10, 4, -1, p, 10, None) == EINVAL
    assert f(p, p, 10, 4, 5, p, 9, None) == EINVAL  # ldq < n
    assert f(p, p, -1, 4, 0, p, 1, None) == EINVAL
    assert f(p, p, 10, 4, 5, None, 10, None) == EINVAL  # null q
    assert L.tbbt_trans_ev_tridi_to_band_z(p, p, 10, 4, 5, p, 3, None) == EINVAL
    plan = ctypes.c_void_p()
    assert L.tbbt_plan_create(ctypes.byref(plan), 7, 10, 4, 5, None) == EINVAL  # bad dtype
    assert L.tbbt_plan_create(ctypes.byref(plan), 0, 10, 0, 5, None) == EINVAL
    assert L.tbbt_plan_create(None, 0, 10, 4, 5, None) == EINVAL
    assert L.tbbt_plan_execute(None, p, 10, None) == EINVAL
    assert L.tbbt_plan_destroy(None) == 0
    # nothing to do is not an error and touches no device
    assert f(None, None, 10, 4, 0, p, 10, None) == 0


def test_generator_is_deterministic_and_counter_based():
    from paper_2002_10991_gb300 import inputs as I

    a = I.splitmix64(5, 1, 100)
    b = I.splitmix64(5, 1, 60, offset=40)
    assert np.array_equal(a[40:], b)
    x = I.normal(3, 2, (20000,))
    assert abs(x.mean()) < 0.03 and abs(x.std() - 1) < 0.03
    u = I.uniform(3, 2, (20000,), -1, 1)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.03
    W = I.band_dft(300, 16, 9, True)
    assert np.all(np.diff(W[0].real) >= 0) and np.all(W[0].imag == 0)
    v, tau = I.synthetic_store(50, 6, 1, True)
    V = v.reshape(-1, 6)
    nrm2 = np.sum(np.abs(V) ** 2, axis=1)
    # unitary: 2 Re(tau) = |tau|^2 |v|^2
    assert np.abs(2 * tau.real - np.abs(tau) ** 2 * nrm2).max() < 1e-13


def test_batch_argument_checks_fail_before_any_device_work(L):
    from paper_2002_10991_gb300.api import Problem

    EINVAL = 1
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(16)
    good = Problem(0, 0, 10, 4, 5, 16, 16, 16, 10)
    arr = (Problem * 2)(good, Problem(0, 0, 10, 4, 11, 16, 16, 16, 10))  # nev > n
    assert L.tbbt_batch_create(ctypes.byref(h), 2, ctypes.cast(arr, ctypes.c_void_p), None) == EINVAL
    arr2 = (Problem * 1)(Problem(7, 0, 10, 4, 5, 16, 16, 16, 10))  # bad dtype
    assert L.tbbt_batch_create(ctypes.byref(h), 1, ctypes.cast(arr2, ctypes.c_void_p), None) == EINVAL
    arr3 = (Problem * 1)(Problem(1, 0, 10, 4, 5, 16, 16, 24, 10))  # complex q not 16-byte aligned
    assert L.tbbt_batch_create(ctypes.byref(h), 1, ctypes.cast(arr3, ctypes.c_void_p), None) == EINVAL
    assert L.tbbt_batch_create(ctypes.byref(h), 0, fake, None) == EINVAL
    assert L.tbbt_batch_create(None, 1, fake, None) == EINVAL
    assert L.tbbt_batch_execute(None, None) == EINVAL
    assert L.tbbt_batch_destroy(None) == 0


def test_band_to_full_argument_checks(L):
    # rejected (or a no-op) on the host, before any CUDA call
    buf = (ctypes.c_double * 4)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    EINVAL = 1
    for f in (L.tbbt_trans_ev_band_to_full_d, L.tbbt_trans_ev_band_to_full_z, L.tbbt_trans_ev_band_to_full_split_d):
        assert f(p, 10, p, 10, 0, 5, p, 10, None) == EINVAL  # nbw < 1
        assert f(p, 10, p, 10, 4, 11, p, 10, None) == EINVAL  # nev > n
        assert f(p, 10, p, 10, 4, -1, p, 10, None) == EINVAL  # nev < 0
        assert f(p, 9, p, 10, 4, 5, p, 10, None) == EINVAL  # lda < n
        assert f(p, 10, p, 10, 4, 5, p, 9, None) == EINVAL  # ldq < n
        assert f(p, 10, p, -1, 4, 0, p, 10, None) == EINVAL  # n < 0
        assert f(None, 10, p, 10, 4, 5, p, 10, None) == EINVAL  # null a
        assert f(p, 10, None, 10, 4, 5, p, 10, None) == EINVAL  # null tau
        assert f(p, 10, p, 10, 4, 5, None, 10, None) == EINVAL  # null q
        assert f(None, 10, None, 10, 10, 5, None, 10, None) == 0  # nbw >= n: identity, nothing to do
        assert f(None, 10, None, 10, 4, 0, None, 10, None) == 0  # nev = 0
        assert f(None, 1, None, 0, 4, 0, None, 1, None) == 0  # n = 0
    odd = ctypes.c_void_p(ctypes.addressof(buf) + 4)
    assert L.tbbt_trans_ev_band_to_full_d(p, 10, p, 10, 4, 5, odd, 10, None) == EINVAL  # misaligned q
    assert L.tbbt_trans_ev_band_to_full_split_d(p, 10, p, 10, 4, 5, odd, 10, None) == EINVAL
    f = L.tbbt_trans_ev_band_to_full_split_opts_d
    assert f(p, 10, p, 10, 4, 5, p, 10, -1, -1, None) == EINVAL  # negative wait limit
    assert f(p, 10, p, 10, 4, 5, p, 10, 0, -2, None) == EINVAL  # withhold index below -1
    assert f(p, 10, p, 10, 0, 5, p, 10, 0, -1, None) == EINVAL  # nbw < 1
    assert f(None, 10, None, 10, 10, 5, None, 10, 0, -1, None) == 0  # nbw >= n: nothing to do


def test_bulge_chase_shape_limits_on_the_host(L):
    # rejected before any CUDA call: the shared-memory form holds the b x b
    # diagonal block, which caps a Hermitian band at nbw = 117
    buf = (ctypes.c_double * 8)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    ENOTSUP, EINVAL = 5, 1
    assert L.tbbt_bulge_chase_z(p, 119, 200, 118, p, p, p, p, None) == ENOTSUP
    assert L.tbbt_bulge_chase_d(p, 129, 200, 129, p, p, p, p, None) == EINVAL  # nbw > 128
    assert L.tbbt_bulge_chase_d(p, 4, 0, 3, None, None, None, None, None) == 0  # n = 0: nothing to do


def test_tridiag_eig_argument_checks(L):
    # rejected (or a no-op) on the host, before any CUDA call
    buf = (ctypes.c_double * 8)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    EINVAL = 1
    f = L.tbbt_tridiag_eig
    assert f(p, p, -1, 0, p, p, 1, 0, None) == EINVAL  # n < 0
    assert f(p, p, 10, 11, p, p, 10, 0, None) == EINVAL  # nev > n
    assert f(p, p, 10, -1, p, p, 10, 0, None) == EINVAL  # nev < 0
    assert f(p, p, 10, 5, p, p, 9, 0, None) == EINVAL  # ldx < n
    assert f(p, p, 10, 5, p, p, 10, 7, None) == EINVAL  # xtype
    assert f(None, p, 10, 5, p, p, 10, 0, None) == EINVAL  # null d
    assert f(p, None, 10, 5, p, p, 10, 0, None) == EINVAL  # null e with n > 1
    assert f(p, p, 10, 5, None, p, 10, 0, None) == EINVAL  # null w
    assert f(p, p, 10, 5, p, None, 10, 0, None) == EINVAL  # null x
    odd = ctypes.c_void_p(ctypes.addressof(buf) + 8)
    assert f(p, p, 10, 5, p, odd, 10, 1, None) == EINVAL  # complex x not 16-byte aligned
    assert f(None, None, 10, 0, None, None, 10, 0, None) == 0  # nev = 0: nothing to do
    assert f(None, None, 0, 0, None, None, 1, 0, None) == 0  # n = 0


def test_fp64_probe_argument_checks(L):
    buf = (ctypes.c_double * 8)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    fl = ctypes.c_double()
    EINVAL = 1
    f = L.tbbt_fp64_probe
    assert f(2, 1, 32, 1, p, ctypes.byref(fl), None) == EINVAL  # kind
    assert f(0, 0, 32, 1, p, ctypes.byref(fl), None) == EINVAL  # blocks
    assert f(0, 1, 48, 1, p, ctypes.byref(fl), None) == EINVAL  # threads not a multiple of 32
    assert f(0, 1, 32, 0, p, ctypes.byref(fl), None) == EINVAL  # iters
    assert f(0, 1, 32, 1, None, ctypes.byref(fl), None) == EINVAL  # sink
