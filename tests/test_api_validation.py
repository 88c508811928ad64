"""The Python binding rejects, before anything reaches the library, the
arguments that would make a kernel read outside the caller's memory: host
tensors given to a device entry point, element types that do not match, and
arrays shorter than the problem's geometry needs. No GPU is needed: every
case raises on the host."""

import pytest

torch = pytest.importorskip("torch")

import paper_2002_10991_gb300 as P  # noqa: E402
from paper_2002_10991_gb300 import _native  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    _native.build()


def f64(*shape):
    return torch.zeros(*shape, dtype=torch.float64)


def c128(*shape):
    return torch.zeros(*shape, dtype=torch.complex128)


def test_tridi_to_band_rejects_host_tensors_and_short_stores():
    n, b, nev = 40, 4, 5
    K = P.num_reflectors(n, b, False)
    q = f64(nev, n).t()
    with pytest.raises(ValueError, match="CUDA"):
        P.trans_ev_tridi_to_band(f64(K * b), f64(K), n, b, nev, q)
    with pytest.raises(ValueError, match="CUDA"):
        P.trans_ev_tridi_to_band_noalloc(f64(K * b), f64(K), n, b, nev, q)


def test_band_to_full_rejects_bad_arguments():
    n, b, nev = 10, 4, 3
    q = f64(nev, n).t()
    a = f64(n, n).t()
    with pytest.raises(ValueError, match="CUDA"):
        P.trans_ev_band_to_full(a, f64(n - b), n, b, nev, q)
    with pytest.raises(ValueError, match="rows"):
        P.trans_ev_band_to_full(f64(n, n - 1).t(), f64(n - b), n, b, nev, q)  # 9 rows
    with pytest.raises(ValueError, match="2-D"):
        P.trans_ev_band_to_full(f64(n * n), f64(n - b), n, b, nev, q)
    # the split-precision form takes real data only; variant 1 has no band -> full form
    with pytest.raises(ValueError, match="variant"):
        P.trans_ev_band_to_full(c128(n, n).t(), c128(n - b), n, b, nev, c128(nev, n).t(), variant=2)
    with pytest.raises(ValueError, match="variant"):
        P.trans_ev_band_to_full(a, f64(n - b), n, b, nev, q, variant=1)
    with pytest.raises(ValueError, match="CUDA"):
        P.trans_ev_band_to_full(a, f64(n - b), n, b, nev, q, variant=2)


def test_bulge_chase_rejects_host_and_short_bands():
    with pytest.raises(ValueError, match="CUDA"):
        P.bulge_chase(f64(20, 5).t())  # (5, 20): nbw = 4, n = 20
    with pytest.raises(ValueError, match="nbw\\+1"):
        P.bulge_chase(f64(20, 5).t(), nbw=8)
    with pytest.raises(ValueError, match="2-D"):
        P.bulge_chase(f64(20))


def test_validation_helpers_check_type_and_size():
    from paper_2002_10991_gb300 import api

    # the helpers' type and size rules, independent of device placement
    class FakeCuda:
        def __init__(self, t):
            self.t = t
            self.is_cuda = True
            self.dtype = t.dtype

        def numel(self):
            return self.t.numel()

        def is_contiguous(self):
            return self.t.is_contiguous()

    with pytest.raises(TypeError):
        api._need_flat(FakeCuda(c128(8)), "hh_v", torch.float64, 8)
    with pytest.raises(ValueError, match="at least 9"):
        api._need_flat(FakeCuda(f64(8)), "hh_v", torch.float64, 9)
    with pytest.raises(ValueError, match="contiguous"):
        api._need_flat(FakeCuda(f64(4, 4).t()), "hh_v", torch.float64, 16)
    api._need_flat(FakeCuda(f64(16)), "hh_v", torch.float64, 16)  # accepted
    api._need_device(f64(0), "empty", torch.float64, 0)  # nothing to read: accepted anywhere


def test_host_entry_point_checks_its_buffers():
    import numpy as np

    n, b, nev = 40, 4, 5
    K = P.num_reflectors(n, b, False)
    q = np.zeros((n, nev), order="F")
    with pytest.raises(ValueError, match="at least"):
        P.trans_ev_tridi_to_band_host(np.zeros(K * b - 1), np.zeros(K), n, b, nev, q)
    with pytest.raises(TypeError):
        P.trans_ev_tridi_to_band_host(np.zeros(K * b, np.complex128), np.zeros(K), n, b, nev, q)
    with pytest.raises(TypeError):
        P.trans_ev_tridi_to_band_host(f64(K * b), torch.zeros(K, dtype=torch.float32), n, b, nev, q)


def test_leading_dimension_must_match_the_view():
    from paper_2002_10991_gb300 import api

    n, nev = 40, 5
    q = f64(nev, n).t()  # column-major view, column stride n
    assert api._resolve_ldq(q, n, nev, None) == n
    assert api._resolve_ldq(q, n, nev, n) == n
    with pytest.raises(ValueError, match="column stride"):
        api._resolve_ldq(q, n, nev, n + 8)  # would reach 8 * (nev - 1) elements past q
    with pytest.raises(ValueError, match="column-major"):
        api._resolve_ldq(f64(n, nev), n, nev, n)  # row-major storage
    with pytest.raises(ValueError, match="column-major"):
        api._resolve_ldq(f64(n, 3)[:, :1], n, 1, None)  # one column of a row-major matrix
    with pytest.raises(ValueError, match="columns"):
        api._resolve_ldq(f64(nev - 1, n).t(), n, nev, None)
    with pytest.raises(ValueError, match="exceeds"):
        api._resolve_ldq(f64(1, n).t(), n, 1, n + 1)
    padded = f64(nev, n + 3).t()[:n]  # ldq = n + 3 > n rows of the view
    assert api._resolve_ldq(padded, n, nev, None) == n + 3


def test_host_entry_point_checks_the_leading_dimension():
    import numpy as np

    n, b, nev = 40, 4, 5
    K = P.num_reflectors(n, b, False)
    v, tau = np.zeros(K * b), np.zeros(K)
    q = np.zeros((n, nev), order="F")
    with pytest.raises(ValueError, match="leading dimension"):
        P.trans_ev_tridi_to_band_host(v, tau, n, b, nev, q, ldq=n + 8)  # the copies would overrun q
    with pytest.raises(ValueError, match="2-D"):
        P.trans_ev_tridi_to_band_host(v, tau, n, b, nev, np.zeros(n * nev))
    with pytest.raises(ValueError, match="Fortran"):
        P.trans_ev_tridi_to_band_host(v, tau, n, b, nev, np.zeros((n, nev)))
    with pytest.raises(ValueError, match="at least"):
        P.trans_ev_tridi_to_band_host(v, tau, n, b, nev, np.zeros((n, nev - 1), order="F"))
    with pytest.raises(ValueError, match="column stride"):
        P.trans_ev_tridi_to_band_host(torch.from_numpy(v), torch.from_numpy(tau), n, b, nev, f64(nev, n).t(),
                                      ldq=n + 1)
