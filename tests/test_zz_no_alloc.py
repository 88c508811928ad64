"""The entry point that allocates nothing (tbbt_trans_ev_tridi_to_band_noalloc).

It serves callers that cannot allocate device memory when they call (the
GPU's memory belongs to another allocator, or the host-device
synchronisation of cudaMalloc/cudaFree is not acceptable in their loop). Its
scratch is one fixed array per device that every call reuses, so these tests
call it twice in a row and compare each result with the allocating entry
point's, within the parity tolerance of the other GPU tests. The file is
named to be collected last; it passes alone in a fresh process and after the
other tests.
"""

import numpy as np
import pytest

from paper_2002_10991_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module")
def P():
    from paper_2002_10991_gb300 import _native

    _native.build()
    import paper_2002_10991_gb300 as P

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return P


def col_major(X):
    return torch.from_numpy(np.asfortranarray(X).T.copy()).cuda().t()


def run_both(P, n, b, nev, cplx, seed, ldq_pad=0):
    v, tau = I.synthetic_store(n, b, seed, cplx)
    X = I.eigvec_block(n, nev, seed + 1, cplx, ldq=n + ldq_pad)
    dv, dt = torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda()
    q_ref = col_major(X)
    P.trans_ev_tridi_to_band(dv, dt, n, b, nev, q_ref, ldq=X.shape[0])
    q_new = col_major(X)
    P.trans_ev_tridi_to_band_noalloc(dv, dt, n, b, nev, q_new, ldq=X.shape[0])
    P.stream_check()
    a, c = q_ref.cpu().numpy(), q_new.cpu().numpy()
    return a[:n], c[:n], c[n:]


@pytest.mark.parametrize("cplx", [False, True])
def test_noalloc_matches_allocating_entry_point_twice_in_a_row(P, cplx):
    # two different problems back to back: the second call starts from the
    # scratch contents the first one left behind
    for n, b, nev, seed, pad in [(1500, 64, 333, 5, 0), (1000, 32, 129, 9, 3)]:
        ref, got, tail = run_both(P, n, b, nev, cplx, seed, pad)
        assert np.abs(got - ref).max() <= TOL
        if pad:
            assert np.all(np.isnan(tail))


@pytest.mark.parametrize("cplx", [False, True])
def test_noalloc_small_call_then_larger_call(P, cplx):
    # the second problem needs more store, stage offsets and progress flags
    # than the first left in the array: stale tails must not leak into it
    big = (1800, 64, 500, 13, 2) if cplx else (2000, 64, 500, 13, 2)
    for n, b, nev, seed, pad in [(1000, 32, 129, 11, 0), big]:
        ref, got, tail = run_both(P, n, b, nev, cplx, seed, pad)
        assert np.abs(got - ref).max() <= TOL
        if pad:
            assert np.all(np.isnan(tail))


@pytest.mark.parametrize("cplx", [False, True])
def test_noalloc_matches_the_oracle(P, cplx):
    import oracle

    n, b, nev, seed = 700, 64, 150, 17
    v, tau = I.synthetic_store(n, b, seed, cplx)
    X = I.eigvec_block(n, nev, seed + 1, cplx)
    Zo = oracle.back_transform(v, tau, n, b, np.asfortranarray(X.copy()))
    q = col_major(X)
    P.trans_ev_tridi_to_band_noalloc(torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda(), n, b, nev, q)
    P.stream_check()
    assert np.abs(q.cpu().numpy() - Zo).max() <= TOL


def test_noalloc_rejects_problems_beyond_its_scratch(P):
    n, b, nev = 6000, 64, 64  # sweep-major store alone is about 140 MB
    v, tau = I.synthetic_store(n, b, 1, False)
    X = I.eigvec_block(n, nev, 2, False)
    q = col_major(X)
    with pytest.raises(P.TbbtError) as ei:
        P.trans_ev_tridi_to_band_noalloc(torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda(), n, b, nev, q)
    assert ei.value.status == 5  # TBBT_ENOTSUP
    assert np.array_equal(q.cpu().numpy(), X)  # nothing was touched
