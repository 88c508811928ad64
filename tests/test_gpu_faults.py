"""Failure detection on the GPU without a GPU fault.

The apply kernel's only waits are bounded waits for the progress of the work
unit ahead in the same strip. A test hook withholds one unit's progress so
that the unit behind it must give up: the kernel records TBBT_ETIMEOUT,
abandons the dependent work, exits normally, and the context stays usable.
"""

import numpy as np
import pytest

import oracle
from paper_2002_10991_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2002_10991_gb300 import _native

    _native.build()
    import paper_2002_10991_gb300 as P

    return P


def test_withheld_progress_times_out_and_context_survives(P):
    n, b, nev = 600, 16, 64  # 2 strips, ceil(37 / 8) = 5 epochs each
    v, tau = I.synthetic_store(n, b, 3, False)
    X = I.eigvec_block(n, nev, 4, False)
    dv, dt = torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda()
    plan = P.Plan(False, n, b, nev, sweeps_per_block=8, stages_per_step=4, wait_timeout_ms=300,
                  debug_withhold_unit=0)
    plan.set_reflectors(dv, dt)
    q = torch.from_numpy(X.T.copy()).cuda().t()
    plan.execute(q)
    with pytest.raises(P.TbbtError) as ei:
        P.stream_check()
    assert ei.value.status == 4  # TBBT_ETIMEOUT
    plan.close()
    # the error word was cleared and the device still computes correctly
    P.stream_check()
    good = P.Plan(False, n, b, nev)
    good.set_reflectors(dv, dt)
    q = torch.from_numpy(X.T.copy()).cuda().t()
    good.execute(q)
    P.stream_check()
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"))
    assert np.abs(q.cpu().numpy() - Zo).max() <= 1e-11
    good.close()


def test_withheld_progress_times_out_tcgen05_split(P):
    # the tensor-core split form: the unit behind the withheld one gives up at
    # its first wait, the others abandon their units mid-way (their waits see
    # the error word); every block drains its copies and MMAs, frees its
    # tensor memory and exits
    n, b, nev = 600, 64, 300  # 3 strips of 128 columns, 10 sweeps
    v, tau = I.synthetic_store(n, b, 5, False)
    X = I.eigvec_block(n, nev, 6, False)
    dv, dt = torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda()
    plan = P.Plan(False, n, b, nev, wait_timeout_ms=300, debug_withhold_unit=0, variant=2)
    plan.set_reflectors(dv, dt)
    q = torch.from_numpy(X.T.copy()).cuda().t()
    plan.execute(q)
    with pytest.raises(P.TbbtError) as ei:
        P.stream_check()
    assert ei.value.status == 4  # TBBT_ETIMEOUT
    plan.close()
    P.stream_check()
    good = P.Plan(False, n, b, nev, variant=2)
    good.set_reflectors(dv, dt)
    q = torch.from_numpy(X.T.copy()).cuda().t()
    good.execute(q)
    P.stream_check()
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"))
    assert np.abs(q.cpu().numpy() - Zo).max() <= 1e-11
    good.close()


def test_withheld_w_publication_times_out_split_band_to_full(P):
    # the split band -> full form: CTA 1 (strip 0, slot 1) publishes its
    # partial W but is never counted in, so the slots of strip 0 give up
    # after 300 ms; every CTA drains its copies and products, frees its
    # tensor memory and exits, and the next call computes correctly
    n, b, nev = 600, 64, 300  # 3 strips of 128 columns, 8 slots each
    a, tau = I.synthetic_full_store(n, b, 21, False)
    Y = I.eigvec_block(n, nev, 22, False)
    da = torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()
    dt = torch.from_numpy(tau).cuda()
    q = torch.from_numpy(np.ascontiguousarray(Y.T)).cuda().t()
    P.trans_ev_band_to_full(da, dt, n, b, nev, q, variant=2, wait_timeout_ms=300, debug_withhold_cta=1)
    with pytest.raises(P.TbbtError) as ei:
        P.stream_check()
    assert ei.value.status == 4  # TBBT_ETIMEOUT
    P.stream_check()  # the error word was cleared
    q = torch.from_numpy(np.ascontiguousarray(Y.T)).cuda().t()
    P.trans_ev_band_to_full(da, dt, n, b, nev, q, variant=2)
    P.stream_check()
    Co = oracle.back_transform_full(a, tau, n, b, np.asfortranarray(Y.copy()), nthreads=8)
    assert np.abs(q.cpu().numpy() - Co).max() <= 1e-11
