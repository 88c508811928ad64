"""Batched form: many problems of uneven size, real and complex mixed, in one
persistent launch replayed from a CUDA graph. Each problem's result is
compared with the oracle, and with the single-problem plan (same operations
in the same order, so the same bits)."""

import os

import numpy as np
import pytest

import oracle
from paper_2002_10991_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-11

MIX = [
    # n, b, nev, complex
    (300, 32, 150, False), (500, 64, 77, False), (200, 16, 40, False), (400, 32, 100, True),
    (150, 8, 150, True), (2, 4, 2, False), (60, 32, 0, False), (257, 64, 33, True), (1, 1, 1, True),
    (700, 32, 350, False),
]


@pytest.fixture(scope="module")
def P():
    from paper_2002_10991_gb300 import _native

    _native.build()
    import paper_2002_10991_gb300 as P

    assert torch.cuda.is_available()
    return P


def col_major(X):
    return torch.from_numpy(np.asfortranarray(X).T.copy()).cuda().t() if X.size else \
        torch.zeros((X.shape[0], X.shape[1]), dtype=torch.complex128 if np.iscomplexobj(X) else torch.float64,
                    device="cuda")


def make(mix, seed0=100):
    probs, host = [], []
    for i, (n, b, nev, c) in enumerate(mix):
        v, tau = I.synthetic_store(n, b, seed0 + i, c)
        X = I.eigvec_block(n, nev, seed0 + 50 + i, c)
        dv = torch.from_numpy(v).cuda() if v.size else torch.zeros(1, dtype=torch.complex128 if c else torch.float64,
                                                                    device="cuda")
        dt = torch.from_numpy(tau).cuda() if tau.size else torch.zeros(1, dtype=dv.dtype, device="cuda")
        probs.append((dv, dt, n, b, nev, col_major(X)))
        host.append((v, tau, X))
    return probs, host


def oracle_result(v, tau, n, b, X, times=1):
    Z = X.copy(order="F")
    for _ in range(times):
        if Z.size:
            oracle.back_transform(v, tau, n, b, Z, nthreads=4)
    return Z


def test_batch_matches_oracle_and_plans(P):
    probs, host = make(MIX)
    batch = P.Batch(probs)
    info = batch.info()
    assert info["units"] > 0 and info["blocks"] > 0
    batch.execute()
    P.stream_check()
    for (dv, dt, n, b, nev, q), (v, tau, X) in zip(probs, host):
        got = q.cpu().numpy()
        assert np.abs(got - oracle_result(v, tau, n, b, X)).max(initial=0) <= TOL, (n, b, nev)
        if nev and n:
            plan = P.Plan(np.iscomplexobj(X), n, b, nev)
            plan.set_reflectors(dv, dt)
            q2 = col_major(X)
            plan.execute(q2)
            P.stream_check()
            if np.iscomplexobj(X):
                # the single-problem complex kernel sums v^H x in two halves
                # (a lane pair per column), the batched one in one chain
                assert np.abs(q2.cpu().numpy() - got).max() <= TOL, (n, b, nev)
            else:
                assert np.array_equal(q2.cpu().numpy(), got), (n, b, nev)
            plan.close()
    batch.close()


def test_batch_replays_apply_again(P):
    mix = MIX[:4]
    probs, host = make(mix, seed0=300)
    batch = P.Batch(probs, stages_per_step_real=4, stages_per_step_complex=4)
    batch.execute()
    batch.execute()
    P.stream_check()
    for (dv, dt, n, b, nev, q), (v, tau, X) in zip(probs, host):
        assert np.abs(q.cpu().numpy() - oracle_result(v, tau, n, b, X, times=2)).max() <= TOL
    batch.close()


def test_batch_autotune_and_cache(P, tmp_path):
    mix = [(400, 32, 200, False), (300, 32, 150, True), (600, 32, 100, False)]
    cache = str(tmp_path / "tune.txt")
    probs, host = make(mix, seed0=500)
    batch = P.Batch(probs, autotune=True, autotune_cache=cache)
    assert batch.info()["tuned"]
    assert os.path.exists(cache) and open(cache).read().strip()
    batch.execute()
    P.stream_check()
    for (dv, dt, n, b, nev, q), (v, tau, X) in zip(probs, host):
        assert np.abs(q.cpu().numpy() - oracle_result(v, tau, n, b, X)).max() <= TOL
    batch.close()
    # a second batch of the same shapes takes the tuned geometry from the cache
    probs2, host2 = make(mix, seed0=600)
    b2 = P.Batch(probs2, autotune=True, autotune_cache=cache)
    assert b2.info()["tuned"]
    b2.execute()
    P.stream_check()
    for (dv, dt, n, b, nev, q), (v, tau, X) in zip(probs2, host2):
        assert np.abs(q.cpu().numpy() - oracle_result(v, tau, n, b, X)).max() <= TOL
    b2.close()


def test_batch_full_size_64_mixed_sampled_columns(P):
    # the batched workload: 64 problems, N in [1000, 6000], nev = N/2, b = 32, half complex
    specs = I.batch_workload()
    probs, host = [], []
    for s in specs:
        n, b, nev, c = s["n"], s["b"], s["nev"], s["complex_"]
        v, tau = I.synthetic_store(n, b, s["seed"], c)
        X = I.eigvec_block(n, nev, s["seed"] + 1, c)
        probs.append((torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda(), n, b, nev, col_major(X)))
        host.append((v, tau, X))
    batch = P.Batch(probs)
    batch.execute()
    P.stream_check()
    rng = np.random.default_rng(11)
    for (dv, dt, n, b, nev, q), (v, tau, X) in zip(probs, host):
        # 16 columns per problem: both ends, a strip boundary, the rest random
        cols = np.unique(np.concatenate([[0, 31, 32, nev - 1], rng.choice(nev, 12, replace=False)]))
        got = q[:, torch.from_numpy(cols).cuda()].cpu().numpy()
        Zo = oracle.back_transform(v, tau, n, b, np.asfortranarray(X[:, cols]), nthreads=oracle.num_cpus())
        assert np.abs(got - Zo).max() <= TOL, (n, b, nev)
    batch.close()
