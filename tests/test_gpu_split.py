"""Split-precision variants (BF16 tensor cores, exact digit slices, 64-bit
fixed point; warp-level mma.sync and tcgen05 with tensor memory): results
against the FP64 oracle. The error budget is relative
to each column's norm (the fixed-point scale): about 2^-48 per block
application before accumulation; the bound used here is the FP64 parity
bound, 1e-11 on unit-norm columns, and the chain test checks the residual and
orthogonality bounds of the benchmark definition."""

import numpy as np
import pytest

import oracle
from paper_2002_10991_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-11
SPLIT, SPLIT_TC = 1, 2


@pytest.fixture(scope="module")
def P():
    from paper_2002_10991_gb300 import _native

    _native.build()
    import paper_2002_10991_gb300 as P

    assert torch.cuda.is_available()
    return P


@pytest.fixture(params=[SPLIT, SPLIT_TC], ids=["mma_sync", "tcgen05"])
def variant(request):
    return request.param


def run_split(P, v, tau, n, b, X, variant):
    nev = X.shape[1]
    plan = P.Plan(False, n, b, nev, variant=variant, wait_timeout_ms=5000)
    plan.set_reflectors(torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda())
    q = torch.from_numpy(np.asfortranarray(X).T.copy()).cuda().t()
    plan.execute(q, ldq=X.shape[0])
    P.stream_check()
    out = q.cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("n,b,nev,pad", [(40, 32, 7, 0), (100, 32, 33, 2), (257, 64, 65, 0), (600, 64, 130, 1),
                                        (1000, 32, 64, 0), (2048, 64, 200, 0)])
def test_split_matches_oracle(P, variant, n, b, nev, pad):
    v, tau = I.synthetic_store(n, b, 70 + n + b, False)
    X = I.eigvec_block(n, nev, 71 + n, False, ldq=n + pad)
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"), nthreads=8)
    Zs = run_split(P, v, tau, n, b, X, variant)
    err = np.abs(Zs[:n] - Zo[:n]).max()
    assert err <= TOL, err
    if pad:
        assert np.all(np.isnan(Zs[n:]))


def test_split_bulge_chased_chain_n512(P, variant):
    n, b = 512, 32
    W = I.band_uniform(n, b, I.SEED_BASE + 1, False)
    v, tau, d, e = oracle.bulge_chase(W)
    lam, Xr = oracle.tridiag_ql(d, e)
    X = np.asfortranarray(Xr)
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"), nthreads=8)
    Zs = run_split(P, v, tau, n, b, X, variant)
    assert np.abs(Zs - Zo).max() <= TOL
    A = I.band_to_dense(W)
    nrmB = np.abs(lam).max()
    res = np.linalg.norm(A @ Zs - Zs * lam, axis=0).max() / nrmB
    assert res <= 1e-12, res
    assert np.abs(Zs.T @ Zs - np.eye(n)).max() <= 1e-12


def test_split_dft_store_n2048(P, variant):
    n, b, nev = 2048, 64, 256
    v, tau, d, e = oracle.bulge_chase(I.band_dft(n, b, 91, False))
    X = I.eigvec_block(n, nev, 92, False)
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"), nthreads=8)
    Zs = run_split(P, v, tau, n, b, X, variant)
    assert np.abs(Zs - Zo).max() <= TOL


def test_split_identity_store_round_trip(P, variant):
    n, b, nev = 300, 64, 40
    v, tau = I.synthetic_store(n, b, 5, False)
    tau[:] = 0
    X = I.eigvec_block(n, nev, 6, False)
    Zs = run_split(P, v, tau, n, b, X, variant)
    # only the fixed-point round trip: within 2^-60 of each column's norm
    assert np.abs(Zs - X).max() <= 2.0 ** -58


def test_split_rejects_unsupported_shapes(P, variant):
    with pytest.raises(P.TbbtError) as ei:
        P.Plan(True, 100, 32, 10, variant=variant)
    assert ei.value.status == 5
    with pytest.raises(P.TbbtError):
        P.Plan(False, 100, 16, 10, variant=variant)


def test_split_full_size_n32768_sampled_columns(P, variant):
    # the precision form's own workload: n=32768, b=64, nev=0.3 n
    w = I.WORKLOADS["real-n32768-b64-dft"]
    n, b, nev = w["n"], w["b"], w["nev"]
    v, tau = I.synthetic_store(n, b, w["seed"], False)
    X = I.eigvec_block(n, nev, w["seed"], False)
    Zs = run_split(P, v, tau, n, b, X, variant)
    rng = np.random.default_rng(7)
    cols = np.unique(np.concatenate([[0, 63, 64, nev - 1], rng.choice(nev, 4, replace=False)]))
    Zo = oracle.back_transform(v, tau, n, b, np.asfortranarray(X[:, cols]), nthreads=oracle.num_cpus())
    assert np.abs(Zs[:, cols] - Zo).max() <= TOL
    ratio = np.linalg.norm(Zs, axis=0) / np.linalg.norm(X, axis=0)
    assert np.abs(ratio - 1).max() <= 1e-12


@pytest.mark.parametrize("n,b,nev", [(3, 32, 1), (34, 32, 1), (35, 32, 3), (66, 64, 2), (200, 64, 129), (130, 64, 128),
                                     (300, 64, 257), (700, 32, 385)])
def test_split_edge_shapes(P, variant, n, b, nev):
    # one sweep / one block / partial strips / several 128-column strips with a ragged tail
    v, tau = I.synthetic_store(n, b, 300 + n + nev, False)
    X = I.eigvec_block(n, nev, 301 + n, False)
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"), nthreads=8)
    Zs = run_split(P, v, tau, n, b, X, variant)
    assert np.abs(Zs - Zo).max() <= TOL


def test_split_tc_matches_mma_sync_variant(P):
    # two implementations of the same arithmetic: equal up to the digit truncation
    n, b, nev = 1500, 64, 300
    v, tau = I.synthetic_store(n, b, 17, False)
    X = I.eigvec_block(n, nev, 18, False)
    Z1 = run_split(P, v, tau, n, b, X, SPLIT)
    Z2 = run_split(P, v, tau, n, b, X, SPLIT_TC)
    assert np.abs(Z1 - Z2).max() <= 2e-13


def test_split_tc_replay_is_deterministic(P):
    n, b, nev = 900, 32, 260
    v, tau = I.synthetic_store(n, b, 23, False)
    X = I.eigvec_block(n, nev, 24, False)
    plan = P.Plan(False, n, b, nev, variant=SPLIT_TC, wait_timeout_ms=5000)
    plan.set_reflectors(torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda())
    outs = []
    for _ in range(2):
        q = torch.from_numpy(np.asfortranarray(X).T.copy()).cuda().t()
        plan.execute(q, ldq=n)
        P.stream_check()
        outs.append(q.cpu().numpy())
    plan.close()
    assert np.array_equal(outs[0], outs[1])
