"""GPU parity: the CUDA library against the CPU oracle on identical inputs.

Every test calls the library through its C ABI (via the thin Python binding)
and compares element by element with the oracle's reflector-by-reflector
back-transform (Eq. 6d / Eq. 8). Tolerance: max |z_gpu - z_oracle| <= 1e-11
on columns of unit norm (modulus for complex entries). The two sides sum each
v^H x in the same ascending order but the GPU fuses multiply-adds, so the
results differ by rounding only.
"""

import numpy as np
import pytest

import oracle
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a) if a.ndim == 1 else a).cuda()


def gpu_apply(P, v, tau, n, b, X, nev=None):
    """Copy X (Fortran (ldq, nev)) to the device, apply, copy back."""
    nev = X.shape[1] if nev is None else nev
    q = torch.from_numpy(np.asfortranarray(X).T.copy()).cuda().t()  # column-major view
    assert q.numel() == 0 or q.shape[1] == 1 or q.stride(0) == 1
    P.trans_ev_tridi_to_band(dev(v), dev(tau), n, b, nev, q, ldq=X.shape[0])
    P.stream_check()
    return np.asfortranarray(q.cpu().numpy())


def maxdiff(a, b):
    return float(np.max(np.abs(a - b))) if a.size else 0.0


# ---------------------------------------------------------------------------
# the whole chain at the plain-method size (N=512, b=32, all eigenvectors)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("cplx", [False, True])
def test_chain_n512_b32_all_eigenvectors(P, cplx):
    n, b = 512, 32
    W = I.band_uniform(n, b, I.SEED_BASE + 1, cplx)
    v, tau, d, e = oracle.bulge_chase(W)
    lam, Xr = oracle.tridiag_ql(d, e)
    X = np.asfortranarray(Xr.astype(W.dtype))
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"), nthreads=8)
    Zg = gpu_apply(P, v, tau, n, b, X)
    assert maxdiff(Zg, Zo) <= TOL
    A = I.band_to_dense(W)
    res = np.linalg.norm(A @ Zg - Zg * lam) / (np.linalg.norm(A) * n * np.finfo(float).eps)
    assert res <= 10
    assert np.abs(Zg.conj().T @ Zg - np.eye(n)).max() <= 1e-12


# ---------------------------------------------------------------------------
# shapes: tiles, ragged tails, degenerate sizes, every band width class
# ---------------------------------------------------------------------------

SHAPES = [
    # n, b, nev, extra ldq rows
    (0, 4, 0, 0), (1, 1, 1, 0), (2, 1, 2, 1), (2, 3, 1, 0), (3, 1, 3, 0), (3, 8, 2, 2), (5, 2, 5, 0),
    (17, 4, 12, 0), (17, 4, 17, 3), (33, 5, 33, 0), (40, 1, 9, 0), (64, 63, 31, 1), (65, 64, 65, 0),
    (100, 3, 33, 2), (129, 32, 70, 0), (200, 16, 1, 0), (257, 32, 97, 5), (300, 128, 64, 0),
    (301, 127, 65, 0), (400, 64, 129, 0), (513, 33, 257, 1),
]


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b,nev,pad", SHAPES)
def test_shapes_synthetic_store(P, n, b, nev, pad, cplx):
    v, tau = I.synthetic_store(n, b, 1000 + n * 7 + b, cplx)
    X = I.eigvec_block(n, nev, 2000 + n + b, cplx, ldq=max(n + pad, 1))
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"), nthreads=4)
    Zg = gpu_apply(P, v, tau, n, b, X)
    assert maxdiff(Zg[:n], Zo[:n]) <= TOL
    if pad:
        assert np.all(np.isnan(Zg[n:]))  # rows n..ldq-1 untouched


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b,nev", [(97, 7, 40), (256, 32, 100), (500, 64, 77)])
def test_shapes_bulge_chased_store(P, n, b, nev, cplx):
    W = I.band_dft(n, b, 31 + n, cplx)
    v, tau, d, e = oracle.bulge_chase(W)
    X = I.eigvec_block(n, nev, 5 + n, cplx)
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"), nthreads=4)
    Zg = gpu_apply(P, v, tau, n, b, X)
    assert maxdiff(Zg, Zo) <= TOL


@pytest.mark.parametrize("cplx", [False, True])
def test_identity_store_is_exact(P, cplx):
    n, b, nev = 300, 32, 50
    v, tau = I.synthetic_store(n, b, 4, cplx)
    tau[:] = 0
    X = I.eigvec_block(n, nev, 5, cplx)
    Zg = gpu_apply(P, v, tau, n, b, X)
    assert np.array_equal(Zg, X)


@pytest.mark.parametrize("cplx", [False, True])
def test_launch_geometry_does_not_change_bits(P, cplx):
    # Every element sees the same sequence of operations whatever the number
    # of concurrent sweeps or the step length, so results agree bitwise.
    n, b, nev = 700, 64, 70
    v, tau = I.synthetic_store(n, b, 8, cplx)
    X = I.eigvec_block(n, nev, 9, cplx)
    outs = []
    for G, NB in [(1, 1), (2, 3), (3, 8), (4, 4), (8, 8), (16, 2)]:
        plan = P.Plan(cplx, n, b, nev, sweeps_per_block=G, stages_per_step=NB)
        plan.set_reflectors(dev(v), dev(tau))
        q = torch.from_numpy(X.T.copy()).cuda().t()
        plan.execute(q)
        P.stream_check()
        outs.append(q.cpu().numpy())
        plan.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"), nthreads=4)
    assert maxdiff(outs[0], Zo) <= TOL


@pytest.mark.parametrize("b", [32, 64])
def test_register_window_matches_shared_window_bitwise(P, b):
    # real b = 32 / 64 plans keep each column's window in registers; the
    # allocation-free entry point runs the shared-memory window kernel. Both
    # apply the same operations in the same order.
    n, nev = 1500, 200
    v, tau = I.synthetic_store(n, b, 40 + b, False)
    X = I.eigvec_block(n, nev, 41 + b, False)
    reg = gpu_apply(P, v, tau, n, b, X)
    q = torch.from_numpy(X.T.copy()).cuda().t()
    P.trans_ev_tridi_to_band_noalloc(dev(v), dev(tau), n, b, nev, q)
    P.stream_check()
    assert np.array_equal(reg, q.cpu().numpy())


def test_repeat_runs_bitwise_identical(P):
    n, b, nev = 1000, 64, 200
    v, tau = I.synthetic_store(n, b, 11, False)
    X = I.eigvec_block(n, nev, 12, False)
    a = gpu_apply(P, v, tau, n, b, X)
    c = gpu_apply(P, v, tau, n, b, X)
    assert np.array_equal(a, c)


def test_plan_reuse_with_new_reflectors(P):
    n, b, nev = 333, 32, 45
    plan = P.Plan(False, n, b, nev)
    for seed in (1, 2):
        v, tau = I.synthetic_store(n, b, seed, False)
        X = I.eigvec_block(n, nev, seed + 10, False)
        plan.set_reflectors(dev(v), dev(tau))
        q = torch.from_numpy(X.T.copy()).cuda().t()
        plan.execute(q)
        P.stream_check()
        Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"))
        assert maxdiff(q.cpu().numpy(), Zo) <= TOL
    plan.close()


def test_smaller_plan_does_not_break_earlier_plan(P):
    # plans share the kernel; a later plan with less shared memory must not
    # invalidate the launch configuration of an earlier one
    n, b, nev = 400, 64, 40
    big = P.Plan(False, n, b, nev)
    small = P.Plan(False, 100, 4, 10, sweeps_per_block=1, stages_per_step=1)
    assert big.info()["smem_bytes"] > small.info()["smem_bytes"]
    v, tau = I.synthetic_store(n, b, 31, False)
    X = I.eigvec_block(n, nev, 32, False)
    big.set_reflectors(dev(v), dev(tau))
    q = torch.from_numpy(X.T.copy()).cuda().t()
    big.execute(q)
    P.stream_check()
    Zo = oracle.back_transform(v, tau, n, b, X.copy(order="F"))
    assert maxdiff(q.cpu().numpy(), Zo) <= TOL
    big.close()
    small.close()


@pytest.mark.parametrize("cplx", [False, True])
def test_host_buffer_entry_point_matches_device_path(P, cplx):
    n, b, nev = 600, 64, 90
    v, tau = I.synthetic_store(n, b, 21, cplx)
    X = I.eigvec_block(n, nev, 22, cplx, ldq=n + 2)
    Zd = gpu_apply(P, v, tau, n, b, X)
    Zh = X.copy(order="F")
    P.trans_ev_tridi_to_band_host(v, tau, n, b, nev, Zh)
    assert np.array_equal(Zh[:n], Zd[:n])
    assert np.all(np.isnan(Zh[n:]))


# ---------------------------------------------------------------------------
# full sizes of the named workloads, on sampled columns
# ---------------------------------------------------------------------------

def sample_columns(nev, k, seed):
    rng = np.random.default_rng(seed)
    cols = set([0, 31, 32, nev - 1, nev - 32, nev // 2])
    cols |= set(rng.choice(nev, size=min(k, nev), replace=False).tolist())
    return np.array(sorted(c for c in cols if 0 <= c < nev))


def test_full_size_real_n8192_b64_nev4096_synthetic_store(P):
    w = I.WORKLOADS["real-n8192-b64-dft"]
    n, b, nev = w["n"], w["b"], w["nev"]
    v, tau = I.synthetic_store(n, b, w["seed"], False)
    X = I.eigvec_block(n, nev, w["seed"], False)
    Zg = gpu_apply(P, v, tau, n, b, X)
    cols = sample_columns(nev, 40, 3)
    Zo = oracle.back_transform(v, tau, n, b, np.asfortranarray(X[:, cols]), nthreads=oracle.num_cpus())
    assert maxdiff(Zg[:, cols], Zo) <= TOL
    # unitary invariance on every column
    ratio = np.linalg.norm(Zg, axis=0) / np.linalg.norm(X, axis=0)
    assert np.abs(ratio - 1).max() <= 1e-12


@pytest.mark.slow
def test_full_size_real_n8192_b64_bulge_chased_store(P):
    w = I.WORKLOADS["real-n8192-b64-dft"]
    n, b, nev = w["n"], w["b"], w["nev"]
    v, tau, d, e = oracle.bulge_chase(I.band_for("real-n8192-b64-dft"))
    X = I.eigvec_block(n, nev, w["seed"] + 100, False)
    Zg = gpu_apply(P, v, tau, n, b, X)
    cols = sample_columns(nev, 24, 4)
    Zo = oracle.back_transform(v, tau, n, b, np.asfortranarray(X[:, cols]), nthreads=oracle.num_cpus())
    assert maxdiff(Zg[:, cols], Zo) <= TOL


def test_full_size_complex_n20000_b64_nev6000_synthetic_store(P):
    w = I.WORKLOADS["complex-n20000-b64-dft"]
    n, b, nev = w["n"], w["b"], w["nev"]
    v, tau = I.synthetic_store(n, b, w["seed"], True)
    X = I.eigvec_block(n, nev, w["seed"], True)
    Zg = gpu_apply(P, v, tau, n, b, X)
    cols = sample_columns(nev, 6, 5)
    Zo = oracle.back_transform(v, tau, n, b, np.asfortranarray(X[:, cols]), nthreads=oracle.num_cpus())
    assert maxdiff(Zg[:, cols], Zo) <= TOL
    ratio = np.linalg.norm(Zg, axis=0) / np.linalg.norm(X, axis=0)
    assert np.abs(ratio - 1).max() <= 1e-12
