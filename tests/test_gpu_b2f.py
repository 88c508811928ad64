"""Band -> full back-transformation on the GPU (Eq. 6e) against the oracle,
in FP64 and in the split-precision tensor-core form: element by element on
seeded stores (ragged blocks and strips, padded leading dimensions,
degenerate shapes), at the full n = 8192 size on sampled columns, and
through the chain whose eigenpairs belong to the dense matrix."""

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

    assert torch.cuda.is_available()
    return P


def dev_fortran(x, ld=None):
    """A column-major device tensor holding x (rows padded to ld)."""
    rows, cols = x.shape
    ld = rows if ld is None else ld
    buf = np.zeros((cols, ld), x.dtype)
    buf[:, :rows] = x.T
    return torch.from_numpy(buf).cuda().t()[:rows] if ld == rows else torch.from_numpy(buf).cuda().t()


def run_gpu(P, a, tau, n, b, Y, lda=None, ldq=None, variant=0):
    da = dev_fortran(a, lda)
    dt = torch.from_numpy(np.ascontiguousarray(tau)).cuda()
    dq = dev_fortran(Y, ldq)
    P.trans_ev_band_to_full(da, dt, n, b, Y.shape[1], dq, variant=variant)
    P.stream_check()
    return dq.cpu().numpy()[:n]


@pytest.mark.parametrize("n,b,nev,cplx", [(1, 1, 1, False), (2, 1, 2, False), (2, 1, 2, True), (5, 2, 3, True),
                                          (33, 1, 33, False), (100, 8, 37, True), (257, 32, 100, False),
                                          (300, 64, 300, True), (513, 64, 200, False), (200, 128, 50, False),
                                          (1000, 64, 500, False), (700, 5, 613, True), (64, 63, 9, False)])
def test_matches_oracle(P, n, b, nev, cplx):
    a, tau = I.synthetic_full_store(n, b, 1000 + n + b, cplx)
    Y = I.eigvec_block(n, nev, 7 + n, cplx)
    Co = oracle.back_transform_full(a, tau, n, b, np.asfortranarray(Y.copy()), nthreads=8)
    Cg = run_gpu(P, a, tau, n, b, Y)
    assert np.abs(Cg - Co).max() <= TOL


def test_padded_leading_dimensions(P):
    n, b, nev = 300, 16, 70
    a, tau = I.synthetic_full_store(n, b, 5, False)
    Y = I.eigvec_block(n, nev, 6, False)
    Co = oracle.back_transform_full(a, tau, n, b, np.asfortranarray(Y.copy()), nthreads=4)
    Cg = run_gpu(P, a, tau, n, b, Y, lda=n + 13, ldq=n + 7)
    assert np.abs(Cg - Co).max() <= TOL


@pytest.mark.parametrize("cplx", [False, True])
def test_band_as_wide_as_matrix_is_identity(P, cplx):
    n = 40
    a, tau = I.synthetic_full_store(n, n, 3, cplx)
    Y = I.eigvec_block(n, 10, 4, cplx)
    assert np.array_equal(run_gpu(P, a, tau, n, n + 3, Y), Y)


@pytest.mark.parametrize("cplx", [False, True])
def test_gpu_back_transforms_give_eigenpairs_of_dense_matrix(P, cplx):
    # 6a by the oracle on the host; 6b, 6d and 6e on the GPU; 6c by QL
    n, b, nev = 400 if not cplx else 200, 32, 120
    A = I.normal(77, 41, (n, n))
    if cplx:
        A = A + 1j * I.normal(77, 42, (n, n))
    A = (A + A.conj().T) / 2
    a, tau1 = oracle.full_to_band(A, b)
    W = np.zeros((b + 1, n), a.dtype)
    for d in range(b + 1):
        W[d, : n - d] = np.diag(a, -d)
    band = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()
    v, tau2, d, e = P.bulge_chase(band)
    P.stream_check()
    lam, X = oracle.tridiag_ql(d.cpu().numpy(), e.cpu().numpy())
    q = dev_fortran(np.asfortranarray(X[:, :nev].astype(a.dtype)))
    P.trans_ev_tridi_to_band(v, tau2, n, b, nev, q)
    P.trans_ev_band_to_full(dev_fortran(a), torch.from_numpy(tau1).cuda(), n, b, nev, q)
    P.stream_check()
    C = q.cpu().numpy()
    lam = lam[:nev]
    res = np.linalg.norm(A @ C - C * lam, axis=0).max() / np.abs(lam).max()
    assert res <= 1e-12, res
    assert np.abs(C.conj().T @ C - np.eye(nev)).max() <= 1e-12
    assert np.abs(lam - np.linalg.eigvalsh(A)[:nev]).max() <= 1e-10


def test_full_size_sampled_columns(P):
    # the benchmark's size: every column on the GPU, 12 of them by the oracle
    n, b, nev = 8192, 64, 4096
    a, tau = I.synthetic_full_store(n, b, I.SEED_BASE + 8, False)
    Y = I.eigvec_block(n, nev, I.SEED_BASE + 9, False)
    Cg = run_gpu(P, a, tau, n, b, Y)
    cols = np.unique(np.linspace(0, nev - 1, 12).astype(int))
    Co = oracle.back_transform_full(a, tau, n, b, np.asfortranarray(Y[:, cols]), nthreads=12)
    assert np.abs(Cg[:, cols] - Co).max() <= TOL
    # unitary Q1: column norms are kept for every column
    assert np.abs(np.linalg.norm(Cg, axis=0) - np.linalg.norm(Y, axis=0)).max() <= 1e-12 * n


# ---------------------------------------------------------------------------
# split-precision form (digit slices on the tensor cores), real data
# ---------------------------------------------------------------------------
SPLIT = 2  # api.VARIANT_SPLIT_BF16_TC
# 6 digits of 8 bits per operand: a few units of 2^-48 of a column's norm per
# block; the tolerance leaves room for the growth over ~n / 32 blocks
SPLIT_TOL = 1e-11


@pytest.mark.parametrize("n,b,nev", [(2, 1, 2), (5, 2, 3), (33, 1, 33), (100, 8, 37), (257, 32, 100),
                                     (300, 64, 300), (513, 64, 200), (200, 128, 50), (1000, 64, 500),
                                     (700, 5, 613), (64, 63, 9), (129, 96, 129), (2100, 64, 1000)])
def test_split_matches_oracle(P, n, b, nev):
    a, tau = I.synthetic_full_store(n, b, 1000 + n + b, False)
    Y = I.eigvec_block(n, nev, 7 + n, False)
    Co = oracle.back_transform_full(a, tau, n, b, np.asfortranarray(Y.copy()), nthreads=8)
    Cg = run_gpu(P, a, tau, n, b, Y, variant=SPLIT)
    assert np.abs(Cg - Co).max() <= SPLIT_TOL


def test_split_padded_leading_dimensions_and_scaled_columns(P):
    # columns of very different norms (each has its own fixed-point exponent)
    n, b, nev = 300, 16, 70
    a, tau = I.synthetic_full_store(n, b, 5, False)
    Y = I.eigvec_block(n, nev, 6, False) * np.logspace(-30, 30, nev)[None, :]
    Co = oracle.back_transform_full(a, tau, n, b, np.asfortranarray(Y.copy()), nthreads=4)
    Cg = run_gpu(P, a, tau, n, b, Y, lda=n + 13, ldq=n + 7, variant=SPLIT)
    scale = np.linalg.norm(Y, axis=0)
    assert (np.abs(Cg - Co).max(axis=0) / scale).max() <= SPLIT_TOL


def test_split_zero_columns_and_localised_vectors(P):
    # zero columns stay zero; unit vectors (one nonzero row) are transformed
    # as accurately as dense ones
    n, b, nev = 400, 32, 40
    a, tau = I.synthetic_full_store(n, b, 11, False)
    Y = np.zeros((n, nev))
    for j in range(1, nev):
        Y[(37 * j) % n, j] = 1.0
    Co = oracle.back_transform_full(a, tau, n, b, np.asfortranarray(Y.copy()), nthreads=4)
    Cg = run_gpu(P, a, tau, n, b, Y, variant=SPLIT)
    assert np.array_equal(Cg[:, 0], np.zeros(n))
    assert np.abs(Cg - Co).max() <= SPLIT_TOL


def test_split_band_as_wide_as_matrix_is_identity(P):
    n = 40
    a, tau = I.synthetic_full_store(n, n, 3, False)
    Y = I.eigvec_block(n, 10, 4, False)
    assert np.array_equal(run_gpu(P, a, tau, n, n + 3, Y, variant=SPLIT), Y)


def test_split_rejects_complex(P):
    n = 20
    a, tau = I.synthetic_full_store(n, 4, 3, True)
    Y = I.eigvec_block(n, 5, 4, True)
    with pytest.raises(ValueError):
        run_gpu(P, a, tau, n, 4, Y, variant=SPLIT)


def test_split_full_size_sampled_columns(P):
    # the benchmark's size: every column on the GPU, 12 of them by the oracle
    n, b, nev = 8192, 64, 4096
    a, tau = I.synthetic_full_store(n, b, I.SEED_BASE + 8, False)
    Y = I.eigvec_block(n, nev, I.SEED_BASE + 9, False)
    Cg = run_gpu(P, a, tau, n, b, Y, variant=SPLIT)
    cols = np.unique(np.linspace(0, nev - 1, 12).astype(int))
    Co = oracle.back_transform_full(a, tau, n, b, np.asfortranarray(Y[:, cols]), nthreads=12)
    assert np.abs(Cg[:, cols] - Co).max() <= SPLIT_TOL
    assert np.abs(np.linalg.norm(Cg, axis=0) - np.linalg.norm(Y, axis=0)).max() <= 1e-12 * n


def test_split_gives_eigenpairs_of_dense_matrix(P):
    # 6a by the oracle; 6b, 6d (FP64) and 6e (split form) on the GPU; 6c by QL
    n, b, nev = 400, 32, 120
    A = I.normal(77, 41, (n, n))
    A = (A + A.T) / 2
    a, tau1 = oracle.full_to_band(A, b)
    W = np.zeros((b + 1, n))
    for d in range(b + 1):
        W[d, : n - d] = np.diag(a, -d)
    v, tau2, d, e = P.bulge_chase(torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t())
    P.stream_check()
    lam, X = oracle.tridiag_ql(d.cpu().numpy(), e.cpu().numpy())
    q = dev_fortran(np.asfortranarray(X[:, :nev]))
    P.trans_ev_tridi_to_band(v, tau2, n, b, nev, q)
    P.trans_ev_band_to_full(dev_fortran(a), torch.from_numpy(tau1).cuda(), n, b, nev, q, variant=SPLIT)
    P.stream_check()
    C = q.cpu().numpy()
    lam = lam[:nev]
    res = np.linalg.norm(A @ C - C * lam, axis=0).max() / np.abs(lam).max()
    assert res <= 1e-12, res
    assert np.abs(C.T @ C - np.eye(nev)).max() <= 1e-12
