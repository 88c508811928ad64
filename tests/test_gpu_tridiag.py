"""Tridiagonal eigensolver on the GPU (Eq. 6c, only the nev wanted
eigenpairs) against the oracle's implicit QL, the closed form of a Toeplitz
tridiagonal matrix, and the residual and orthogonality bounds, including
clustered spectra (Wilkinson matrices, glued copies, exactly repeated
eigenvalues); and the whole GPU chain Eq. 6b -> 6c -> 6d on band matrices."""

import numpy as np
import pytest

import oracle
from paper_2002_10991_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def P():
    from paper_2002_10991_gb300 import _native

    _native.build()
    import paper_2002_10991_gb300 as P

    assert torch.cuda.is_available()
    return P


def gpu_eig(P, d, e, nev, complex_out=False):
    w, X = P.tridiag_eig(torch.from_numpy(np.ascontiguousarray(d)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(e)).cuda(), nev, complex_out=complex_out)
    P.stream_check()
    return w.cpu().numpy(), X.cpu().numpy()


def tnorm(d, e):
    r = np.abs(d).copy()
    r[1:] += np.abs(e)
    r[:-1] += np.abs(e)
    return max(r.max(initial=0.0), np.finfo(float).tiny)


def residual(d, e, w, X):
    """max_j ||T x_j - w_j x_j|| / ||T||_1-bound"""
    TX = d[:, None] * X
    TX[1:] += e[:, None] * X[:-1]
    TX[:-1] += e[:, None] * X[1:]
    R = TX - X * w[None, :]
    return float(np.sqrt((np.abs(R) ** 2).sum(0)).max(initial=0.0) / tnorm(d, e))


def orthogonality(X):
    G = X.conj().T @ X
    return float(np.abs(G - np.eye(G.shape[0])).max(initial=0.0))


def check_against_ql(P, d, e, nev, vec_gap=1e-5):
    w, X = gpu_eig(P, d, e, nev)
    lam, Z = oracle.tridiag_ql(d, e)
    tn = tnorm(d, e)
    assert np.abs(w - lam[:nev]).max(initial=0) <= 1e-12 * tn
    assert residual(d, e, w, X) <= 1e-13
    assert orthogonality(X) <= 1e-12
    # vectors of eigenvalues with a relative gap of at least vec_gap agree up to sign
    n = len(d)
    for k in range(nev):
        gap = min([abs(lam[k] - lam[j]) for j in (k - 1, k + 1) if 0 <= j < n] or [tn])
        if gap < vec_gap * tn:
            continue
        z, x = Z[:, k], X[:, k]
        assert np.abs(z * np.sign(z @ x) - x).max() <= 1e-9, k
    return w, X


@pytest.mark.parametrize("n,b,nev,seed", [(40, 4, 40, 1), (300, 16, 150, 2), (600, 32, 300, 3), (777, 64, 233, 4)])
def test_tridiag_of_bulge_chased_dft_band_matches_ql(P, n, b, nev, seed):
    W = I.band_dft(n, b, 4000 + seed, False)
    _, _, d, e = oracle.bulge_chase(W)
    check_against_ql(P, d, e, nev)


@pytest.mark.parametrize("n,nev", [(1, 1), (2, 2), (3, 1), (64, 64), (513, 200)])
def test_tridiag_of_random_matrix_matches_ql(P, n, nev):
    d = I.uniform(77, 1, (n,), -1.0, 1.0)
    e = I.uniform(77, 2, (max(n - 1, 0),), -1.0, 1.0)
    check_against_ql(P, d, e, nev)


@pytest.mark.parametrize("n,a,b", [(300, 2.0, -1.0), (1000, -3.0, 0.25)])
def test_toeplitz_closed_form(P, n, a, b):
    # eigenvalues a + 2 b cos(k pi / (n+1)), eigenvectors sqrt(2/(n+1)) sin(j k pi / (n+1))
    d = np.full(n, a)
    e = np.full(n - 1, b)
    nev = n // 2
    w, X = gpu_eig(P, d, e, nev)
    k = np.arange(1, n + 1)
    lam = np.sort(a + 2.0 * b * np.cos(k * np.pi / (n + 1)))
    assert np.abs(w - lam[:nev]).max() <= 1e-12 * (abs(a) + 2 * abs(b))
    j = np.arange(1, n + 1)[:, None]
    # ascending order: k = n, n-1, ... for b < 0 (cos decreasing), k = 1, 2, ... reversed for b > 0
    ks = (n + 1 - np.arange(1, nev + 1)) if b > 0 else np.arange(1, nev + 1)
    S = np.sqrt(2.0 / (n + 1)) * np.sin(j * ks[None, :] * np.pi / (n + 1))
    S *= np.sign(np.sum(S * X, axis=0))[None, :]
    # a computed eigenvector's error is bounded by about eps ||T|| / gap
    tn = abs(a) + 2 * abs(b)
    gap = np.diff(lam)[:nev].min()
    assert np.abs(X - S).max() <= max(1e-12, 100 * EPS * tn / gap)


def wilkinson(m):
    return np.abs(np.arange(-m, m + 1)).astype(np.float64), np.ones(2 * m)


@pytest.mark.parametrize("copies,glue", [(1, 0.0), (4, 1e-10), (6, 1e-14), (3, 0.0)])
def test_clustered_spectra(P, copies, glue):
    # Wilkinson W21+: pairs of eigenvalues equal to ~1e-14; glued copies:
    # clusters of `copies` nearly equal eigenvalues; glue 0: exact repeats
    dw, ew = wilkinson(10)
    d = np.concatenate([dw] * copies)
    parts = [ew]
    for _ in range(copies - 1):
        parts += [np.array([glue]), ew]
    e = np.concatenate(parts)
    n = len(d)
    w, X = gpu_eig(P, d, e, n)
    lam, _ = oracle.tridiag_ql(d, e)
    tn = tnorm(d, e)
    assert np.abs(w - lam).max() <= 1e-12 * tn
    assert residual(d, e, w, X) <= 1e-13
    assert orthogonality(X) <= 1e-12


def test_diagonal_matrix_with_repeated_entries(P):
    d = np.array([3.0, 1.0, 1.0, 2.0, 1.0, 2.0, 0.5])
    e = np.zeros(6)
    w, X = gpu_eig(P, d, e, 7)
    assert np.abs(w - np.sort(d)).max() <= 4 * EPS * 3.0
    assert residual(d, e, w, X) <= 1e-15
    assert orthogonality(X) <= 1e-14


def test_complex_output_and_padding(P):
    n, nev = 200, 70
    d = I.uniform(5, 1, (n,), -2.0, 2.0)
    e = I.uniform(5, 2, (n - 1,), -1.0, 1.0)
    w, X = gpu_eig(P, d, e, nev)
    wc, Xc = gpu_eig(P, d, e, nev, complex_out=True)
    assert np.array_equal(w, wc)
    assert np.array_equal(Xc.real, X) and not np.any(Xc.imag)
    # caller-provided output with ldx > n: padding rows untouched
    x = torch.full((nev, n + 5), float("nan"), dtype=torch.float64, device="cuda").t()
    P.tridiag_eig(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), nev, x=x)
    P.stream_check()
    xh = x.cpu().numpy()
    assert np.array_equal(xh[:n], X) and np.all(np.isnan(xh[n:]))
    w0, X0 = gpu_eig(P, d, e, 0)
    assert w0.size == 0 and X0.size == 0


@pytest.mark.parametrize("cplx", [False, True])
def test_gpu_chain_6b_6c_6d(P, cplx):
    # band -> tridiagonal, tridiagonal eigensolver and back-transformation,
    # all on the GPU: eigenpairs of the band matrix
    n, b, nev = 600, 32, 250
    W = I.band_dft(n, b, 31 if cplx else 30, cplx)
    band = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()
    v, tau, d, e = P.bulge_chase(band)
    w, X = P.tridiag_eig(d, e, nev, complex_out=cplx)
    P.trans_ev_tridi_to_band(v, tau, n, b, nev, X)
    P.stream_check()
    Z, w = X.cpu().numpy(), w.cpu().numpy()
    B = I.band_to_dense(W)
    lam = np.linalg.eigvalsh(B)
    nrm = np.abs(lam).max()
    assert np.abs(w - lam[:nev]).max() <= 1e-12 * nrm
    R = B @ Z - Z * w[None, :]
    assert np.sqrt((np.abs(R) ** 2).sum(0)).max() / nrm <= 1e-12
    assert orthogonality(Z) <= 1e-12
    assert np.linalg.norm(R) / (np.linalg.norm(B) * n * EPS) <= 10


def test_benchmark_size_tridiagonal(P):
    # T of the benchmark's band (n = 8192, b = 64, DFT-like) from the GPU bulge
    # chase; nev = 4096: eigenvalues against LAPACK's bisection, residual and
    # orthogonality on the device
    from scipy.linalg import eigvalsh_tridiagonal

    n, b, nev = 8192, 64, 4096
    W = I.band_dft(n, b, 2002109910 + n, False)
    _, _, d, e = P.bulge_chase(torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t())
    w, X = P.tridiag_eig(d, e, nev)
    P.stream_check()
    dh, eh = d.cpu().numpy(), e.cpu().numpy()
    lam = eigvalsh_tridiagonal(dh, eh, select="i", select_range=(0, nev - 1))
    tn = tnorm(dh, eh)
    assert np.abs(w.cpu().numpy() - lam).max() <= 1e-12 * tn
    TX = d[:, None] * X
    TX[1:] += e[:, None] * X[:-1]
    TX[:-1] += e[:, None] * X[1:]
    res = torch.linalg.vector_norm(TX - X * w[None, :], dim=0).max().item() / tn
    assert res <= 1e-13
    G = X.t() @ X
    G.diagonal().sub_(1.0)
    assert G.abs().max().item() <= 1e-12
