"""Pins of the oracle's full -> band reduction (Eq. 6a) and band -> full
back-transformation (Eq. 6e) to facts outside the oracle (no GPU needed).

* b = 1 is the one-stage tridiagonalisation: LAPACK's ?sytrd / ?hetrd (lower)
  with the same Householder convention give the same d, e, tau and stored
  reflectors.
* Any b: B is a similarity transform of A (its spectrum equals LAPACK's on
  the dense A), Q1 built by the back-transformation is unitary and
  reconstructs A = Q1 B Q1^H, Q1 leaves the first b coordinates alone, and
  Q1 equals the explicit dense product of its reflectors.
* The whole two-stage chain 6a -> 6b -> 6c -> 6d -> 6e gives eigenpairs of
  the dense matrix (residual and orthogonality).
* Copies of the oracle with planted mistakes fail these pins.
"""

import numpy as np
import pytest

import oracle
from paper_2002_10991_gb300 import inputs as I

scipy_lapack = pytest.importorskip("scipy.linalg.lapack")


def dense_hermitian(n, seed, cplx):
    # a seeded dense symmetric/Hermitian matrix from the shared generators
    A = I.normal(seed, 41, (n, n))
    if cplx:
        A = A + 1j * I.normal(seed, 42, (n, n))
    return (A + A.conj().T) / 2


def q1_of(a, tau, n, b):
    Q = np.asfortranarray(np.eye(n, dtype=a.dtype))
    return oracle.back_transform_full(a, tau, n, b, Q)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [2, 3, 17, 64, 150])
def test_b1_matches_lapack_tridiagonalisation(n, cplx):
    A = dense_hermitian(n, 100 + n, cplx)
    a, tau = oracle.full_to_band(A, 1)
    f = scipy_lapack.zhetrd if cplx else scipy_lapack.dsytrd
    c, d, e, tl, info = f(A, lower=1)
    assert info == 0
    scale = np.abs(A).max()
    assert np.abs(np.diag(a).real - d).max() <= 1e-13 * scale * n
    assert np.abs(np.diag(a, -1) - e).max(initial=0) <= 1e-13 * scale * n
    assert np.abs(tau - tl[: n - 1]).max(initial=0) <= 1e-12
    assert np.abs(np.tril(a, -2) - np.tril(c, -2)).max() <= 1e-12 * n


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b", [(40, 3), (97, 5), (128, 16), (65, 64), (64, 64), (33, 1), (90, 32)])
def test_similarity_reconstruction_and_unitarity(n, b, cplx):
    A = dense_hermitian(n, 7 * n + b, cplx)
    a, tau = oracle.full_to_band(A, b)
    B = oracle.band_of(a, b)
    i, j = np.indices((n, n))
    assert np.all(a[i < j - b] == 0)
    assert np.allclose(B, B.conj().T, rtol=0, atol=0)
    Q = q1_of(a, tau, n, b)
    tol = 1e-13 * n * max(1.0, np.abs(A).max())
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() <= 1e-13 * n
    assert np.abs(Q @ B @ Q.conj().T - A).max() <= tol
    lam = np.linalg.eigvalsh(A)
    assert np.abs(np.linalg.eigvalsh(B) - lam).max() <= tol
    # reflectors start at row c+b >= b: the first b coordinates are untouched
    assert np.array_equal(Q[:b, :b], np.eye(min(b, n), dtype=Q.dtype)[:b, :b])
    assert np.all(Q[:b, b:] == 0) and np.all(Q[b:, :b] == 0)


@pytest.mark.parametrize("cplx", [False, True])
def test_back_transform_full_equals_dense_product(cplx):
    n, b, nev = 50, 4, 13
    A = dense_hermitian(n, 5, cplx)
    a, tau = oracle.full_to_band(A, b)
    P = np.eye(n, dtype=a.dtype)
    for c in range(n - b):
        v = np.zeros(n, a.dtype)
        v[c + b] = 1.0
        v[c + b + 1:] = a[c + b + 1:, c]
        P = P @ (np.eye(n) - tau[c] * np.outer(v, v.conj()))
    Y = I.normal(9, 1, (n, nev)).astype(a.dtype)
    C = oracle.back_transform_full(a, tau, n, b, np.asfortranarray(Y), nthreads=3)
    assert np.abs(C - P @ Y).max() <= 1e-13 * n


@pytest.mark.parametrize("cplx", [False, True])
def test_band_wider_than_matrix_is_identity(cplx):
    n = 12
    A = dense_hermitian(n, 3, cplx)
    for b in (n, n + 5):
        a, tau = oracle.full_to_band(A, b)
        assert tau.size == 0
        assert np.array_equal(a, A)
        Y = np.asfortranarray(I.normal(2, 2, (n, 4)).astype(a.dtype))
        assert np.array_equal(oracle.back_transform_full(a, tau, n, b, Y.copy(order="F")), Y)


def two_stage_chain(A, b, nev):
    """6a -> 6b -> 6c -> 6d -> 6e with the oracle: eigenpairs of A."""
    n = A.shape[0]
    a, tau1 = oracle.full_to_band(A, b)
    W = np.zeros((b + 1, n), a.dtype)
    for d in range(b + 1):
        W[d, : n - d] = np.diag(a, -d)
    v, tau2, dd, e = oracle.bulge_chase(W)
    lam, X = oracle.tridiag_ql(dd, e)
    Y = np.asfortranarray(X[:, :nev].astype(a.dtype))
    oracle.back_transform(v, tau2, n, b, Y, nthreads=4)
    C = oracle.back_transform_full(a, tau1, n, b, Y, nthreads=4)
    return lam[:nev], C


@pytest.mark.parametrize("cplx", [False, True])
def test_two_stage_chain_gives_eigenpairs_of_dense_matrix(cplx):
    n, b, nev = 120, 8, 70
    A = dense_hermitian(n, 11, cplx)
    lam, C = two_stage_chain(A, b, nev)
    assert np.abs(lam - np.linalg.eigvalsh(A)[:nev]).max() <= 1e-12 * n
    res = np.linalg.norm(A @ C - C * lam, axis=0).max() / np.abs(np.linalg.eigvalsh(A)).max()
    assert res <= 1e-13 * n
    assert np.abs(C.conj().T @ C - np.eye(nev)).max() <= 1e-13 * n


# ---------------------------------------------------------------------------
# planted mistakes in the two new functions
# ---------------------------------------------------------------------------

MUTATIONS = {
    "full_forward_order": [("tbbt_oracle_impl.h", "for (int64_t k = J->K1 - 1; k >= 0; --k) {",
                            "for (int64_t k = 0; k < J->K1; ++k) {")],
    "full_dot_without_conj": [("tbbt_oracle_impl.h", "w += CONJ(tail[t - 1]) * y[t];", "w += tail[t - 1] * y[t];")],
    "full_rows_shifted": [("tbbt_oracle_impl.h", "int64_t r = k + J->b, L = J->n - r;",
                           "int64_t r = k + J->b - 1, L = J->n - r;")],
    "full_unit_entry_dropped": [("tbbt_oracle_impl.h", "    y[0] -= tauw;\n", "\n")],
    "reduction_right_update_conj_tau": [("tbbt_oracle_impl.h", "A[i + (r + t) * n] -= tk * w * CONJ(v[t]);",
                                         "A[i + (r + t) * n] -= CONJ(tk) * w * CONJ(v[t]);")],
    "reduction_column_offset": [("tbbt_oracle_impl.h", "for (int64_t t = 0; t < L; ++t) x[t] = A[r + t + c * n];",
                                 "for (int64_t t = 0; t < L; ++t) x[t] = A[r + t + (c + 1) * n];")],
}


def _pins_pass(cplx):
    try:
        n, b = 40, 4
        A = dense_hermitian(n, 77, cplx)
        a, tau = oracle.full_to_band(A, b)
        B = oracle.band_of(a, b)
        Q = q1_of(a, tau, n, b)
        ok = np.abs(Q @ B @ Q.conj().T - A).max() <= 1e-11
        ok = ok and np.abs(np.linalg.eigvalsh(B) - np.linalg.eigvalsh(A)).max() <= 1e-11
        lam, C = two_stage_chain(A, b, 20)
        res = np.linalg.norm(A @ C - C * lam, axis=0).max()
        return bool(ok and res <= 1e-10)
    except Exception:
        return False


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    assert _pins_pass(False) and _pins_pass(True)
    path = oracle.build_variant(MUTATIONS[name], str(tmp_path / f"liboracle_{name}.so"))
    with oracle.use_library(path):
        caught = (not _pins_pass(False)) or (not _pins_pass(True))
    assert caught, f"mutation {name} was not caught by the pins"


@pytest.mark.parametrize("cplx", [False, True])
def test_synthetic_full_store_is_unitary_and_fills_unread_entries(cplx):
    # the GPU parity tests and the benchmark use this store: its reflectors
    # are unitary (so Q1 keeps column norms), and the entries at or above the
    # b-th sub-diagonal hold N(0, 1) values, which a kernel that read them
    # would turn into a parity failure
    n, b = 90, 7
    a, tau = I.synthetic_full_store(n, b, 31, cplx)
    assert a.shape == (n, n) and a.flags.f_contiguous and tau.size == n - b
    Q = q1_of(a, tau, n, b)
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() <= 1e-13 * n
    i, j = np.indices((n, n))
    unread = i <= j + b
    assert np.all(a[unread] != 0)
    assert np.abs(a[unread]).mean() > 0.5  # N(0, 1) scale, not the N(0, 1/b) tails
    # the same seed gives the same store
    a2, tau2 = I.synthetic_full_store(n, b, 31, cplx)
    assert np.array_equal(a, a2) and np.array_equal(tau, tau2)
