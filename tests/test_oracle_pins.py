"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test ties one oracle function to something the paper or mathematics
fixes: index facts printed for the N=17, b=4 example (tests/golden), closed
forms (Toeplitz spectra and sine eigenvectors, polynomials of them), brute
force (Jacobi), LAPACK on the dense matrix, and invariants of the whole
chain (residual and orthogonality bounds). The last block builds copies of
the oracle with planted mistakes and checks that the pins reject them.
"""

import math
import os

import numpy as np
import pytest

import oracle
from paper_2002_10991_gb300 import inputs as I

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_n17_b4_index_facts.txt")


# ---------------------------------------------------------------------------
# helpers (checks only; no arithmetic of the method)
# ---------------------------------------------------------------------------

def chain(W, nev=None, nthreads=4):
    """band -> store, (d, e) -> eigenpairs of T -> back-transformed Z."""
    n = W.shape[1]
    b = W.shape[0] - 1
    v, tau, d, e = oracle.bulge_chase(W)
    lam, X = oracle.tridiag_ql(d, e)
    nev = n if nev is None else nev
    Z = np.asfortranarray(X[:, :nev].astype(W.dtype))
    oracle.back_transform(v, tau, n, b, Z, nthreads=nthreads)
    return v, tau, d, e, lam[:nev], Z


def residual(A, Z, lam):
    n = A.shape[0]
    return np.linalg.norm(A @ Z - Z * lam) / (np.linalg.norm(A) * n * EPS)


def orth(Z):
    return np.abs(Z.conj().T @ Z - np.eye(Z.shape[1])).max()


def dense_reflector(n, r, L, v, tau):
    H = np.eye(n, dtype=np.result_type(v, tau))
    vv = np.zeros(n, dtype=H.dtype)
    vv[r:r + L] = v[:L]
    return H - tau * np.outer(vv, vv.conj())


def read_golden():
    facts = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            facts.append(line.split())
    return facts


# ---------------------------------------------------------------------------
# store geometry: the paper's N=17, b=4 example (Sec. 2.2, Figs. 2-4)
# ---------------------------------------------------------------------------

def test_paper_index_facts_n17_b4():
    n, b = 17, 4
    stage, sweep = oracle.reflector_stage_sweep(n, b, False)
    r, L = oracle.reflector_rows(n, b, False)
    by_ij = {(int(i) + 1, int(j) + 1): (int(rr) + 1, int(ll)) for i, j, rr, ll in zip(stage, sweep, r, L)}
    gen_index = {(int(i) + 1, int(j) + 1): k for k, (i, j) in enumerate(zip(stage, sweep))}
    facts = read_golden()
    assert facts, "golden file empty"
    for f in facts:
        if f[0] == "sweeps_in_stage":
            st, cnt = int(f[1]), int(f[2])
            assert int(np.sum(stage == st - 1)) == cnt
        elif f[0] == "rows":
            i, j, lo, hi = map(int, f[1:])
            r1, ll = by_ij[(i, j)]
            assert (r1, r1 + ll - 1) == (lo, hi)
            assert hi == n  # "the last four rows"
        elif f[0] == "length_b_except_last_sweep":
            for st in range(1, n - 1):
                js = sorted(j for (i, j) in by_ij if i == st)
                for j in js[:-1]:
                    assert by_ij[(st, j)][1] == b
        elif f[0] == "apply_order":
            seq = [tuple(map(int, s.split(","))) for s in f[1:]]
            # applied in reverse generation order: generation index decreases
            ks = [gen_index[s] for s in seq]
            assert ks == sorted(ks, reverse=True)
            # consecutive transformations shift the touched rows up by one
            rows = [by_ij[s][0] for s in seq]
            assert all(rows[t] - rows[t + 1] == 1 for t in range(len(rows) - 1))
        elif f[0] == "local_rows":
            pass
        elif f[0] == "local_height":
            pass
    # the local window of Fig. 4: rows touched by (8,1)..(5,1) span N_R rows,
    # and (8,1), (7,1) sit at the printed local positions
    loc = {tuple(map(int, f[1:3])): (int(f[3]), int(f[4])) for f in facts if f[0] == "local_rows"}
    height = [int(f[1]) for f in facts if f[0] == "local_height"][0]
    seq = [(8, 1), (7, 1), (6, 1), (5, 1)]
    lo = min(by_ij[s][0] for s in seq)
    hi = max(by_ij[s][0] + by_ij[s][1] - 1 for s in seq)
    assert hi - lo + 1 == height
    for s, (a, z) in loc.items():
        r1, ll = by_ij[s]
        assert (r1 - lo + 1, r1 - lo + ll) == (a, z)


@pytest.mark.parametrize("n,b", [(17, 4), (2, 1), (3, 1), (5, 2), (64, 8), (100, 32), (129, 64), (300, 128)])
def test_geometry_matches_generator_and_brute_force(n, b):
    for cplx in (False, True):
        r, L = oracle.reflector_rows(n, b, cplx)
        assert len(L) == len(I.store_lengths(n, b, cplx))
        assert np.array_equal(L, I.store_lengths(n, b, cplx))
        # brute force: a stage needs another sweep while the previous sweep's
        # right update reached below the band, i.e. while rows remain below
        K = 0
        for i in range(0, n - 2):
            rr = i + 1
            while rr <= n - 2:  # a reflector needs at least two rows
                K += 1
                rr += b
        K += 1 if (cplx and n >= 2) else 0
        assert K == len(L)
        assert np.all(L >= 1) and np.all(L <= b) and np.all(r + L <= n)


def test_reflector_counts_of_named_workloads():
    # K and sum(L) follow from the store rule; they are the unit counts of the
    # algorithmic work (4 * nev * sum(L) real flops, 16 * nev * sum(L) complex).
    assert oracle.num_reflectors(512, 32, False) == 4320
    assert oracle.num_reflectors(8192, 64, False) == 528128
    r, L = oracle.reflector_rows(8192, 64, False)
    assert int(L.sum()) == 33550208
    assert int(L.sum()) == sum(I.store_lengths(8192, 64, False))


# ---------------------------------------------------------------------------
# Eq. 6c: implicit QL against closed forms and brute force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 10, 65, 200])
def test_ql_toeplitz_closed_form(n):
    a, bo = 0.7, -1.3
    lam, Z = oracle.tridiag_ql(np.full(n, a), np.full(max(n - 1, 0), bo))
    k = np.arange(1, n + 1)
    exact = np.sort(a + 2 * bo * np.cos(k * math.pi / (n + 1)))
    assert np.abs(lam - exact).max() <= 8 * n * EPS * (abs(a) + 2 * abs(bo))
    # eigenvectors: sqrt(2/(n+1)) sin(j k pi/(n+1)), matched by eigenvalue, up to sign
    j = np.arange(1, n + 1)[:, None]
    S = math.sqrt(2.0 / (n + 1)) * np.sin(j * k[None, :] * math.pi / (n + 1))
    lam_k = a + 2 * bo * np.cos(k * math.pi / (n + 1))
    order = np.argsort(lam_k)
    S = S[:, order]
    dots = np.abs(np.sum(S * Z, axis=0))
    assert np.abs(dots - 1).max() <= 1e-12 * max(n, 1)


def test_ql_matches_jacobi_random():
    rng = np.random.default_rng(5)
    for n in (4, 17, 40, 64):
        d = rng.uniform(-3, 3, n)
        e = rng.normal(size=n - 1)
        T = np.diag(d) + np.diag(e, -1) + np.diag(e, 1)
        lam, Z = oracle.tridiag_ql(d, e)
        w = oracle.jacobi(T)
        assert np.abs(lam - w).max() <= 1e-13 * np.abs(w).max() * n
        assert orth(Z) <= 1e-13
        assert residual(T, Z, lam) <= 10


def test_jacobi_matches_lapack():
    rng = np.random.default_rng(7)
    A = rng.normal(size=(30, 30))
    A = A + A.T
    assert np.abs(oracle.jacobi(A) - np.linalg.eigvalsh(A)).max() <= 1e-12 * np.abs(A).max()
    Hc = rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12))
    Hc = Hc + Hc.conj().T
    assert np.abs(oracle.jacobi(Hc) - np.linalg.eigvalsh(Hc)).max() <= 1e-12 * np.abs(Hc).max()


# ---------------------------------------------------------------------------
# Eq. 6b: bulge chasing
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b", [(17, 4), (40, 5), (64, 8), (64, 1), (33, 32), (64, 63)])
def test_bulge_chase_is_similarity_to_tridiagonal(n, b, cplx):
    W = I.band_uniform(n, b, 1000 + n + b, cplx)
    A = I.band_to_dense(W)
    v, tau, d, e, work = oracle.bulge_chase(W, return_work=True)
    # everything beyond the first sub-diagonal is exactly zero
    if work.shape[0] > 2:
        assert np.count_nonzero(work[2:, :]) == 0
    # the spectrum is preserved: brute-force Jacobi and LAPACK on the dense band
    T = np.diag(d) + np.diag(e, -1) + np.diag(e, 1)
    lamT = np.linalg.eigvalsh(T)
    assert np.abs(lamT - oracle.jacobi(A)).max() <= 1e-12 * max(1.0, np.abs(lamT).max()) * n
    assert np.abs(lamT - np.linalg.eigvalsh(A)).max() <= 1e-12 * max(1.0, np.abs(lamT).max()) * n
    # backward error of the accumulated transform: Qh = H_0 ... H_{K-1}
    Qh = np.asfortranarray(np.eye(n, dtype=A.dtype))
    oracle.back_transform(v, tau, n, b, Qh)
    berr = np.linalg.norm(Qh.conj().T @ A @ Qh - T) / np.linalg.norm(A)
    assert berr <= 20 * n * EPS
    # every tau makes a unitary reflector
    vv = v.reshape(-1, b)
    nrm2 = np.sum(np.abs(vv) ** 2, axis=1)
    assert np.abs(2 * tau.real - np.abs(tau) ** 2 * nrm2).max() <= 1e-13 * (1 + np.abs(tau).max() ** 2 * nrm2.max())
    assert np.all(vv[:, 0] == 1.0)


def test_bulge_chase_on_tridiagonal_is_identity_real():
    n, b = 50, 6
    W = I.toeplitz_band(n, b, 0.3, -0.8)
    v, tau, d, e = oracle.bulge_chase(W)
    assert np.all(tau == 0.0)
    # tau = 0 keeps beta = alpha: the tridiagonal comes back unchanged
    assert np.array_equal(d, np.full(n, 0.3)) and np.array_equal(e, np.full(n - 1, -0.8))


def test_bulge_chase_complex_toeplitz_phase_only():
    # complex off-diagonal b' e^{i phi}: the reduction only rotates phases, so
    # every reflector is diagonal (v = e_1) and |e| = |b'|
    n, b, phi = 30, 4, 0.9
    W = I.toeplitz_band(n, b, 1.1, complex(0.6 * math.cos(phi), 0.6 * math.sin(phi)))
    v, tau, d, e = oracle.bulge_chase(W)
    vv = v.reshape(-1, b)
    assert np.all(vv[:, 1:] == 0.0)
    assert np.allclose(np.abs(e), 0.6, atol=1e-15)
    A = I.band_to_dense(W)
    v2, t2, d2, e2, lam, Z = chain(W)
    k = np.arange(1, n + 1)
    exact = np.sort(1.1 + 2 * 0.6 * np.cos(k * math.pi / (n + 1)))
    assert np.abs(lam - exact).max() <= 1e-13
    assert residual(A, Z, lam) <= 10


@pytest.mark.parametrize("cplx", [False, True])
def test_polynomial_of_toeplitz_known_spectrum_and_vectors(cplx):
    # B = p(T) with T tridiagonal Toeplitz and p(x) = x^3 + 3x (monotone):
    # B has semi-bandwidth 3, eigenvalues p(lambda_k) and the sine eigenvectors
    # of T. The reduction produces non-trivial reflectors with a known answer.
    n = 48
    a, bo = 0.25, 0.5
    T = np.diag(np.full(n, a)) + np.diag(np.full(n - 1, bo), -1) + np.diag(np.full(n - 1, bo), 1)
    if cplx:
        ph = np.exp(1j * np.linspace(0.1, 2.0, n))
        D = np.diag(ph)
        T = D @ T @ D.conj().T  # unitarily similar, complex entries, same spectrum
    B = T @ T @ T + 3 * T
    b = 3
    W = np.zeros((b + 1, n), dtype=B.dtype)
    for dd in range(b + 1):
        W[dd, : n - dd] = np.diagonal(B, -dd)
    W[0] = W[0].real
    v, tau, d, e, lam, Z = chain(W)
    assert np.count_nonzero(tau) > 0
    k = np.arange(1, n + 1)
    lk = a + 2 * bo * np.cos(k * math.pi / (n + 1))
    exact = np.sort(lk ** 3 + 3 * lk)
    assert np.abs(lam - exact).max() <= 1e-12 * np.abs(exact).max()
    j = np.arange(1, n + 1)[:, None]
    S = math.sqrt(2.0 / (n + 1)) * np.sin(j * k[None, :] * math.pi / (n + 1))
    S = S[:, np.argsort(lk ** 3 + 3 * lk)]
    if cplx:
        S = D @ S
    overlap = np.abs(np.sum(S.conj() * Z, axis=0))
    assert np.abs(overlap - 1).max() <= 1e-10


# ---------------------------------------------------------------------------
# Eq. 6d / Eq. 8: the back-transformation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("cplx", [False, True])
def test_back_transform_identity_store_is_exact(cplx):
    n, b, nev = 70, 8, 13
    v, tau = I.synthetic_store(n, b, 3, cplx)
    tau[:] = 0
    X = I.eigvec_block(n, nev, 4, cplx, ldq=n + 3)
    Z = X.copy(order="F")
    oracle.back_transform(v, tau, n, b, Z)
    assert np.array_equal(Z[:n], X[:n])
    assert np.all(np.isnan(Z[n:]))  # rows beyond n untouched


@pytest.mark.parametrize("cplx", [False, True])
def test_back_transform_single_reflector_closed_form(cplx):
    n, b, nev = 40, 6, 9
    v, tau = I.synthetic_store(n, b, 8, cplx)
    r, L = oracle.reflector_rows(n, b, cplx)
    keep = len(tau) // 3
    t2 = np.zeros_like(tau)
    t2[keep] = tau[keep]
    X = I.eigvec_block(n, nev, 9, cplx)
    Z = X.copy(order="F")
    oracle.back_transform(v, t2, n, b, Z)
    H = dense_reflector(n, r[keep], L[keep], v[keep * b:(keep + 1) * b], tau[keep])
    assert np.abs(Z - H @ X).max() <= 1e-14


@pytest.mark.parametrize("cplx", [False, True])
def test_back_transform_equals_dense_product(cplx):
    # Z = H_0 H_1 ... H_{K-1} X with the product formed left to right as dense
    # matrices (a different association from applying Eq. 8 column by column)
    n, b, nev = 30, 5, 7
    v, tau = I.synthetic_store(n, b, 12, cplx)
    r, L = oracle.reflector_rows(n, b, cplx)
    Q = np.eye(n, dtype=np.complex128 if cplx else np.float64)
    for k in range(len(tau)):
        Q = Q @ dense_reflector(n, r[k], L[k], v[k * b:(k + 1) * b], tau[k])
    X = I.eigvec_block(n, nev, 13, cplx)
    Z = X.copy(order="F")
    oracle.back_transform(v, tau, n, b, Z, nthreads=3)
    assert np.abs(Z - Q @ X).max() <= 1e-13


@pytest.mark.parametrize("cplx", [False, True])
def test_back_transform_preserves_column_norms(cplx):
    n, b, nev = 300, 32, 20
    v, tau = I.synthetic_store(n, b, 17, cplx)
    X = I.eigvec_block(n, nev, 18, cplx)
    Z = X.copy(order="F")
    oracle.back_transform(v, tau, n, b, Z, nthreads=4)
    nx = np.linalg.norm(X, axis=0)
    nz = np.linalg.norm(Z, axis=0)
    assert np.abs(nz / nx - 1).max() <= 50 * n * EPS


@pytest.mark.parametrize("cplx", [False, True])
def test_chain_residual_and_orthogonality_uniform_n512(cplx):
    # the plain-method workload: N=512, b=32, all eigenvectors
    W = I.band_uniform(512, 32, I.SEED_BASE + 1, cplx)
    A = I.band_to_dense(W)
    v, tau, d, e, lam, Z = chain(W, nthreads=8)
    assert residual(A, Z, lam) <= 10
    assert orth(Z) <= 1e-12
    assert np.abs(lam - np.linalg.eigvalsh(A)).max() <= 1e-12 * np.abs(lam).max()


def test_chain_dft_like_partial_spectrum():
    W = I.band_dft(400, 16, 77, True)
    A = I.band_to_dense(W)
    v, tau, d, e, lam, Z = chain(W, nev=120)
    assert residual(A, Z, lam) <= 10
    assert orth(Z) <= 1e-12


def test_back_transform_threading_is_bitwise_stable():
    n, b, nev = 200, 16, 37
    v, tau = I.synthetic_store(n, b, 5, False)
    X = I.eigvec_block(n, nev, 6, False)
    Z1 = oracle.back_transform(v, tau, n, b, X.copy(order="F"), nthreads=1)
    Z7 = oracle.back_transform(v, tau, n, b, X.copy(order="F"), nthreads=7)
    assert np.array_equal(Z1, Z7)


# ---------------------------------------------------------------------------
# planted mistakes: the pins above must reject each of these oracle variants
# ---------------------------------------------------------------------------

MUTATIONS = {
    "forward_order": [("tbbt_oracle_impl.h", "for (int64_t k = J->K - 1; k >= 0; --k) {",
                       "for (int64_t k = 0; k < J->K; ++k) {")],
    "dot_without_conj": [("tbbt_oracle_impl.h", "for (int64_t t = 0; t < L; ++t) w += CONJ(vk[t]) * x[t];",
                          "for (int64_t t = 0; t < L; ++t) w += vk[t] * x[t];")],
    "conj_tau": [("tbbt_oracle_impl.h", "SCALAR tw = tk * w;", "SCALAR tw = CONJ(tk) * w;")],
    "rows_shifted": [("tbbt_oracle.c", "      r[k] = i + 1 + j * b;\n      L[k]", "      r[k] = i + j * b;\n      L[k]")],
    "short_update": [("tbbt_oracle_impl.h", "for (int64_t t = 0; t < L; ++t) x[t] -= tw * vk[t];",
                      "for (int64_t t = 1; t < L; ++t) x[t] -= tw * vk[t];")],
    "ql_rotation_sign": [("tbbt_oracle.c", "zi1[k] = s * zi[k] + c * t;", "zi1[k] = s * zi[k] - c * t;")],
    "pivot_column": [("tbbt_oracle_impl.h", "int64_t c = (j == 0) ? i : r - b;", "int64_t c = (j == 0) ? i : r - b + 1;")],
}


def _pins_pass(cplx):
    try:
        W = I.band_uniform(48, 6, 4242, cplx)
        A = I.band_to_dense(W)
        v, tau, d, e, lam, Z = chain(W)
        return residual(A, Z, lam) <= 10 and orth(Z) <= 1e-12 and \
            np.abs(lam - np.linalg.eigvalsh(A)).max() <= 1e-10
    except Exception:
        return False


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    assert _pins_pass(False) and _pins_pass(True)
    path = oracle.build_variant(MUTATIONS[name], str(tmp_path / f"liboracle_{name}.so"))
    with oracle.use_library(path):
        caught = (not _pins_pass(False)) or (not _pins_pass(True))
    assert caught, f"mutation {name} was not caught by the chain pins"
