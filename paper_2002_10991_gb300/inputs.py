"""Seeded synthetic inputs for the tridiagonal-to-band eigenvector back-transform.

This module is shared by the CPU oracle tests and the GPU path. It only draws
random numbers and lays them out; it holds none of the method's arithmetic
(no bulge chasing, no eigensolve, no reflector application).

Random numbers come from a counter-based splitmix64 stream: element ``i`` of
stream ``s`` under seed ``seed`` is ``splitmix64(mix(seed, s) + (i+1)*phi)``,
``u = (x >> 11) * 2**-53`` in [0, 1), normals by the Box-Muller cosine branch.
Counter-based draws make every array reproducible independently of the others
and of the order they are generated in.

Workloads (the paper's random / KS-DFT-like problems, Sec. 4 and Sec. 5; the
paper does not state a distribution, so these are this library's choice):

* ``uniform`` band: lower band including the diagonal i.i.d. U[-1, 1],
  mirrored to a symmetric matrix.
* ``dft`` band: diagonal U[-10, 10] sorted ascending, sub-diagonals
  ``d = 1..b`` drawn N(0, 1) * exp(-d/16) (real and imaginary part each for
  Hermitian problems), mirrored (conjugated) to a symmetric/Hermitian matrix.

Band matrices are returned in lower band storage ``W[d, c] = B[c+d, c]`` of
shape ``(b+1, n)``; entries with ``c + d >= n`` are zero.
"""

from __future__ import annotations

import math
import os

import numpy as np

PHI = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seed of workload ``k`` (1-based, in the order listed in the design notes).
SEED_BASE = 2002109910


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream & 0xFFFFFFFF) * _M2)
        return _mix(np.array([k], dtype=np.uint64))[0]


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` 64-bit words of stream ``stream`` starting at counter ``offset``."""
    key = _stream_key(seed, stream)
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + idx * PHI)


# Arrays longer than this are drawn in chunks on several host threads (the
# draws are counter-based, so the result does not depend on the chunking).
_CHUNK = 1 << 21


def _chunked(n: int, fill) -> np.ndarray:
    """out[a:b] = fill(a, b) over chunks of the index range, in parallel."""
    out = np.empty(n, dtype=np.float64)
    if n <= _CHUNK:
        out[:] = fill(0, n)
        return out
    from concurrent.futures import ThreadPoolExecutor

    def work(a):
        b = min(a + _CHUNK, n)
        out[a:b] = fill(a, b)

    with ThreadPoolExecutor(max_workers=min(os.cpu_count() or 1, 32)) as ex:
        list(ex.map(work, range(0, n, _CHUNK)))
    return out


def uniform(seed: int, stream: int, shape, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    n = int(np.prod(shape)) if len(shape) else 1

    def fill(a, b):
        u = (splitmix64(seed, stream, b - a, a) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    return _chunked(n, fill).reshape(shape)


def normal(seed: int, stream: int, shape) -> np.ndarray:
    n = int(np.prod(shape)) if len(shape) else 1

    def fill(a, b):
        w = splitmix64(seed, stream, 2 * (b - a), 2 * a)
        u1 = (w[0::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        u2 = (w[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)

    return _chunked(n, fill).reshape(shape)


# ----------------------------------------------------------------------------
# band matrices (the input of the band -> tridiagonal reduction, Eq. 6b)
# ----------------------------------------------------------------------------

def band_uniform(n: int, b: int, seed: int, complex_: bool = False) -> np.ndarray:
    """Lower band (incl. diagonal) i.i.d. U[-1,1]; Hermitian input gets a real diagonal."""
    W = uniform(seed, 1, (b + 1, n), -1.0, 1.0)
    if complex_:
        im = uniform(seed, 2, (b + 1, n), -1.0, 1.0)
        im[0, :] = 0.0
        W = W + 1j * im
    _clear_outside(W, n, b)
    return W


def band_dft(n: int, b: int, seed: int, complex_: bool = False, decay: float = 16.0) -> np.ndarray:
    """DFT-like band: sorted U[-10,10] diagonal, N(0,1)*exp(-d/decay) off-diagonals."""
    W = np.zeros((b + 1, n), dtype=np.complex128 if complex_ else np.float64)
    W[0, :] = np.sort(uniform(seed, 1, (n,), -10.0, 10.0))
    scale = np.exp(-np.arange(1, b + 1, dtype=np.float64) / decay)[:, None]
    off = normal(seed, 2, (b, n)) * scale
    if complex_:
        off = off + 1j * (normal(seed, 3, (b, n)) * scale)
    W[1:, :] = off
    _clear_outside(W, n, b)
    return W


def _clear_outside(W: np.ndarray, n: int, b: int) -> None:
    for d in range(1, b + 1):
        W[d, max(0, n - d):] = 0.0


def band_to_dense(W: np.ndarray) -> np.ndarray:
    """Dense symmetric/Hermitian matrix from lower band storage (for checks)."""
    b = W.shape[0] - 1
    n = W.shape[1]
    A = np.zeros((n, n), dtype=W.dtype)
    for d in range(0, b + 1):
        idx = np.arange(0, n - d)
        A[idx + d, idx] = W[d, : n - d]
        if d:
            A[idx, idx + d] = np.conj(W[d, : n - d])
    return A


def toeplitz_band(n: int, b: int, a: float, offdiag: complex) -> np.ndarray:
    """A tridiagonal Toeplitz matrix (diagonal ``a``, sub-diagonal ``offdiag``)
    embedded in lower band storage of semi-bandwidth ``b`` (all other band
    entries zero)."""
    dt = np.complex128 if isinstance(offdiag, complex) else np.float64
    W = np.zeros((b + 1, n), dtype=dt)
    W[0, :] = a
    if b >= 1:
        W[1, : n - 1] = offdiag
    return W


# ----------------------------------------------------------------------------
# eigenvector blocks and reflector stores (the inputs of Eq. 6d)
# ----------------------------------------------------------------------------

def eigvec_block(n: int, nev: int, seed: int, complex_: bool = False, ldq: int | None = None) -> np.ndarray:
    """A dense n x nev block (column-major, leading dimension ``ldq``) with
    N(0, 1/n) entries; returned as an (ldq, nev) Fortran-ordered array whose
    rows n..ldq-1 are NaN so that a kernel touching them is caught."""
    ldq = n if ldq is None else ldq
    X = np.full((ldq, nev), np.nan, dtype=np.complex128 if complex_ else np.float64, order="F")
    s = 1.0 / math.sqrt(max(n, 1))
    body = normal(seed, 11, (nev, n)).T * s
    if complex_:
        body = body + 1j * (normal(seed, 12, (nev, n)).T * s)
        body = body / math.sqrt(2.0)
    X[:n, :] = body
    return X


def store_lengths(n: int, b: int, complex_: bool) -> np.ndarray:
    """Lengths L_k of the reflectors in generation order (the canonical store
    format: stage i = 0..n-3, sweep j = 0..ceil((n-i-2)/b)-1, L = min(b, n-r)
    with r = i+1+j*b; a Hermitian store ends with one length-1 reflector)."""
    i = np.arange(max(n - 2, 0), dtype=np.int64)
    s = -(-(n - i - 2) // b)  # sweeps of stage i
    stage = np.repeat(i, s)
    first = np.repeat(np.cumsum(s) - s, s)  # index of reflector (i, 0)
    j = np.arange(stage.size, dtype=np.int64) - first
    L = np.minimum(b, n - (stage + 1 + j * b))
    if complex_ and n >= 2:
        L = np.append(L, 1)
    return L.astype(np.int64)


def synthetic_store(n: int, b: int, seed: int, complex_: bool = False):
    """Random unitary Householder reflectors in the canonical store layout.

    Returns ``(hh_v, hh_tau)``: ``hh_v`` is K x b column-major (reflector k is
    the contiguous slice ``hh_v[k*b:(k+1)*b]``) with ``v[0] = 1`` stored and
    zeros at positions >= L_k; ``hh_tau`` has K entries. Entries v[1:L] are
    N(0, 1/b) draws; tau is chosen so that I - tau v v^H is unitary:
    tau = 2/|v|^2 for real data and tau = (1 - exp(i*theta))/|v|^2 with
    theta ~ U[0, 2pi) for complex data. Used where the stores of real
    reductions are too slow to produce on the host; the back-transform's cost
    does not depend on the values.
    """
    L = store_lengths(n, b, complex_)
    K = len(L)
    dt = np.complex128 if complex_ else np.float64
    V = normal(seed, 21, (K, b)) / math.sqrt(max(b, 1))
    if complex_:
        V = V + 1j * (normal(seed, 22, (K, b)) / math.sqrt(max(b, 1)))
    V = V.astype(dt, copy=False)
    short = np.nonzero(L < b)[0]  # only the last sweeps of a stage are truncated
    cols = np.arange(b)[None, :]
    V[short] = np.where(cols >= L[short][:, None], 0.0, V[short])
    V[:, 0] = 1.0
    nrm2 = np.einsum("kj,kj->k", V.real, V.real)
    if complex_:
        nrm2 = nrm2 + np.einsum("kj,kj->k", V.imag, V.imag)
    if complex_:
        theta = uniform(seed, 23, (K,), 0.0, 2.0 * math.pi)
        tau = (1.0 - np.exp(1j * theta)) / nrm2
    else:
        tau = 2.0 / nrm2
    return np.ascontiguousarray(V.reshape(-1)), np.ascontiguousarray(tau.astype(dt))


def synthetic_full_store(n: int, b: int, seed: int, complex_: bool = False):
    """Random unitary reflectors in the layout the full -> band reduction
    leaves (LAPACK style): ``a`` (n x n, Fortran order) holds reflector c's
    v[1:] in ``a[c+b+1:, c]`` (v[0] = 1 implicit at row c+b) and N(0, 1)
    values everywhere else, which the back-transformation must not read;
    ``tau`` (max(n-b, 0) entries) makes each I - tau v v^H unitary, as in
    ``synthetic_store``. Tails are N(0, 1/b) draws."""
    dt = np.complex128 if complex_ else np.float64
    a = normal(seed, 51, (n, n))
    if complex_:
        a = a + 1j * normal(seed, 52, (n, n))
    a = np.asfortranarray(a.astype(dt).reshape(n, n).T)  # column c = draws c*n .. c*n+n-1
    K1 = max(n - b, 0)
    i = np.arange(n)[:, None]
    c = np.arange(n)[None, :]
    below = i > c + b
    a[below] *= 1.0 / math.sqrt(max(b, 1))
    nrm2 = 1.0 + np.sum(np.where(below, np.abs(a) ** 2, 0.0), axis=0)[:K1]
    if complex_:
        theta = uniform(seed, 53, (K1,), 0.0, 2.0 * math.pi)
        tau = (1.0 - np.exp(1j * theta)) / nrm2
    else:
        tau = 2.0 / nrm2
    return a, np.ascontiguousarray(tau.astype(dt))


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

WORKLOADS = {
    # name: (n, b, nev, complex, band kind, seed)
    "real-n512-b32-uniform": dict(n=512, b=32, nev=512, complex_=False, kind="uniform", seed=SEED_BASE + 1),
    "real-n8192-b64-dft": dict(n=8192, b=64, nev=4096, complex_=False, kind="dft", seed=SEED_BASE + 2),
    "complex-n20000-b64-dft": dict(n=20000, b=64, nev=6000, complex_=True, kind="dft", seed=SEED_BASE + 3),
    "real-n32768-b64-dft": dict(n=32768, b=64, nev=9830, complex_=False, kind="dft", seed=SEED_BASE + 4),
    # a smaller case of the same kernel for profiler captures (q still larger than L2)
    "real-n4096-b64-dft": dict(n=4096, b=64, nev=4096, complex_=False, kind="dft", seed=SEED_BASE + 6),
    "complex-n4096-b64-dft": dict(n=4096, b=64, nev=2048, complex_=True, kind="dft", seed=SEED_BASE + 7),
}


def band_for(name: str, n: int | None = None) -> np.ndarray:
    w = WORKLOADS[name]
    n = w["n"] if n is None else n
    f = band_uniform if w["kind"] == "uniform" else band_dft
    return f(n, w["b"], w["seed"], w["complex_"])


def batch_sizes(count: int = 64, seed: int = SEED_BASE + 5, lo: int = 1000, hi: int = 6000) -> np.ndarray:
    """Problem sizes of the batched workload: N_p = lo + floor(u*(hi-lo+1))."""
    u = uniform(seed, 31, (count,))
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def batch_workload(count: int = 64, seed: int = SEED_BASE + 5, b: int = 32):
    """The batched workload: ``count`` problems with N_p drawn from
    ``batch_sizes``, even p real and odd p complex, semi-bandwidth ``b``,
    nev = floor(N_p / 2). Returns a list of dicts (n, b, nev, complex_, seed)."""
    sizes = batch_sizes(count, seed)
    return [dict(n=int(n), b=b, nev=int(n) // 2, complex_=bool(p % 2), seed=seed * 131 + p)
            for p, n in enumerate(sizes)]
