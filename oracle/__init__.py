"""CPU oracle for the tridiagonal -> band eigenvector back-transformation
(arXiv 2002.10991, Eq. 6b-6d).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package; the
product library never does. The arithmetic lives in plain C
(``tbbt_oracle.c``); this module compiles it with gcc on first use and
marshals numpy arrays through ctypes.

Every function states the passage of the paper it follows. Functions and
their pins (the tests that tie them to something other than themselves):

* ``num_reflectors`` / ``reflector_rows`` / ``reflector_stage_sweep``:
  Sec. 2.2.1 and Figs. 2-4 (N=17, b=4 facts in tests/golden).
* ``bulge_chase``: Eq. 6b, Sec. 2.2.1 -- tridiagonal output, spectrum equal
  to brute-force Jacobi and to LAPACK on the dense band matrix, backward
  error of the accumulated transform.
* ``tridiag_ql``: Eq. 6c -- closed-form Toeplitz spectrum and sine basis,
  Jacobi.
* ``back_transform``: Eq. 6d / Eq. 8 -- identity store, explicit dense
  reflector products, residual ||BZ - Z Lambda|| and orthogonality of the
  whole chain, unitary invariance of column norms; planted mistakes (forward
  order, conjugation dropped, shifted rows) fail these.
* ``full_to_band``: Eq. 6a -- LAPACK's tridiagonalisation (?sytrd / ?hetrd,
  lower) at b = 1, spectrum of B equal to LAPACK's on the dense matrix,
  reconstruction A = Q1 B Q1^H with the back-transformation below.
* ``back_transform_full``: Eq. 6e -- the same reconstruction, unitarity of
  Q1, explicit dense reflector products, the identity on the first b rows,
  and the residual and orthogonality of the whole two-stage chain
  (6a -> 6b -> 6c -> 6d -> 6e) on the dense matrix.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "tbbt_oracle.c"), os.path.join(_HERE, "tbbt_oracle_impl.h")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: no -march, works on x86
    and aarch64). Returns the path of the shared library."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or any(os.path.getmtime(s) > os.path.getmtime(_LIB) for s in _SRC)
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC[0],
               "-lpthread", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class use_library:
    """Context manager that points this module at another compiled copy of
    the oracle (the tests build copies with planted mistakes to show that
    the pins catch them)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = None
        _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def build_variant(replacements, out_path: str) -> str:
    """Compile a copy of the oracle with textual replacements applied to its
    sources (``[(file, old, new), ...]``, each ``old`` must occur once)."""
    import shutil
    import tempfile

    tmp = tempfile.mkdtemp(prefix="oracle_variant_")
    for s in _SRC:
        shutil.copy(s, tmp)
    for fname, old, new in replacements:
        p = os.path.join(tmp, fname)
        text = open(p).read()
        if text.count(old) != 1:
            raise ValueError(f"replacement target not unique in {fname}: {old!r}")
        open(p, "w").write(text.replace(old, new))
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", out_path,
           os.path.join(tmp, "tbbt_oracle.c"), "-lpthread", "-lm"]
    subprocess.run(cmd, check=True)
    shutil.rmtree(tmp, ignore_errors=True)
    return out_path


def _configure(L):
    global _lib
    i64, p = ctypes.c_int64, ctypes.c_void_p
    L.orc_num_reflectors.restype = i64
    L.orc_num_reflectors.argtypes = [i64, i64, ctypes.c_int]
    L.orc_reflector_rows.argtypes = [i64, i64, ctypes.c_int, p, p]
    L.orc_reflector_stage_sweep.argtypes = [i64, i64, ctypes.c_int, p, p]
    for s in ("d", "z"):
        f = getattr(L, f"orc_bulge_chase_{s}")
        f.restype = i64
        f.argtypes = [i64, i64, p, i64, p, p, p, p, p]
        g = getattr(L, f"orc_back_transform_{s}")
        g.restype = ctypes.c_int
        g.argtypes = [i64, i64, i64, p, p, p, i64, ctypes.c_int]
    for s in ("d", "z"):
        f = getattr(L, f"orc_full_to_band_{s}")
        f.restype = i64
        f.argtypes = [i64, i64, p, i64, p]
        g = getattr(L, f"orc_back_transform_full_{s}")
        g.restype = ctypes.c_int
        g.argtypes = [i64, i64, i64, p, i64, p, p, i64, ctypes.c_int]
    L.orc_tridiag_ql.restype = ctypes.c_int
    L.orc_tridiag_ql.argtypes = [i64, p, p, p, i64]
    L.orc_jacobi.restype = ctypes.c_int
    L.orc_jacobi.argtypes = [i64, p, p, p]
    L.orc_num_cpus.restype = ctypes.c_int
    _lib = L


def lib():
    with _lock:
        if _lib is None:
            _configure(ctypes.CDLL(build()))
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_cpus() -> int:
    """Hardware threads in this process's CPU affinity mask."""
    return int(lib().orc_num_cpus())


# --------------------------------------------------------------------------
# store geometry (Sec. 2.2.1, Figs. 2-4)
# --------------------------------------------------------------------------

def num_reflectors(n: int, b: int, complex_: bool) -> int:
    return int(lib().orc_num_reflectors(n, b, int(complex_)))


def reflector_rows(n: int, b: int, complex_: bool):
    """(r_k, L_k) of every reflector in generation order (0-based rows)."""
    K = num_reflectors(n, b, complex_)
    r = np.zeros(max(K, 1), np.int64)
    L = np.zeros(max(K, 1), np.int64)
    lib().orc_reflector_rows(n, b, int(complex_), _ptr(r), _ptr(L))
    return r[:K], L[:K]


def reflector_stage_sweep(n: int, b: int, complex_: bool):
    """(stage i, sweep j) of every reflector in generation order (0-based)."""
    K = num_reflectors(n, b, complex_)
    i = np.zeros(max(K, 1), np.int64)
    j = np.zeros(max(K, 1), np.int64)
    lib().orc_reflector_stage_sweep(n, b, int(complex_), _ptr(i), _ptr(j))
    return i[:K], j[:K]


# --------------------------------------------------------------------------
# Eq. 6b: band -> tridiagonal by bulge chasing
# --------------------------------------------------------------------------

def bulge_chase(band: np.ndarray, return_work: bool = False):
    """Reduce the banded symmetric/Hermitian matrix given in lower band
    storage ``band[d, c] = B[c+d, c]`` (shape (b+1, n)) to tridiagonal form.

    Returns ``(hh_v, hh_tau, d, e)`` with ``hh_v`` the K x b column-major
    reflector store (flat, reflector k at ``hh_v[k*b:(k+1)*b]``), ``hh_tau``
    (K,), and the real diagonal ``d`` (n,) and sub-diagonal ``e`` (n-1,).
    With ``return_work`` also the reduced (2b+1) x n working band.
    """
    cplx = np.iscomplexobj(band)
    dt = np.complex128 if cplx else np.float64
    b = band.shape[0] - 1
    n = band.shape[1]
    bandF = np.asfortranarray(band.astype(dt))
    K = num_reflectors(n, b, cplx)
    hh_v = np.zeros(max(K * b, 1), dt)
    hh_tau = np.zeros(max(K, 1), dt)
    d = np.zeros(max(n, 1), np.float64)
    e = np.zeros(max(n - 1, 1), np.float64)
    work = np.zeros((2 * b + 1) * max(n, 1), dt) if return_work else None
    fn = lib().orc_bulge_chase_z if cplx else lib().orc_bulge_chase_d
    k = fn(n, b, _ptr(bandF), b + 1, _ptr(hh_v), _ptr(hh_tau), _ptr(d), _ptr(e), _ptr(work))
    assert k == K
    out = (hh_v[: K * b], hh_tau[:K], d[:n], e[: max(n - 1, 0)])
    if return_work:
        return out + (work.reshape((2 * b + 1, max(n, 1)), order="F")[:, :n],)
    return out


# --------------------------------------------------------------------------
# Eq. 6c: tridiagonal eigensolve
# --------------------------------------------------------------------------

def tridiag_ql(d: np.ndarray, e: np.ndarray):
    """Eigenvalues (ascending) and eigenvectors (n x n, Fortran order) of the
    symmetric tridiagonal matrix with diagonal ``d`` and sub-diagonal ``e``."""
    n = len(d)
    dd = np.array(d, np.float64, copy=True)
    ee = np.zeros(max(n, 1), np.float64)
    ee[: n - 1] = e[: n - 1]
    z = np.zeros((n, n), np.float64, order="F")
    rc = lib().orc_tridiag_ql(n, _ptr(dd), _ptr(ee), _ptr(z), max(n, 1))
    if rc != 0:
        raise RuntimeError("QL iteration did not converge")
    return dd, z


def jacobi(a: np.ndarray, vectors: bool = False):
    """Brute-force eigenvalues (ascending) of a dense symmetric matrix; a
    Hermitian matrix goes through its real 2n x 2n embedding and every other
    eigenvalue of the embedding is returned."""
    if np.iscomplexobj(a):
        n = a.shape[0]
        m = np.block([[a.real, -a.imag], [a.imag, a.real]])
        w = jacobi(m)
        return w[0::2]
    n = a.shape[0]
    A = np.asfortranarray(a.astype(np.float64).copy())
    w = np.zeros(max(n, 1), np.float64)
    v = np.zeros((n, n), np.float64, order="F") if vectors else None
    rc = lib().orc_jacobi(n, _ptr(A), _ptr(w), _ptr(v))
    if rc != 0:
        raise RuntimeError("Jacobi did not converge")
    return (w[:n], v) if vectors else w[:n]


# --------------------------------------------------------------------------
# Eq. 6d / Eq. 8: the back-transformation (the path the GPU library computes)
# --------------------------------------------------------------------------

def back_transform(hh_v: np.ndarray, hh_tau: np.ndarray, n: int, b: int, q: np.ndarray, nthreads: int = 1):
    """Apply every stored reflector to the columns of ``q`` (shape (ldq, nev),
    Fortran order, rows 0..n-1 used) in reverse generation order, in place.
    Returns ``q``."""
    cplx = np.iscomplexobj(q)
    dt = np.complex128 if cplx else np.float64
    assert q.dtype == dt and q.flags.f_contiguous
    ldq, nev = q.shape
    v = np.ascontiguousarray(hh_v, dtype=dt)
    t = np.ascontiguousarray(hh_tau, dtype=dt)
    K = num_reflectors(n, b, cplx)
    assert v.size >= K * b and t.size >= K
    fn = lib().orc_back_transform_z if cplx else lib().orc_back_transform_d
    rc = fn(n, b, nev, _ptr(v), _ptr(t), _ptr(q), max(ldq, 1), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle back-transform failed")
    return q


# --------------------------------------------------------------------------
# Eq. 6a: full -> band, and Eq. 6e: band -> full back-transformation
# --------------------------------------------------------------------------

def num_full_reflectors(n: int, b: int) -> int:
    """Reflectors of the full -> band reduction: one per column c = 0..n-b-1."""
    return max(n - b, 0)


def full_to_band(A: np.ndarray, b: int):
    """Reduce the dense symmetric/Hermitian ``A`` (n x n, both triangles) to
    a band matrix of semi-bandwidth ``b``. Returns ``(a, tau)``: ``a``
    (Fortran order) holds the band of B in |i-j| <= b and the reflector of
    column c below it (v[0] = 1 implicit at row c+b, v[1:] in
    ``a[c+b+1:, c]``); ``tau`` has max(n-b, 0) entries."""
    cplx = np.iscomplexobj(A)
    dt = np.complex128 if cplx else np.float64
    n = A.shape[0]
    a = np.asfortranarray(np.array(A, dtype=dt))
    tau = np.zeros(max(n - b, 1), dt)
    fn = lib().orc_full_to_band_z if cplx else lib().orc_full_to_band_d
    k = fn(n, b, _ptr(a), max(n, 1), _ptr(tau))
    assert k == num_full_reflectors(n, b)
    return a, tau[: num_full_reflectors(n, b)]


def band_of(a: np.ndarray, b: int) -> np.ndarray:
    """The dense band matrix B held in the |i-j| <= b entries of ``a``."""
    n = a.shape[0]
    i, j = np.indices((n, n))
    return np.where(np.abs(i - j) <= b, a, 0)


def back_transform_full(a: np.ndarray, tau: np.ndarray, n: int, b: int, q: np.ndarray, nthreads: int = 1):
    """Apply Q1 = H_0 ... H_{n-b-1} (the reflectors held below the band of
    ``a``) to the columns of ``q`` (shape (ldq, nev), Fortran order), last
    reflector first, in place. Returns ``q``."""
    cplx = np.iscomplexobj(q)
    dt = np.complex128 if cplx else np.float64
    assert q.dtype == dt and q.flags.f_contiguous
    ldq, nev = q.shape
    a = np.asfortranarray(a, dtype=dt)
    t = np.ascontiguousarray(tau, dtype=dt)
    assert t.size >= num_full_reflectors(n, b) and a.shape[0] >= n
    fn = lib().orc_back_transform_full_z if cplx else lib().orc_back_transform_full_d
    rc = fn(n, b, nev, _ptr(a), max(a.shape[0], 1), _ptr(t), _ptr(q), max(ldq, 1), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle band -> full back-transform failed")
    return q
