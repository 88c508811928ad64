"""Python binding of libtbbt (names follow the C ABI in include/tbbt.h).

Argument marshalling only: tensors are passed as raw pointers and the
caller's current CUDA stream; every step of the computation runs in the
library's kernels. PyTorch provides device memory and streams.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _native

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP = range(6)
REAL64, COMPLEX128 = 0, 1


class TbbtError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _native.load().tbbt_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def _check(status: int, where: str):
    if status != OK:
        raise TbbtError(status, where)


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _is_complex_dtype(t) -> bool:
    import torch

    if t.dtype == torch.complex128:
        return True
    if t.dtype == torch.float64:
        return False
    raise TypeError(f"expected float64 or complex128, got {t.dtype}")


def num_reflectors(n: int, nbw: int, is_complex: bool) -> int:
    return int(_native.load().tbbt_num_reflectors(n, nbw, int(is_complex)))


def schedule_max_live_rows(n: int, nbw: int, is_complex: bool, sweeps_per_block: int, stages_per_step: int) -> int:
    return int(_native.load().tbbt_schedule_max_live_rows(n, nbw, int(is_complex), sweeps_per_block, stages_per_step))


def _need_device(t, name: str, dtype=None, min_numel: int = 0):
    """A device API gets raw pointers: reject what would make a kernel read
    outside the caller's memory (a host tensor, a mismatched element type, too
    few elements) before anything reaches the library."""
    if min_numel <= 0 and t.numel() == 0:
        return
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if t.numel() < min_numel:
        raise ValueError(f"{name} has {t.numel()} elements, needs at least {min_numel}")


def _need_flat(t, name: str, dtype, numel: int):
    """A flat (contiguous) device array of at least ``numel`` elements."""
    _need_device(t, name, dtype, numel)
    if numel > 0 and not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _q_layout(q, n):
    """(ldq, nev) of a column-major (Fortran-ordered) 2-D tensor view."""
    if q.dim() != 2:
        raise ValueError("q must be 2-D (ldq >= n rows, nev columns), column-major")
    rows, nev = q.shape
    if rows > 1 and q.numel() > 0 and q.stride(0) != 1:
        raise ValueError("q must be column-major (stride(0) == 1)")
    ldq = q.stride(1) if nev > 1 else max(rows, 1)
    if rows < n:
        raise ValueError("q has fewer than n rows")
    return ldq, nev


def _resolve_ldq(q, n: int, nev: int, ldq):
    """The leading dimension the library is given for q. It is the view's own
    column stride: the kernels touch ldq * (nev - 1) + n elements from q's
    first one, so an ldq larger than the stride (or a row-major view) would
    reach past the caller's memory. An explicit ldq must agree with it."""
    lay, cols = _q_layout(q, n)
    if nev > 0 and cols < nev:
        raise ValueError(f"q has {cols} columns, needs at least {nev}")
    if ldq is None:
        return lay
    if ldq < max(n, 1):
        return ldq  # the library reports a leading dimension below n
    if nev > 1 and ldq != lay:
        raise ValueError(f"ldq={ldq} does not match q's column stride {lay}")
    if nev <= 1 and ldq > lay:
        raise ValueError(f"ldq={ldq} exceeds q's {lay} rows")
    return ldq


def _check_q(q, n: int, nev: int, dtype):
    if n > 0 and nev > 0:
        _need_device(q, "q", dtype, 1)
        if q.dim() != 2 or q.shape[0] < n or q.shape[1] < nev:
            raise ValueError(f"q must be at least {n} x {nev}")


def _check_store_and_q(hh_v, hh_tau, n: int, nbw: int, nev: int, q, cplx: bool):
    import torch

    dt = torch.complex128 if cplx else torch.float64
    if n < 0 or nbw < 1:
        return  # the library reports the shape error
    K = num_reflectors(n, nbw, cplx)
    if K > 0 and nev > 0:
        _need_flat(hh_v, "hh_v", dt, K * nbw)
        _need_flat(hh_tau, "hh_tau", dt, K)
    _check_q(q, n, nev, dt)


def trans_ev_tridi_to_band(hh_v, hh_tau, n: int, nbw: int, nev: int, q, ldq: int | None = None, stream=None):
    """Eq. 6d on device tensors: q[:n, :nev] <- H_0 ... H_{K-1} q[:n, :nev].

    hh_v (K*nbw,), hh_tau (K,), q (ldq x >=nev, column-major) are CUDA
    tensors of dtype float64 (real symmetric) or complex128 (Hermitian)."""
    cplx = _is_complex_dtype(q)
    _check_store_and_q(hh_v, hh_tau, n, nbw, nev, q, cplx)
    ldq = _resolve_ldq(q, n, nev, ldq)
    L = _native.load()
    f = L.tbbt_trans_ev_tridi_to_band_z if cplx else L.tbbt_trans_ev_tridi_to_band_d
    st = f(ctypes.c_void_p(hh_v.data_ptr() if hh_v.numel() else 0),
           ctypes.c_void_p(hh_tau.data_ptr() if hh_tau.numel() else 0),
           n, nbw, nev, ctypes.c_void_p(q.data_ptr() if q.numel() else 0), ldq, _stream_handle(stream))
    _check(st, "tbbt_trans_ev_tridi_to_band")
    return q


def bulge_chase(band, nbw: int | None = None, stream=None):
    """Eq. 6b on the GPU: reduce the banded Hermitian matrix given in lower
    band storage (CUDA tensor, shape (nbw+1, n), column-major: band[d, c] =
    B[c+d, c]) to tridiagonal form. Returns (hh_v (K*nbw,), hh_tau (K,),
    d (n,), e (n-1,)) as CUDA tensors; the store is in generation order, ready
    for trans_ev_tridi_to_band or a Plan."""
    import torch

    cplx = _is_complex_dtype(band)
    if band.dim() != 2:
        raise ValueError("band must be 2-D, (nbw+1) x n")
    if nbw is None:
        nbw = band.shape[0] - 1
    n = band.shape[1]
    if band.shape[0] < nbw + 1:
        raise ValueError("band must have at least nbw+1 rows")
    _need_device(band, "band")
    if band.numel() and band.stride(0) != 1:
        raise ValueError("band must be column-major (stride 1 along the band index)")
    ldb = band.stride(1) if n > 1 else nbw + 1
    K = num_reflectors(n, nbw, cplx)
    dev = band.device
    vdt = torch.complex128 if cplx else torch.float64
    hh_v = torch.zeros(K * nbw, dtype=vdt, device=dev)
    hh_tau = torch.zeros(K, dtype=vdt, device=dev)
    d = torch.zeros(n, dtype=torch.float64, device=dev)
    e = torch.zeros(max(n - 1, 0), dtype=torch.float64, device=dev)
    L = _native.load()
    f = L.tbbt_bulge_chase_z if cplx else L.tbbt_bulge_chase_d

    def ptr(t):
        return ctypes.c_void_p(t.data_ptr() if t.numel() else 0)

    st = f(ptr(band), ldb, n, nbw, ptr(hh_v), ptr(hh_tau), ptr(d), ptr(e), _stream_handle(stream))
    _check(st, "tbbt_bulge_chase")
    return hh_v, hh_tau, d, e


def tridiag_eig(d, e, nev: int, complex_out: bool = False, x=None, stream=None):
    """Eq. 6c on the GPU: the nev smallest eigenvalues (ascending) and their
    orthonormal eigenvectors of the symmetric tridiagonal matrix with
    diagonal ``d`` (n,) and sub-diagonal ``e`` (n-1,), float64 CUDA tensors.
    Returns (w (nev,), X (n x nev, column-major)); X is complex128 with zero
    imaginary parts when ``complex_out`` (the X of a Hermitian problem), or
    written into ``x`` if given (column-major, ldx >= n)."""
    import torch

    n = int(d.numel())
    if nev < 0 or nev > n:
        raise ValueError(f"nev={nev} outside [0, {n}]")
    _need_flat(d, "d", torch.float64, n)
    _need_flat(e, "e", torch.float64, max(n - 1, 0))
    dt = torch.complex128 if complex_out else torch.float64
    w = torch.empty(nev, dtype=torch.float64, device=d.device)
    if x is None:
        x = torch.empty((nev, n), dtype=dt, device=d.device).t()
    else:
        _check_q(x, n, nev, dt)
    ldx = _resolve_ldq(x, n, nev, None)
    st = _native.load().tbbt_tridiag_eig(
        ctypes.c_void_p(d.data_ptr() if n else 0), ctypes.c_void_p(e.data_ptr() if n > 1 else 0), n, nev,
        ctypes.c_void_p(w.data_ptr() if nev else 0), ctypes.c_void_p(x.data_ptr() if x.numel() else 0), ldx,
        COMPLEX128 if complex_out else REAL64, _stream_handle(stream))
    _check(st, "tbbt_tridiag_eig")
    return w, x


def trans_ev_band_to_full(a, tau, n: int, nbw: int, nev: int, q, stream=None, variant: int = 0,
                          wait_timeout_ms: int = 0, debug_withhold_cta: int = -1):
    """Eq. 6e on device tensors: q[:n, :nev] <- H_0 ... H_{n-nbw-1} q[:n, :nev]
    with the full -> band reflectors held LAPACK-style below the band of
    ``a`` (n x n, column-major; reflector c has v[0] = 1 at row c+nbw and
    v[1:] in a[c+nbw+1:, c]) and ``tau`` (n-nbw entries). float64 or
    complex128 CUDA tensors; q column-major. ``variant``: VARIANT_FP64 (0)
    or, for float64 data, VARIANT_SPLIT_BF16_TC (2), the digit-slice form on
    the tensor cores; for that form ``wait_timeout_ms`` bounds the waits
    between its CTAs (0: 20 s) and ``debug_withhold_cta`` (a test hook, -1 in
    normal use) makes one CTA's W publications go uncounted."""
    cplx = _is_complex_dtype(q)
    if variant not in (VARIANT_FP64, VARIANT_SPLIT_BF16_TC) or (cplx and variant != VARIANT_FP64):
        raise ValueError("variant must be VARIANT_FP64, or VARIANT_SPLIT_BF16_TC for float64 data")
    K1 = max(n - nbw, 0) if nbw >= 1 else 0
    if K1 > 0 and nev > 0:
        if a.dim() != 2 or a.shape[0] < n or a.shape[1] < K1 or (a.shape[1] > 1 and a.stride(0) != 1):
            raise ValueError(f"a must be a column-major 2-D tensor with at least {n} rows and {K1} columns")
        _need_device(a, "a", q.dtype, 1)
        _need_flat(tau, "tau", q.dtype, K1)
        _check_q(q, n, nev, q.dtype)
    elif a.dim() != 2:
        raise ValueError("a must be 2-D")
    lda = a.stride(1) if a.shape[1] > 1 else max(a.shape[0], 1)
    ldq, _ = _q_layout(q, n)
    L = _native.load()
    if cplx:
        f = L.tbbt_trans_ev_band_to_full_z
    elif variant == VARIANT_SPLIT_BF16_TC:
        f = L.tbbt_trans_ev_band_to_full_split_d
    else:
        f = L.tbbt_trans_ev_band_to_full_d

    def ptr(t):
        return ctypes.c_void_p(t.data_ptr() if t.numel() else 0)

    if variant == VARIANT_SPLIT_BF16_TC:
        st = L.tbbt_trans_ev_band_to_full_split_opts_d(ptr(a), lda, ptr(tau), n, nbw, nev, ptr(q), ldq,
                                                       wait_timeout_ms, debug_withhold_cta, _stream_handle(stream))
    else:
        st = f(ptr(a), lda, ptr(tau), n, nbw, nev, ptr(q), ldq, _stream_handle(stream))
    _check(st, "tbbt_trans_ev_band_to_full")
    return q


def _check_host_args(hh_v, hh_tau, n: int, nbw: int, nev: int, q, ldq: int, cplx: bool):
    """The host entry point copies from these buffers (and back into q, at
    pitch ldq): host memory, the problem's element type, long enough."""
    if n < 1 or nbw < 1 or nev < 1:
        return
    K = num_reflectors(n, nbw, cplx)
    want = np.complex128 if cplx else np.float64
    q_need = ldq * (nev - 1) + n
    for name, t, need in (("hh_v", hh_v, K * nbw), ("hh_tau", hh_tau, K), ("q", q, q_need)):
        if need <= 0:
            continue
        if isinstance(t, np.ndarray):
            dt, size = t.dtype, t.size
        else:
            if t.is_cuda:
                raise ValueError(f"{name} must be in host memory for the host entry point")
            dt, size = np.dtype(str(t.dtype).replace("torch.", "")), t.numel()
        if dt != want:
            raise TypeError(f"{name} has dtype {dt}, expected {np.dtype(want)}")
        if size < need:
            raise ValueError(f"{name} has {size} elements, needs at least {need}")


def trans_ev_tridi_to_band_host(hh_v, hh_tau, n: int, nbw: int, nev: int, q, ldq: int | None = None, stream=None,
                                synchronize: bool = True):
    """The same with every array in host memory (numpy arrays or CPU
    tensors; pinned memory makes the copies asynchronous). q is updated in
    place; with ``synchronize`` the call waits for the stream."""
    def ptr(a):
        if isinstance(a, np.ndarray):
            return a.ctypes.data if a.size else 0
        return a.data_ptr() if a.numel() else 0

    if isinstance(q, np.ndarray):
        cplx = np.iscomplexobj(q)
        if q.ndim != 2:
            raise ValueError("q must be 2-D (ldq >= n rows, nev columns), Fortran-ordered")
        if not q.flags.f_contiguous:
            raise ValueError("q must be Fortran-ordered")
        rows, cols = q.shape
        if rows < n or (nev > 0 and cols < nev):
            raise ValueError(f"q must be at least {n} x {nev}")
        if ldq is None:
            ldq = max(rows, 1)
        elif ldq >= max(n, 1) and ldq != max(rows, 1) and nev > 1:
            raise ValueError(f"ldq={ldq} does not match q's leading dimension {rows}")
        elif ldq > max(rows, 1):
            raise ValueError(f"ldq={ldq} exceeds q's {rows} rows")
    else:
        cplx = _is_complex_dtype(q)
        if q.is_cuda:
            raise ValueError("q must be in host memory for the host entry point")
        ldq = _resolve_ldq(q, n, nev, ldq)
    _check_host_args(hh_v, hh_tau, n, nbw, nev, q, ldq, cplx)
    L = _native.load()
    f = L.tbbt_trans_ev_tridi_to_band_host_z if cplx else L.tbbt_trans_ev_tridi_to_band_host_d
    h = _stream_handle(stream)
    st = f(ctypes.c_void_p(ptr(hh_v)), ctypes.c_void_p(ptr(hh_tau)), n, nbw, nev, ctypes.c_void_p(ptr(q)), ldq, h)
    _check(st, "tbbt_trans_ev_tridi_to_band_host")
    if synchronize:
        _check(L.tbbt_stream_check(h), "tbbt_stream_check")
    return q


def trans_ev_tridi_to_band_noalloc(hh_v, hh_tau, n: int, nbw: int, nev: int, q, ldq: int | None = None,
                                   stream=None):
    """The same as trans_ev_tridi_to_band, through the entry point that
    allocates no memory (for callers that cannot allocate; its scratch is a
    fixed 32 MiB array per device, and concurrent calls race on it). Raises
    TbbtError (ENOTSUP) for problems whose scratch does not fit."""
    cplx = _is_complex_dtype(q)
    _check_store_and_q(hh_v, hh_tau, n, nbw, nev, q, cplx)
    ldq = _resolve_ldq(q, n, nev, ldq)
    st = _native.load().tbbt_trans_ev_tridi_to_band_noalloc(
        COMPLEX128 if cplx else REAL64, ctypes.c_void_p(hh_v.data_ptr() if hh_v.numel() else 0),
        ctypes.c_void_p(hh_tau.data_ptr() if hh_tau.numel() else 0), n, nbw, nev,
        ctypes.c_void_p(q.data_ptr() if q.numel() else 0), ldq, _stream_handle(stream))
    _check(st, "tbbt_trans_ev_tridi_to_band_noalloc")
    return q


def release_cache():
    _check(_native.load().tbbt_release_cache(), "tbbt_release_cache")


def stream_check(stream=None):
    """Synchronise the stream and raise TbbtError if an in-kernel wait gave up."""
    _check(_native.load().tbbt_stream_check(_stream_handle(stream)), "tbbt_stream_check")


class Options(ctypes.Structure):
    _fields_ = [("sweeps_per_block", ctypes.c_int32), ("stages_per_step", ctypes.c_int32),
                ("wait_timeout_ms", ctypes.c_int32), ("debug_withhold_unit_plus1", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


VARIANT_FP64, VARIANT_SPLIT_BF16, VARIANT_SPLIT_BF16_TC = 0, 1, 2


class Plan:
    """tbbt_plan: workspace allocated once, then set_reflectors / execute."""

    def __init__(self, dtype_complex: bool, n: int, nbw: int, nev: int, sweeps_per_block: int = 0,
                 stages_per_step: int = 0, wait_timeout_ms: int = 0, debug_withhold_unit: int = -1,
                 variant: int = 0):
        self.n, self.nbw, self.nev, self.complex = n, nbw, nev, dtype_complex
        self._h = ctypes.c_void_p()
        opt = Options(sweeps_per_block, stages_per_step, wait_timeout_ms, debug_withhold_unit + 1, variant)
        st = _native.load().tbbt_plan_create(ctypes.byref(self._h), COMPLEX128 if dtype_complex else REAL64,
                                             n, nbw, nev, ctypes.byref(opt))
        _check(st, "tbbt_plan_create")

    def set_reflectors(self, hh_v, hh_tau, stream=None):
        import torch

        K = num_reflectors(self.n, self.nbw, self.complex)
        if K > 0:
            dt = torch.complex128 if self.complex else torch.float64
            _need_flat(hh_v, "hh_v", dt, K * self.nbw)
            _need_flat(hh_tau, "hh_tau", dt, K)
        st = _native.load().tbbt_plan_set_reflectors(
            self._h, ctypes.c_void_p(hh_v.data_ptr() if hh_v.numel() else 0),
            ctypes.c_void_p(hh_tau.data_ptr() if hh_tau.numel() else 0), _stream_handle(stream))
        _check(st, "tbbt_plan_set_reflectors")

    def execute(self, q, ldq: int | None = None, stream=None):
        import torch

        _check_q(q, self.n, self.nev, torch.complex128 if self.complex else torch.float64)
        ldq = _resolve_ldq(q, self.n, self.nev, ldq)
        st = _native.load().tbbt_plan_execute(self._h, ctypes.c_void_p(q.data_ptr() if q.numel() else 0), ldq,
                                              _stream_handle(stream))
        _check(st, "tbbt_plan_execute")
        return q

    def info(self):
        vals = [ctypes.c_int32() for _ in range(5)]
        _check(_native.load().tbbt_plan_info(self._h, *[ctypes.byref(v) for v in vals]), "tbbt_plan_info")
        keys = ("sweeps_per_block", "stages_per_step", "ring_rows", "smem_bytes", "blocks")
        return dict(zip(keys, (v.value for v in vals)))

    def close(self):
        if self._h:
            _native.load().tbbt_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem(ctypes.Structure):
    """tbbt_problem: one problem of a batch (device pointers)."""
    _fields_ = [("dtype", ctypes.c_int), ("reserved0", ctypes.c_int32), ("n", ctypes.c_int64),
                ("nbw", ctypes.c_int64), ("nev", ctypes.c_int64), ("hh_v", ctypes.c_void_p),
                ("hh_tau", ctypes.c_void_p), ("q", ctypes.c_void_p), ("ldq", ctypes.c_int64)]


class BatchOptions(ctypes.Structure):
    _fields_ = [("sweeps_per_block", ctypes.c_int32), ("stages_per_step_real", ctypes.c_int32),
                ("stages_per_step_complex", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("autotune_cache", ctypes.c_char_p), ("wait_timeout_ms", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class Batch:
    """tbbt_batch: many problems back-transformed by one persistent launch,
    replayed from a CUDA graph. ``problems`` is a list of
    ``(hh_v, hh_tau, n, nbw, nev, q)`` with CUDA tensors (q column-major);
    the tensors must stay alive and at the same addresses while the batch is
    used (the batch keeps references)."""

    def __init__(self, problems, sweeps_per_block: int = 0, stages_per_step_real: int = 0,
                 stages_per_step_complex: int = 0, autotune: bool = False, autotune_cache: str | None = None,
                 wait_timeout_ms: int = 0):
        self._keep = []
        arr = (Problem * len(problems))()
        for i, (hh_v, hh_tau, n, nbw, nev, q) in enumerate(problems):
            cplx = _is_complex_dtype(q)
            _check_store_and_q(hh_v, hh_tau, n, nbw, nev, q, cplx)
            ldq, _ = _q_layout(q, n)
            arr[i] = Problem(COMPLEX128 if cplx else REAL64, 0, n, nbw, nev,
                             hh_v.data_ptr() if hh_v.numel() else None,
                             hh_tau.data_ptr() if hh_tau.numel() else None,
                             q.data_ptr() if q.numel() else None, ldq)
            self._keep += [hh_v, hh_tau, q]
        self._cache = autotune_cache.encode() if autotune_cache else None
        opt = BatchOptions(sweeps_per_block, stages_per_step_real, stages_per_step_complex, int(autotune),
                           self._cache, wait_timeout_ms)
        self._h = ctypes.c_void_p()
        st = _native.load().tbbt_batch_create(ctypes.byref(self._h), len(problems), ctypes.cast(arr, ctypes.c_void_p),
                                              ctypes.byref(opt))
        _check(st, "tbbt_batch_create")

    def execute(self, stream=None):
        _check(_native.load().tbbt_batch_execute(self._h, _stream_handle(stream)), "tbbt_batch_execute")

    def info(self):
        i32 = [ctypes.c_int32() for _ in range(4)]
        units = ctypes.c_int64()
        tuned = ctypes.c_int32()
        _check(_native.load().tbbt_batch_info(self._h, *[ctypes.byref(v) for v in i32], ctypes.byref(units),
                                              ctypes.byref(tuned)), "tbbt_batch_info")
        return {"sweeps_per_block": i32[0].value, "stages_real": i32[1].value, "stages_complex": i32[2].value,
                "blocks": i32[3].value, "units": units.value, "tuned": bool(tuned.value)}

    def close(self):
        if self._h:
            _native.load().tbbt_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
