"""Builds and loads libtbbt.so (the CUDA library behind the C ABI in
include/tbbt.h). The library is compiled in-tree for sm_103a only; there is
no fallback: if it is missing or cannot be loaded, every entry point raises."""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libtbbt.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

_lock = threading.Lock()
_lib = None


def sources():
    out = [os.path.join(INCLUDE, "tbbt.h")]
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def nvcc_command(out_path: str):
    return ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
            "-o", out_path, os.path.join(CSRC, "tbbt.cu")]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libtbbt.so if it is missing or older than its sources."""
    os.makedirs(BUILD, exist_ok=True)
    stale = (not os.path.exists(LIB)) or any(os.path.getmtime(s) > os.path.getmtime(LIB) for s in sources())
    if force or stale:
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = nvcc_command(tmp)
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def load():
    """The loaded library with argument types set. Raises if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB):
            raise RuntimeError(f"libtbbt.so is not built ({LIB}); run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB)
        i64, i32, p, c_int = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int
        L.tbbt_status_string.restype = ctypes.c_char_p
        L.tbbt_status_string.argtypes = [c_int]
        L.tbbt_num_reflectors.restype = i64
        L.tbbt_num_reflectors.argtypes = [i64, i64, c_int]
        for name in ("tbbt_trans_ev_tridi_to_band_d", "tbbt_trans_ev_tridi_to_band_z",
                     "tbbt_trans_ev_tridi_to_band_host_d", "tbbt_trans_ev_tridi_to_band_host_z"):
            f = getattr(L, name)
            f.restype = c_int
            f.argtypes = [p, p, i64, i64, i64, p, i64, p]
        L.tbbt_release_cache.restype = c_int
        L.tbbt_release_cache.argtypes = []
        L.tbbt_plan_create.restype = c_int
        L.tbbt_plan_create.argtypes = [ctypes.POINTER(p), c_int, i64, i64, i64, p]
        L.tbbt_plan_set_reflectors.restype = c_int
        L.tbbt_plan_set_reflectors.argtypes = [p, p, p, p]
        L.tbbt_plan_execute.restype = c_int
        L.tbbt_plan_execute.argtypes = [p, p, i64, p]
        L.tbbt_plan_destroy.restype = c_int
        L.tbbt_plan_destroy.argtypes = [p]
        L.tbbt_plan_info.restype = c_int
        L.tbbt_plan_info.argtypes = [p] + [ctypes.POINTER(i32)] * 5
        L.tbbt_stream_check.restype = c_int
        L.tbbt_stream_check.argtypes = [p]
        L.tbbt_trans_ev_tridi_to_band_noalloc.restype = c_int
        L.tbbt_trans_ev_tridi_to_band_noalloc.argtypes = [c_int, p, p, i64, i64, i64, p, i64, p]
        L.tbbt_batch_create.restype = c_int
        L.tbbt_batch_create.argtypes = [ctypes.POINTER(p), i32, p, p]
        L.tbbt_batch_execute.restype = c_int
        L.tbbt_batch_execute.argtypes = [p, p]
        L.tbbt_batch_info.restype = c_int
        L.tbbt_batch_info.argtypes = [p, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                      ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)]
        L.tbbt_batch_destroy.restype = c_int
        L.tbbt_batch_destroy.argtypes = [p]
        for name in ("tbbt_bulge_chase_d", "tbbt_bulge_chase_z"):
            f = getattr(L, name)
            f.restype = c_int
            f.argtypes = [p, i64, i64, i64, p, p, p, p, p]
        for name in ("tbbt_trans_ev_band_to_full_d", "tbbt_trans_ev_band_to_full_z",
                     "tbbt_trans_ev_band_to_full_split_d"):
            f = getattr(L, name)
            f.restype = c_int
            f.argtypes = [p, i64, p, i64, i64, i64, p, i64, p]
        L.tbbt_trans_ev_band_to_full_split_opts_d.restype = c_int
        L.tbbt_trans_ev_band_to_full_split_opts_d.argtypes = [p, i64, p, i64, i64, i64, p, i64, i32, i32, p]
        L.tbbt_tridiag_eig.restype = c_int
        L.tbbt_tridiag_eig.argtypes = [p, p, i64, i64, p, p, i64, c_int, p]
        L.tbbt_fp64_probe.restype = c_int
        L.tbbt_fp64_probe.argtypes = [i32, i32, i32, i64, p, ctypes.POINTER(ctypes.c_double), p]
        L.tbbt_b2f_split_layout_check.restype = i64
        L.tbbt_b2f_split_layout_check.argtypes = [i64, i64, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(i64)]
        L.tbbt_schedule_max_live_rows.restype = i64
        L.tbbt_schedule_max_live_rows.argtypes = [i64, i64, c_int, i32, i32]
        _lib = L
        return L
