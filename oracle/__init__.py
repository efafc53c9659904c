"""FP64 CPU oracle for NSGA-III environmental selection -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``emo_oracle.c`` (plain C,
FP64, no fused multiply-add), which shares nothing with the CUDA path.

Functions follow the paper (arXiv 2503.20286):
  * ``dominance_bits`` / ``domination_counts`` -- Listing 1 (Section III-C).
  * ``nd_sort_deb`` -- Algorithm S.2; ``nd_sort_peel`` -- Algorithm S.3.
  * ``nsga3_select`` -- Algorithm S.1 with Algorithm S.5 and the
    perpendicular-distance association of Section IV-A.
  * ``philox4x32_10`` -- the counter-based generator whose stream breaks the
    ties of the niching step (Salmon et al., SC'11).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emo_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NOT_RANKED = np.iinfo(np.int32).max


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction). Returns the .so path."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Trace(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_void_p), ("z", ctypes.c_void_p), ("extreme", ctypes.c_void_p),
                ("a", ctypes.c_void_p), ("fnorm", ctypes.c_void_p), ("pi", ctypes.c_void_p),
                ("dist", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("picked", ctypes.c_void_p),
                ("last_rank", ctypes.c_int32), ("n_before", ctypes.c_int32),
                ("n_last", ctypes.c_int32), ("fallback", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("near_ties", ctypes.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.oracle_nd_sort_deb.restype = ctypes.c_int64
            _lib.oracle_nd_sort_peel.restype = ctypes.c_int64
            _lib.oracle_nsga3_select.restype = ctypes.c_int
            _lib.oracle_nsga3_select.argtypes = [
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int32,
                ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                ctypes.POINTER(_Trace)]
            _lib.oracle_hype_select.restype = ctypes.c_int
            _lib.oracle_hype_select.argtypes = [
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            _lib.oracle_nsga3_select_mode.restype = ctypes.c_int
            _lib.oracle_nsga3_select_mode.argtypes = [
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int32,
                ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                ctypes.POINTER(_Trace)]
            _lib.oracle_dominance_bits.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                                   ctypes.c_void_p, ctypes.c_int64]
            _lib.oracle_domination_counts.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                                      ctypes.c_void_p]
            _lib.oracle_nd_sort_deb.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                                ctypes.c_void_p]
            _lib.oracle_nd_sort_peel.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                                 ctypes.c_void_p]
            _lib.oracle_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            _lib.oracle_dominates.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        return _lib


def _f32(F) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(F, dtype=np.float32))


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def dominates(a, b) -> bool:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return bool(lib().oracle_dominates(_p(a), _p(b), a.shape[0]))


def dominance_bits(F, ld: int | None = None) -> np.ndarray:
    """Bit-packed ``D``: row i, word w, bit b <=> F_i dominates F_{32w+b}."""
    F = _f32(F)
    n, m = F.shape
    ld = (n + 31) // 32 if ld is None else ld
    D = np.zeros((n, ld), dtype=np.uint32)
    lib().oracle_dominance_bits(_p(F), n, m, _p(D), ld)
    return D


def domination_counts(F) -> np.ndarray:
    F = _f32(F)
    c = np.zeros(F.shape[0], dtype=np.int32)
    lib().oracle_domination_counts(_p(F), F.shape[0], F.shape[1], _p(c))
    return c


def nd_sort_deb(F) -> np.ndarray:
    F = _f32(F)
    r = np.zeros(F.shape[0], dtype=np.int32)
    if lib().oracle_nd_sort_deb(_p(F), F.shape[0], F.shape[1], _p(r)) < 0:
        raise MemoryError("oracle nd sort")
    return r


def nd_sort_peel(F) -> np.ndarray:
    F = _f32(F)
    r = np.zeros(F.shape[0], dtype=np.int32)
    if lib().oracle_nd_sort_peel(_p(F), F.shape[0], F.shape[1], _p(r)) < 0:
        raise MemoryError("oracle peel")
    return r


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


class OracleError(RuntimeError):
    pass


NICHE_EXACT = 0    # niching of Algorithm S.1 (level form)
NICHE_ONESHOT = 1  # one-shot niche selection of Algorithm S.4 + Update-Rank (Algorithm S.6)


def nsga3_select(F, R, n_keep: int, seed: int, generation: int = 0, trace: bool = True,
                 mode: int = NICHE_EXACT):
    """Survivor indices (ascending) and, with ``trace``, every intermediate."""
    F = _f32(F)
    R = _f32(R)
    n2, m = F.shape
    n_r = R.shape[0]
    surv = np.zeros(n_keep, dtype=np.int32)
    t = _Trace()
    bufs = {}
    if trace:
        bufs = {"rank": np.zeros(n2, np.int32), "z": np.zeros(m, np.float64),
                "extreme": np.zeros(m, np.int32), "a": np.zeros(m, np.float64),
                "fnorm": np.zeros((n2, m), np.float64), "pi": np.zeros(n2, np.int32),
                "dist": np.zeros(n2, np.float64), "rho": np.zeros(n_r, np.int32),
                "picked": np.zeros(n2, np.uint8)}
        for k, v in bufs.items():
            setattr(t, k, _p(v))
    rc = lib().oracle_nsga3_select_mode(_p(F), n2, m, _p(R), n_r, n_keep,
                                        seed & 0xFFFFFFFFFFFFFFFF, generation & 0xFFFFFFFFFFFFFFFF, int(mode),
                                        _p(surv), ctypes.byref(t))
    if rc != 0:
        raise OracleError(f"oracle_nsga3_select status {rc}")
    out = dict(bufs)
    for k in ("last_rank", "n_before", "n_last", "fallback", "n_levels", "near_ties"):
        out[k] = int(getattr(t, k))
    return surv, out


def hype_select(F, v_ref, U, n_keep: int):
    """TensorHypE selection (Algorithms S.10, S.11): survivors (ascending),
    the estimated hypervolume contribution of every point and l. ``U`` holds
    the s x m uniform [0, 1) numbers of the Monte Carlo samples."""
    F = _f32(F)
    v_ref = _f32(v_ref).reshape(-1)
    U = _f32(U)
    n2, m = F.shape
    surv = np.zeros(n_keep, dtype=np.int32)
    vhv = np.zeros(n2, dtype=np.float64)
    last = np.zeros(1, dtype=np.int32)
    rc = lib().oracle_hype_select(_p(F), n2, m, _p(v_ref), _p(U), U.shape[0], n_keep, _p(surv), _p(vhv), _p(last))
    if rc != 0:
        raise OracleError(f"oracle_hype_select status {rc}")
    return surv, vhv, int(last[0])
