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

``emo_oracle_ops.c`` holds the generation around the selection and the
second algorithm family:
  * ``sbx_pair`` / ``pm_value`` / ``variation`` -- random mating, simulated
    binary crossover and polynomial mutation (Appendix S.I).
  * ``pbi`` / ``moead_select`` / ``moead_offspring`` -- the TensorMOEA/D
    environmental selection of Algorithm S.8 and its reproduction.
  * ``igd`` -- inverted generational distance to a reference front.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emo_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "emo_oracle_ops.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp = None

NOT_RANKED = np.iinfo(np.int32).max


def _compile(path: str, extra: list[str], force: bool) -> str:
    if (not force and os.path.exists(path)
            and all(os.path.getmtime(path) >= os.path.getmtime(src) for src in _SRCS)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                           *_SRCS, "-o", tmp, "-lm"])
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction): the single-threaded
    library and, where the compiler has OpenMP, the all-core build of the
    same source (``liboracle_omp.so``). Returns the single-threaded path."""
    path = _compile(_LIB_PATH, [], force)
    try:
        _compile(_OMP_PATH, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass  # no OpenMP runtime: only the single-threaded oracle exists
    return path


def has_parallel() -> bool:
    """True when the all-core build of the oracle is available."""
    build()
    return os.path.exists(_OMP_PATH)


class _Trace(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_void_p), ("z", ctypes.c_void_p), ("extreme", ctypes.c_void_p),
                ("a", ctypes.c_void_p), ("fnorm", ctypes.c_void_p), ("pi", ctypes.c_void_p),
                ("dist", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("picked", ctypes.c_void_p),
                ("last_rank", ctypes.c_int32), ("n_before", ctypes.c_int32),
                ("n_last", ctypes.c_int32), ("fallback", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("near_ties", ctypes.c_int32)]


def lib(parallel: bool = False):
    """The single-threaded oracle library, or with ``parallel`` its all-core
    build (same source and arithmetic, OpenMP over points)."""
    global _lib, _omp
    with _lock:
        if parallel:
            if _omp is None:
                build()
                if not os.path.exists(_OMP_PATH):
                    raise OracleError("the all-core oracle needs gcc with OpenMP")
                _omp = _declare(ctypes.CDLL(_OMP_PATH))
            return _omp
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
        return _lib


def _declare(_lib):
    """Argument and return types of the exported oracle routines."""
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
    vp, i64, dbl, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
    _lib.oracle_sbx_pair.restype = None
    _lib.oracle_sbx_pair.argtypes = [dbl, dbl, dbl, dbl, vp, vp]
    _lib.oracle_pm_value.restype = dbl
    _lib.oracle_pm_value.argtypes = [dbl, dbl, dbl, dbl, dbl]
    _lib.oracle_variation.restype = ctypes.c_int
    _lib.oracle_variation.argtypes = [vp, i64, i64, vp, vp, i64, u64, u64, dbl, dbl, dbl, dbl, vp, vp]
    _lib.oracle_pbi.restype = dbl
    _lib.oracle_pbi.argtypes = [vp, vp, vp, ctypes.c_int, dbl]
    _lib.oracle_moead_select.restype = ctypes.c_int
    _lib.oracle_moead_select.argtypes = [vp, vp, vp, vp, i64, i64, ctypes.c_int, vp, vp, vp,
                                         ctypes.c_int32, dbl, vp, vp, vp]
    _lib.oracle_moead_offspring.restype = ctypes.c_int
    _lib.oracle_moead_offspring.argtypes = [vp, i64, i64, vp, vp, vp, ctypes.c_int32, u64, u64,
                                            dbl, dbl, dbl, vp, vp]
    _lib.oracle_igd.restype = dbl
    _lib.oracle_igd.argtypes = [vp, i64, ctypes.c_int, vp, i64]
    _lib.oracle_threads.restype = ctypes.c_int
    _lib.oracle_threads.argtypes = [ctypes.c_int]
    return _lib


def threads(n: int = 0) -> int:
    """Sets (n > 0) and returns the thread count of the all-core oracle."""
    return int(lib(parallel=True).oracle_threads(int(n)))


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


def nd_sort_deb(F, parallel: bool = False) -> np.ndarray:
    F = _f32(F)
    r = np.zeros(F.shape[0], dtype=np.int32)
    if lib(parallel).oracle_nd_sort_deb(_p(F), F.shape[0], F.shape[1], _p(r)) < 0:
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
                 mode: int = NICHE_EXACT, parallel: bool = False):
    """Survivor indices (ascending) and, with ``trace``, every intermediate.
    ``parallel`` runs the all-core build (identical results)."""
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
    rc = lib(parallel).oracle_nsga3_select_mode(_p(F), n2, m, _p(R), n_r, n_keep,
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


def sbx_pair(x1: float, x2: float, mu: float, eta_c: float) -> tuple[float, float]:
    """The two SBX children of one variable (Appendix S.I), FP64."""
    c1, c2 = ctypes.c_double(), ctypes.c_double()
    lib().oracle_sbx_pair(float(x1), float(x2), float(mu), float(eta_c), ctypes.byref(c1), ctypes.byref(c2))
    return c1.value, c2.value


def pm_value(x: float, lo: float, hi: float, mu: float, eta_m: float) -> float:
    """Polynomial mutation of one variable (Appendix S.I, original form), FP64."""
    return lib().oracle_pm_value(float(x), float(lo), float(hi), float(mu), float(eta_m))


def variation(X, lo, hi, n_off: int, seed: int, generation: int, eta_c: float = 20.0, eta_m: float = 20.0,
              p_c: float = 1.0, p_m: float | None = None):
    """Offspring of one generation (random mating, SBX, PM) and the parent
    index pairs. ``p_m`` defaults to 1/D."""
    X = _f32(X)
    n, d = X.shape
    lo = _f32(np.broadcast_to(np.asarray(lo, np.float32), (d,)))
    hi = _f32(np.broadcast_to(np.asarray(hi, np.float32), (d,)))
    p_m = 1.0 / d if p_m is None else p_m
    out = np.zeros((n_off, d), np.float32)
    parents = np.zeros(((n_off + 1) // 2, 2), np.int32)
    rc = lib().oracle_variation(_p(X), n, d, _p(lo), _p(hi), n_off, seed & 0xFFFFFFFFFFFFFFFF,
                                generation & 0xFFFFFFFFFFFFFFFF, eta_c, eta_m, p_c, p_m, _p(out), _p(parents))
    if rc != 0:
        raise OracleError(f"oracle_variation status {rc}")
    return out, parents


def pbi(f, w, z, theta: float) -> float:
    """PBI aggregation d1 + theta d2 of one objective vector (Section IV-B)."""
    f, w, z = _f32(f).reshape(-1), _f32(w).reshape(-1), _f32(z).reshape(-1)
    return lib().oracle_pbi(_p(f), _p(w), _p(z), f.shape[0], float(theta))


def moead_select(X, F1, O, F2, z, W, I_nb, theta: float = 5.0):
    """TensorMOEA/D environmental selection (Algorithm S.8): X_next, F_next,
    the updated ideal point and, per subproblem, the offspring taken (-1 when
    the current solution stays)."""
    X, F1, O, F2, W = _f32(X), _f32(F1), _f32(O), _f32(F2), _f32(W)
    z = _f32(z).reshape(-1).copy()
    I_nb = np.ascontiguousarray(I_nb, dtype=np.int32)
    n, d = X.shape
    m = F1.shape[1]
    Xn = np.zeros_like(X)
    Fn = np.zeros_like(F1)
    win = np.zeros(n, np.int32)
    rc = lib().oracle_moead_select(_p(X), _p(F1), _p(O), _p(F2), n, d, m, _p(z), _p(W), _p(I_nb),
                                   I_nb.shape[1], float(theta), _p(Xn), _p(Fn), _p(win))
    if rc != 0:
        raise OracleError(f"oracle_moead_select status {rc}")
    return Xn, Fn, z, win


def moead_offspring(X, lo, hi, I_nb, seed: int, generation: int, eta_c: float = 20.0, eta_m: float = 20.0,
                    p_m: float | None = None):
    """One offspring per subproblem from two random neighbours (Algorithm S.7
    reproduction, all subproblems at once) and the parent pairs."""
    X = _f32(X)
    n, d = X.shape
    lo = _f32(np.broadcast_to(np.asarray(lo, np.float32), (d,)))
    hi = _f32(np.broadcast_to(np.asarray(hi, np.float32), (d,)))
    I_nb = np.ascontiguousarray(I_nb, dtype=np.int32)
    p_m = 1.0 / d if p_m is None else p_m
    O = np.zeros_like(X)
    parents = np.zeros((n, 2), np.int32)
    rc = lib().oracle_moead_offspring(_p(X), n, d, _p(lo), _p(hi), _p(I_nb), I_nb.shape[1],
                                      seed & 0xFFFFFFFFFFFFFFFF, generation & 0xFFFFFFFFFFFFFFFF, eta_c, eta_m, p_m,
                                      _p(O), _p(parents))
    if rc != 0:
        raise OracleError(f"oracle_moead_offspring status {rc}")
    return O, parents


def igd(F, Ref, parallel: bool = False) -> float:
    """Inverted generational distance of population F to the front Ref
    (``parallel``: the all-core build, identical result)."""
    F, Ref = _f32(F), _f32(Ref)
    return lib(parallel).oracle_igd(_p(F), F.shape[0], F.shape[1], _p(Ref), Ref.shape[0])
