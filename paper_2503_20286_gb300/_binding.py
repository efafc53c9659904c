"""ctypes binding of ``libemo.so`` (include/emo.h) with torch tensors.

Argument marshalling only: every step of the computation runs in the CUDA
library. Functions keep the C names. Tensors must live on the current CUDA
device; calls are enqueued on ``torch.cuda.current_stream()`` unless a
stream is given. There is no CPU fallback: a missing or unloadable library
raises ``EmoLibraryError``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

EMO_OK = 0
STATUS_NAMES = {0: "EMO_OK", 1: "EMO_ERR_INVALID_ARG", 2: "EMO_ERR_NONFINITE", 3: "EMO_ERR_WORKSPACE",
                4: "EMO_ERR_CUDA", 5: "EMO_ERR_TIMEOUT", 6: "EMO_ERR_NOT_IMPLEMENTED"}
EMO_OP_DOMINANCE, EMO_OP_ND_RANK, EMO_OP_NSGA3_SELECT, EMO_OP_HYPE_SELECT, EMO_OP_MOEAD_SELECT, EMO_OP_IGD, \
    EMO_OP_SELECT_RANKED, EMO_OP_DOMINANCE_WS = range(8)
EMO_SHAPE_LINEAR, EMO_SHAPE_SPHERE = 0, 1
EMO_NOT_RANKED = 2147483647
EMO_NICHE_EXACT, EMO_NICHE_ONESHOT = 0, 1
EMO_MAX_BATCH = 128

_lock = threading.Lock()
_lib = None


class EmoLibraryError(RuntimeError):
    pass


class EmoError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")
        self.status = status


class SelectInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("status", "last_rank", "n_before", "n_last", "fallback_used",
                                               "n_recheck", "n_fronts", "n_levels")]


class SelectDebug(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("rank", "z", "extreme", "a", "fnorm", "pi", "dist", "rho",
                                                "picked")]


class Problem(ctypes.Structure):
    _fields_ = [("F", ctypes.c_void_p), ("R", ctypes.c_void_p), ("survivors", ctypes.c_void_p),
                ("info", ctypes.c_void_p), ("n2", ctypes.c_int64), ("n_keep", ctypes.c_int64),
                ("m", ctypes.c_int32), ("n_r", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("generation", ctypes.c_uint64), ("niche_mode", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False) -> ctypes.CDLL:
    """The loaded CUDA library; raises when it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise EmoLibraryError(f"{path} is missing: run paper_2503_20286_gb300.build.build()")
                _build.build()
            try:
                L = ctypes.CDLL(path)
            except OSError as e:
                raise EmoLibraryError(f"cannot load {path}: {e}") from e
            vp, i64, i32, u64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
            L.emo_workspace_size.restype = sz
            L.emo_workspace_size.argtypes = [ctypes.c_int, i64, i32, i32]
            L.emo_dominance.restype = ctypes.c_int
            L.emo_dominance.argtypes = [vp, i64, i32, vp, i64, vp, vp]
            L.emo_dominance_ws.restype = ctypes.c_int
            L.emo_dominance_ws.argtypes = [vp, i64, i32, vp, i64, vp, vp, sz, vp]
            L.emo_dominance_cols.restype = ctypes.c_int
            L.emo_dominance_cols.argtypes = [vp, i64, i32, i64, i64, vp, i64, vp, vp]
            L.emo_front_counts.restype = ctypes.c_int
            L.emo_front_counts.argtypes = [vp, i64, i64, vp, i64, vp, vp, vp]
            L.emo_nsga3_select_ranked.restype = ctypes.c_int
            L.emo_nsga3_select_ranked.argtypes = [vp, i64, i32, vp, i32, i64, u64, u64, vp, vp, vp, vp, sz, vp]
            L.emo_nd_rank.restype = ctypes.c_int
            L.emo_nsga3_associate_range.restype = ctypes.c_int
            L.emo_nsga3_associate_range.argtypes = [vp, i64, i32, vp, i32, i64, vp, i64, i64, vp, vp, vp, vp, vp, sz,
                                                    vp]
            L.emo_nsga3_niche_given.restype = ctypes.c_int
            L.emo_nsga3_niche_given.argtypes = [i64, i32, i64, u64, u64, i32, vp, vp, vp, vp, vp, i64, vp, vp, vp, sz,
                                                vp]
            L.emo_nd_rank.argtypes = [vp, i64, i32, i64, vp, vp, vp, sz, vp]
            L.emo_nsga3_select.restype = ctypes.c_int
            L.emo_nsga3_select.argtypes = [vp, i64, i32, vp, i32, i64, u64, u64, vp, vp, vp, sz, vp]
            L.emo_moead_select.restype = ctypes.c_int
            L.emo_moead_select.argtypes = [vp, vp, vp, vp, i64, i64, i32, vp, vp, vp, i32, ctypes.c_double,
                                           vp, vp, vp, vp, vp, sz, vp]
            dbl = ctypes.c_double
            L.emo_variation.restype = ctypes.c_int
            L.emo_variation.argtypes = [vp, i64, i64, vp, vp, i64, u64, u64, dbl, dbl, dbl, dbl, vp, vp, vp]
            L.emo_standin_objectives.restype = ctypes.c_int
            L.emo_standin_objectives.argtypes = [vp, i64, i64, i32, i32, vp, vp]
            L.emo_igd.restype = ctypes.c_int
            L.emo_igd.argtypes = [vp, i64, i32, vp, i64, vp, vp, sz, vp]
            L.emo_generation_workspace_size.restype = sz
            L.emo_generation_workspace_size.argtypes = [i64, i64, i32, i32]
            L.emo_nsga3_generation.restype = ctypes.c_int
            L.emo_nsga3_generation.argtypes = [vp, vp, i64, i64, i32, vp, i32, i32, u64, u64, dbl, dbl, dbl, dbl,
                                               i32, vp, vp, sz, vp]
            L.emo_autotune.restype = ctypes.c_int
            L.emo_autotune.argtypes = [i32, i64, ctypes.c_char_p]
            L.emo_launch_shape.restype = ctypes.c_int
            L.emo_launch_shape.argtypes = [i32, i64, ctypes.c_void_p]
            L.emo_autotune_reset.restype = None
            L.emo_autotune_reset.argtypes = []
            L.emo_get_last_device_status.restype = ctypes.c_int
            L.emo_get_last_device_status.argtypes = [vp, vp]
            L.emo_hype_select.restype = ctypes.c_int
            L.emo_hype_select.argtypes = [vp, i64, i32, vp, vp, i32, i64, vp, vp, vp, vp, sz, vp]
            L.emo_nsga3_select_ex.restype = ctypes.c_int
            L.emo_nsga3_select_ex.argtypes = [vp, i64, i32, vp, i32, i64, u64, u64, i32, vp, vp,
                                              ctypes.POINTER(SelectDebug), vp, sz, vp]
            L.emo_nsga3_select_debug.restype = ctypes.c_int
            L.emo_nsga3_select_debug.argtypes = [vp, i64, i32, vp, i32, i64, u64, u64, vp, vp,
                                                 ctypes.POINTER(SelectDebug), vp, sz, vp]
            L.emo_batch_workspace_size.restype = sz
            L.emo_batch_workspace_size.argtypes = [ctypes.POINTER(Problem), i32]
            L.emo_nsga3_select_batch.restype = ctypes.c_int
            L.emo_nsga3_select_batch.argtypes = [ctypes.POINTER(Problem), i32, vp, sz, vp]
            L.emo_workspace_status.restype = ctypes.c_int
            L.emo_workspace_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32)]
            L.emo_set_spin_budget.restype = None
            L.emo_set_spin_budget.argtypes = [i64]
            L.emo_status_string.restype = ctypes.c_char_p
            L.emo_status_string.argtypes = [ctypes.c_int]
            L.emo_version.restype = i32
            L.emo_version.argtypes = []
            L.emo_nsga3_select_noalloc.restype = ctypes.c_int
            L.emo_nsga3_select_noalloc.argtypes = [vp, i64, i32, vp, i32, i64, u64, u64, vp, vp, vp]
            L.emo_device_report.restype = i32
            L.emo_device_report.argtypes = [ctypes.c_char_p, i32]
            L.emo_set_stage_timing.restype = None
            L.emo_set_stage_timing.argtypes = [i32]
            L.emo_stage_times.restype = i32
            L.emo_stage_times.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_char_p), i32]
            _lib = L
        return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(rc: int, what: str) -> None:
    if rc != EMO_OK:
        raise EmoError(rc, what)


def _ws(nbytes: int, ws, device) -> torch.Tensor:
    if ws is not None:
        if ws.numel() * ws.element_size() < nbytes:
            raise EmoError(3, "workspace")
        return ws
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def emo_workspace_size(op: int, n2: int, m: int, n_r: int = 0) -> int:
    return int(lib().emo_workspace_size(op, n2, m, n_r))


def emo_dominance(F: torch.Tensor, D: torch.Tensor | None = None, dom_count: torch.Tensor | None = None,
                  with_count: bool = True, stream=None):
    """Bit-packed dominance matrix ``D [n2, ld]`` (uint32 stored as int32) and dominator counts."""
    n2, m = F.shape
    ld = (n2 + 31) // 32
    if D is None:
        D = torch.empty((n2, ld), dtype=torch.int32, device=F.device)
    if dom_count is None and with_count:
        dom_count = torch.empty(n2, dtype=torch.int32, device=F.device)
    _check(lib().emo_dominance(_ptr(F), n2, m, _ptr(D), D.shape[1], _ptr(dom_count), _stream(stream)),
           "emo_dominance")
    return D, dom_count


def emo_dominance_ws(F: torch.Tensor, D: torch.Tensor | None = None, dom_count: torch.Tensor | None = None,
                     ws: torch.Tensor | None = None, stream=None):
    """emo_dominance through sorted prefix sets (m <= 5; a workspace)."""
    n2, m = F.shape
    ld = (n2 + 31) // 32
    if D is None:
        D = torch.empty((n2, ld), dtype=torch.int32, device=F.device)
    if dom_count is None:
        dom_count = torch.empty(n2, dtype=torch.int32, device=F.device)
    nbytes = emo_workspace_size(EMO_OP_DOMINANCE_WS, n2, m, 0)
    wsp = None
    if nbytes:
        ws = _ws(nbytes, ws, F.device)
        wsp = _ptr(ws)
    _check(lib().emo_dominance_ws(_ptr(F), n2, m, _ptr(D), D.shape[1], _ptr(dom_count), wsp, nbytes,
                                  _stream(stream)), "emo_dominance_ws")
    return D, dom_count


def emo_dominance_cols(F: torch.Tensor, col_lo: int, col_hi: int, D: torch.Tensor | None = None,
                       dom_count: torch.Tensor | None = None, stream=None):
    """Columns [col_lo, col_hi) of the dominance matrix (every row) and their
    dominator counts; col_lo a multiple of 1024."""
    n2, m = F.shape
    ncols = col_hi - col_lo
    if D is None:
        D = torch.empty((n2, (ncols + 31) // 32), dtype=torch.int32, device=F.device)
    if dom_count is None:
        dom_count = torch.empty(ncols, dtype=torch.int32, device=F.device)
    _check(lib().emo_dominance_cols(_ptr(F), n2, m, int(col_lo), int(col_hi), _ptr(D), D.shape[1], _ptr(dom_count),
                                    _stream(stream)), "emo_dominance_cols")
    return D, dom_count


def emo_front_counts(D: torch.Tensor, ncols: int, rows: torch.Tensor, counts: torch.Tensor,
                     next_front: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """One peeling step on a rank's columns: counts -= rows' bits; returns
    the uint8 flags of the columns whose count reached zero."""
    if next_front is None:
        next_front = torch.empty(ncols, dtype=torch.uint8, device=D.device)
    _check(lib().emo_front_counts(_ptr(D), D.shape[1], int(ncols), _ptr(rows) if rows.numel() else None,
                                  rows.numel(), _ptr(counts), _ptr(next_front), _stream(stream)), "emo_front_counts")
    return next_front


def emo_nsga3_select_ranked(F: torch.Tensor, R: torch.Tensor, n_keep: int, seed: int, generation: int,
                            rank: torch.Tensor, survivors: torch.Tensor | None = None, info: torch.Tensor | None = None,
                            ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Selection of a population whose ranks are given (no dominance matrix)."""
    n2, m = F.shape
    n_r = R.shape[0]
    if survivors is None:
        survivors = torch.empty(n_keep, dtype=torch.int32, device=F.device)
    nbytes = emo_workspace_size(EMO_OP_SELECT_RANKED, n2, m, n_r)
    if nbytes == 0:
        raise EmoError(1, "emo_workspace_size")
    ws = _ws(nbytes, ws, F.device)
    _check(lib().emo_nsga3_select_ranked(_ptr(F), n2, m, _ptr(R), n_r, n_keep, seed & 0xFFFFFFFFFFFFFFFF,
                                         generation & 0xFFFFFFFFFFFFFFFF, _ptr(rank), _ptr(survivors), _ptr(info),
                                         _ptr(ws), nbytes, _stream(stream)), "emo_nsga3_select_ranked")
    return survivors


def emo_nsga3_associate_range(F: torch.Tensor, R: torch.Tensor, n_keep: int, rank: torch.Tensor, col_lo: int,
                              col_hi: int, info: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                              stream=None):
    """Association of the points [col_lo, col_hi) of a population with given
    ranks (one GPU of a split population): (pi, dist, rho) of that range."""
    n2, m = F.shape
    n_r = R.shape[0]
    k = col_hi - col_lo
    pi = torch.empty(max(k, 0), dtype=torch.int32, device=F.device)
    dist = torch.empty(max(k, 0), dtype=torch.float64, device=F.device)
    rho = torch.empty(n_r, dtype=torch.int32, device=F.device)
    nbytes = emo_workspace_size(EMO_OP_SELECT_RANKED, n2, m, n_r)
    if nbytes == 0:
        raise EmoError(1, "emo_workspace_size")
    ws = _ws(nbytes, ws, F.device)
    _check(lib().emo_nsga3_associate_range(_ptr(F), n2, m, _ptr(R), n_r, n_keep, _ptr(rank), col_lo, col_hi,
                                           _ptr(pi) if k > 0 else None, _ptr(dist) if k > 0 else None, _ptr(rho),
                                           _ptr(info), _ptr(ws), nbytes, _stream(stream)),
           "emo_nsga3_associate_range")
    return pi, dist, rho


def emo_nsga3_niche_given(n2: int, n_r: int, n_keep: int, seed: int, generation: int, rank: torch.Tensor,
                          rho: torch.Tensor, last: torch.Tensor, last_pi: torch.Tensor, last_dist: torch.Tensor,
                          niche_mode: int = 0, survivors: torch.Tensor | None = None,
                          info: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    """Niching and survivors from the association gathered over the GPUs of a
    split population (niche counts of P, front l with references and
    distances, ascending)."""
    if survivors is None:
        survivors = torch.empty(n_keep, dtype=torch.int32, device=rank.device)
    nbytes = emo_workspace_size(EMO_OP_SELECT_RANKED, n2, 2, n_r)
    if nbytes == 0:
        raise EmoError(1, "emo_workspace_size")
    ws = _ws(nbytes, ws, rank.device)
    _check(lib().emo_nsga3_niche_given(n2, n_r, n_keep, seed & 0xFFFFFFFFFFFFFFFF, generation & 0xFFFFFFFFFFFFFFFF,
                                       niche_mode, _ptr(rank), _ptr(rho), _ptr(last), _ptr(last_pi),
                                       _ptr(last_dist), last.numel(), _ptr(survivors), _ptr(info), _ptr(ws), nbytes,
                                       _stream(stream)), "emo_nsga3_niche_given")
    return survivors


def emo_nd_rank(F: torch.Tensor, n_keep: int = 0, rank: torch.Tensor | None = None,
                last_rank: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    n2, m = F.shape
    if rank is None:
        rank = torch.empty(n2, dtype=torch.int32, device=F.device)
    if last_rank is None:
        last_rank = torch.empty(1, dtype=torch.int32, device=F.device)
    nbytes = emo_workspace_size(EMO_OP_ND_RANK, n2, m, 0)
    if nbytes == 0:
        raise EmoError(1, "emo_workspace_size")
    ws = _ws(nbytes, ws, F.device)
    _check(lib().emo_nd_rank(_ptr(F), n2, m, n_keep, _ptr(rank), _ptr(last_rank), _ptr(ws), nbytes,
                             _stream(stream)), "emo_nd_rank")
    return rank, last_rank


def emo_nsga3_select(F: torch.Tensor, R: torch.Tensor, n_keep: int, seed: int = 0, generation: int = 0,
                     survivors: torch.Tensor | None = None, info: torch.Tensor | None = None,
                     ws: torch.Tensor | None = None, debug: dict | None = None, stream=None,
                     niche_mode: int = 0):
    """Survivor indices (ascending, int32 ``[n_keep]``) on the device.

    ``info`` is an int32 tensor of 8 elements (``SelectInfo`` layout);
    ``debug`` maps names of ``SelectDebug`` fields to device tensors;
    ``niche_mode`` is EMO_NICHE_EXACT (0) or EMO_NICHE_ONESHOT (1), which
    goes through emo_nsga3_select_ex.
    """
    n2, m = F.shape
    n_r = R.shape[0]
    if survivors is None:
        survivors = torch.empty(n_keep, dtype=torch.int32, device=F.device)
    nbytes = emo_workspace_size(EMO_OP_NSGA3_SELECT, n2, m, n_r)
    if nbytes == 0:
        raise EmoError(1, "emo_workspace_size")
    ws = _ws(nbytes, ws, F.device)
    seed &= 0xFFFFFFFFFFFFFFFF
    generation &= 0xFFFFFFFFFFFFFFFF
    if niche_mode != EMO_NICHE_EXACT:
        dbg = SelectDebug()
        for k, t in (debug or {}).items():
            setattr(dbg, k, _ptr(t))
        rc = lib().emo_nsga3_select_ex(_ptr(F), n2, m, _ptr(R), n_r, n_keep, seed, generation, int(niche_mode),
                                       _ptr(survivors), _ptr(info), ctypes.byref(dbg) if debug else None,
                                       _ptr(ws), nbytes, _stream(stream))
    elif debug:
        dbg = SelectDebug()
        for k, t in debug.items():
            setattr(dbg, k, _ptr(t))
        rc = lib().emo_nsga3_select_debug(_ptr(F), n2, m, _ptr(R), n_r, n_keep, seed, generation,
                                          _ptr(survivors), _ptr(info), ctypes.byref(dbg), _ptr(ws), nbytes,
                                          _stream(stream))
    else:
        rc = lib().emo_nsga3_select(_ptr(F), n2, m, _ptr(R), n_r, n_keep, seed, generation, _ptr(survivors),
                                    _ptr(info), _ptr(ws), nbytes, _stream(stream))
    _check(rc, "emo_nsga3_select")
    return survivors


def emo_hype_select(F: torch.Tensor, v_ref: torch.Tensor, U: torch.Tensor, n_keep: int,
                    survivors: torch.Tensor | None = None, info: torch.Tensor | None = None,
                    hv: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    """TensorHypE selection: survivor indices (ascending, int32 ``[n_keep]``).
    ``U`` holds the ``[s, m]`` uniform numbers of the Monte Carlo samples;
    ``hv`` (float64 ``[n2]``, optional) receives the contributions of front l."""
    n2, m = F.shape
    ns = U.shape[0]
    if survivors is None:
        survivors = torch.empty(n_keep, dtype=torch.int32, device=F.device)
    nbytes = emo_workspace_size(EMO_OP_HYPE_SELECT, n2, m, ns)
    if nbytes == 0:
        raise EmoError(1, "emo_workspace_size")
    ws = _ws(nbytes, ws, F.device)
    _check(lib().emo_hype_select(_ptr(F), n2, m, _ptr(v_ref), _ptr(U), ns, n_keep, _ptr(survivors), _ptr(info),
                                 _ptr(hv), _ptr(ws), nbytes, _stream(stream)), "emo_hype_select")
    return survivors


def emo_moead_select(X: torch.Tensor, F1: torch.Tensor, O: torch.Tensor, F2: torch.Tensor, z: torch.Tensor,
                     W: torch.Tensor, I_nb: torch.Tensor, theta: float = 5.0, X_next: torch.Tensor | None = None,
                     F_next: torch.Tensor | None = None, winner: torch.Tensor | None = None,
                     status: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    """TensorMOEA/D selection (Algorithm S.8). ``z`` (float32 ``[m]``) is
    updated in place to z_min. Returns X_next, F_next, winner (int32 ``[n]``,
    -1 = kept) and the device status word (int32 ``[1]``)."""
    n, d = X.shape
    m = F1.shape[1]
    T = I_nb.shape[1]
    dev = X.device
    X_next = torch.empty_like(X) if X_next is None else X_next
    F_next = torch.empty_like(F1) if F_next is None else F_next
    winner = torch.empty(n, dtype=torch.int32, device=dev) if winner is None else winner
    status = torch.empty(1, dtype=torch.int32, device=dev) if status is None else status
    nbytes = emo_workspace_size(EMO_OP_MOEAD_SELECT, n, m, T)
    if nbytes == 0:
        raise EmoError(1, "emo_workspace_size")
    ws = _ws(nbytes, ws, dev)
    _check(lib().emo_moead_select(_ptr(X), _ptr(F1), _ptr(O), _ptr(F2), n, d, m, _ptr(z), _ptr(W), _ptr(I_nb), T,
                                  float(theta), _ptr(X_next), _ptr(F_next), _ptr(winner), _ptr(status), _ptr(ws),
                                  nbytes, _stream(stream)), "emo_moead_select")
    return X_next, F_next, winner, status


def emo_variation(X: torch.Tensor, n_off: int, seed: int, generation: int, eta_c: float = 20.0,
                  eta_m: float = 20.0, p_c: float = 1.0, p_m: float | None = None, lo: torch.Tensor | None = None,
                  hi: torch.Tensor | None = None, X_off: torch.Tensor | None = None,
                  parents: torch.Tensor | None = None, stream=None):
    """Offspring of one generation (random mating, SBX, PM); bounds [0, 1]
    unless ``lo``/``hi`` are given; ``p_m`` defaults to 1/D."""
    n, d = X.shape
    p_m = 1.0 / d if p_m is None else p_m
    X_off = torch.empty(n_off, d, dtype=torch.float32, device=X.device) if X_off is None else X_off
    _check(lib().emo_variation(_ptr(X), n, d, _ptr(lo), _ptr(hi), n_off, seed & 0xFFFFFFFFFFFFFFFF,
                               generation & 0xFFFFFFFFFFFFFFFF, float(eta_c), float(eta_m), float(p_c), float(p_m),
                               _ptr(X_off), _ptr(parents), _stream(stream)), "emo_variation")
    return X_off


def emo_standin_objectives(X: torch.Tensor, m: int, shape: int, F: torch.Tensor | None = None, stream=None):
    """Stand-in objectives of decision vectors X (EMO_SHAPE_LINEAR / _SPHERE)."""
    n, d = X.shape
    F = torch.empty(n, m, dtype=torch.float32, device=X.device) if F is None else F
    _check(lib().emo_standin_objectives(_ptr(X), n, d, m, shape, _ptr(F), _stream(stream)),
           "emo_standin_objectives")
    return F


def emo_igd(F: torch.Tensor, Ref: torch.Tensor, out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    """IGD of population F to the front Ref (float64 scalar tensor on the device)."""
    n, m = F.shape
    out = torch.empty(1, dtype=torch.float64, device=F.device) if out is None else out
    nbytes = emo_workspace_size(EMO_OP_IGD, Ref.shape[0], m, 0)
    ws = _ws(nbytes, ws, F.device)
    _check(lib().emo_igd(_ptr(F), n, m, _ptr(Ref), Ref.shape[0], _ptr(out), _ptr(ws), nbytes, _stream(stream)),
           "emo_igd")
    return out


def emo_generation_workspace_size(n: int, d: int, m: int, n_r: int) -> int:
    return int(lib().emo_generation_workspace_size(n, d, m, n_r))


def emo_nsga3_generation(X: torch.Tensor, F: torch.Tensor, R: torch.Tensor, shape: int, seed: int, generation: int,
                         eta_c: float = 20.0, eta_m: float = 20.0, p_c: float = 1.0, p_m: float | None = None,
                         niche_mode: int = EMO_NICHE_EXACT, info: torch.Tensor | None = None,
                         ws: torch.Tensor | None = None, stream=None):
    """One NSGA-III generation in place on (X [N, d], F [N, m])."""
    n, d = X.shape
    m = F.shape[1]
    p_m = 1.0 / d if p_m is None else p_m
    nbytes = emo_generation_workspace_size(n, d, m, R.shape[0])
    if nbytes == 0:
        raise EmoError(1, "emo_generation_workspace_size")
    ws = _ws(nbytes, ws, X.device)
    _check(lib().emo_nsga3_generation(_ptr(X), _ptr(F), n, d, m, _ptr(R), R.shape[0], shape,
                                      seed & 0xFFFFFFFFFFFFFFFF, generation & 0xFFFFFFFFFFFFFFFF, float(eta_c),
                                      float(eta_m), float(p_c), float(p_m), niche_mode, _ptr(info), _ptr(ws),
                                      nbytes, _stream(stream)), "emo_nsga3_generation")
    return X, F


def _problems(problems) -> ctypes.Array:
    arr = (Problem * len(problems))()
    for i, p in enumerate(problems):
        arr[i].F = _ptr(p["F"])
        arr[i].R = _ptr(p["R"])
        arr[i].survivors = _ptr(p["survivors"])
        arr[i].info = _ptr(p.get("info"))
        arr[i].n2 = p["F"].shape[0]
        arr[i].m = p["F"].shape[1]
        arr[i].n_r = p["R"].shape[0]
        arr[i].n_keep = p["n_keep"]
        arr[i].seed = p.get("seed", 0) & 0xFFFFFFFFFFFFFFFF
        arr[i].generation = p.get("generation", 0) & 0xFFFFFFFFFFFFFFFF
        arr[i].niche_mode = int(p.get("niche_mode", EMO_NICHE_EXACT))
    return arr


def emo_batch_workspace_size(problems) -> int:
    arr = _problems(problems)
    return int(lib().emo_batch_workspace_size(arr, len(problems)))


def emo_nsga3_select_batch(problems, ws: torch.Tensor | None = None, stream=None):
    """``problems``: list of dicts with F, R, n_keep, survivors[, info, seed, generation, niche_mode]."""
    arr = _problems(problems)
    nbytes = int(lib().emo_batch_workspace_size(arr, len(problems)))
    if nbytes == 0:
        raise EmoError(1, "emo_batch_workspace_size")
    ws = _ws(nbytes, ws, problems[0]["F"].device)
    _check(lib().emo_nsga3_select_batch(arr, len(problems), _ptr(ws), nbytes, _stream(stream)),
           "emo_nsga3_select_batch")
    return ws


def emo_workspace_status(ws: torch.Tensor, stream=None) -> int:
    out = ctypes.c_int32(0)
    _check(lib().emo_workspace_status(_ptr(ws), _stream(stream), ctypes.byref(out)), "emo_workspace_status")
    return int(out.value)


def emo_launch_shape(m: int, n2: int) -> dict:
    """Launch shapes a selection of (n2, m) uses now on the current device."""
    out = (ctypes.c_int32 * 5)()
    _check(lib().emo_launch_shape(int(m), int(n2), ctypes.addressof(out)), "emo_launch_shape")
    return {"assoc_blocks_per_sm": out[0], "dom_rowblocks_per_item": out[1], "peel_ctas": out[2],
            "other_coop_ctas": out[3], "peel_wavefront": out[4]}


def emo_autotune_reset() -> None:
    """Forget the tuned shapes of this process."""
    lib().emo_autotune_reset()


def emo_autotune(m: int, n2: int, cache_path: str | None = None) -> None:
    """Offline tuning of the launch shapes for (m, about n2) on the current device."""
    _check(lib().emo_autotune(int(m), int(n2), cache_path.encode() if cache_path else None), "emo_autotune")


def emo_get_last_device_status(stream=None) -> int:
    """The first device-detected status since the last read (cleared by the read)."""
    out = ctypes.c_int32(0)
    _check(lib().emo_get_last_device_status(_stream(stream), ctypes.byref(out)), "emo_get_last_device_status")
    return int(out.value)


def emo_set_spin_budget(cycles: int) -> None:
    lib().emo_set_spin_budget(int(cycles))


def emo_status_string(status: int) -> str:
    return lib().emo_status_string(int(status)).decode()


def emo_version() -> int:
    return int(lib().emo_version())


def emo_set_stage_timing(enable: bool) -> None:
    lib().emo_set_stage_timing(1 if enable else 0)


def emo_stage_times() -> list[tuple[str, float]]:
    """(stage, ms) of the last multi-stage call on this host thread."""
    ms = (ctypes.c_float * 16)()
    names = (ctypes.c_char_p * 16)()
    n = lib().emo_stage_times(ms, names, 16)
    if n < 0:
        raise EmoError(4, "emo_stage_times")
    return [(names[i].decode(), float(ms[i])) for i in range(n)]


def emo_nsga3_select_noalloc(F: torch.Tensor, R: torch.Tensor, n_keep: int, seed: int = 0, generation: int = 0,
                             survivors: torch.Tensor | None = None, info: torch.Tensor | None = None,
                             stream=None):
    """Selection in the library's built-in device scratch: for callers that
    cannot allocate a workspace. ``survivors`` (and ``info``) may be given
    pre-allocated; with them the call allocates no device memory at all."""
    n2, m = F.shape
    if survivors is None:
        survivors = torch.empty(n_keep, dtype=torch.int32, device=F.device)
    _check(lib().emo_nsga3_select_noalloc(_ptr(F), n2, m, _ptr(R), R.shape[0], n_keep,
                                          seed & 0xFFFFFFFFFFFFFFFF, generation & 0xFFFFFFFFFFFFFFFF,
                                          _ptr(survivors), _ptr(info), _stream(stream)),
           "emo_nsga3_select_noalloc")
    return survivors


def emo_device_report() -> str:
    buf = ctypes.create_string_buffer(4096)
    lib().emo_device_report(buf, 4096)
    return buf.value.decode()
