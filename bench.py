#!/usr/bin/env python3
"""Throughput of NSGA-III environmental selection on GB300.

Workload: one merged population of 2N = 400,000 points with M = 3 float32
objectives (sphere-front stand-in, D = 12 decision variables) and 200,028
Das-Dennis directions (H = 631), keeping N = 200,000. One step is one full
``emo_nsga3_select`` call (ordering, dominance, peeling, normalisation,
association, niching, survivors) with the inputs resident in HBM.

Prints one JSON line. ``value`` is dominance pairs (2N)^2 per second through
whole selection steps, summed over ranks (weak scaling: every rank selects
its own population, no collective on the data path). ``--impl reference``
times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dominance pairs/s and selections/s at 2N=400k; batched vs plain; % of roofline"
UNIT = "pairs/s"
N2, M, H, D_VARS = 400_000, 3, 631, 12
SAMPLE_N2, SAMPLE_H = 40_000, 199        # oracle sample: first 40,000 points, 20,100 directions (about 10 s)
FLUSH_BYTES = 512 << 20                   # > 129 MB L2
KERNELS_PER_STEP = 12                     # launches of one single-population selection


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n2", type=int, default=N2, help="population size (default: the 400k workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-population batched-vs-plain timing")
    ap.add_argument("--no-parity", action="store_true",
                    help="skip the per-workload oracle timing and error report of the CPU-baseline leg")
    ap.add_argument("--profile-op", choices=["select", "rank", "dominance", "hype", "moead", "generation"],
                    help="profiling mode: run --profile-calls calls of one operation on the sphere-front "
                         "stand-in of --n2 points (M = --profile-m) and print its stage times; nothing else runs")
    ap.add_argument("--profile-m", type=int, default=M)
    ap.add_argument("--profile-calls", type=int, default=2)
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return {"hbm_gbs": p.get("hbm_gbs", 6800.0), "sm_max_mhz": p.get("sm_max_mhz", 2070.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def workload(n2: int, seed_offset: int = 0):
    from paper_2503_20286_gb300 import workloads as wl
    seed = wl.BASE_SEED + 4 + seed_offset
    F = wl.population(n2, M, D_VARS, "sphere", seed)
    h = H if n2 == N2 else wl.h_for_count(n2 // 2, M)
    R = wl.das_dennis(h, M)
    return F, R, n2 // 2, seed


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic of k_dom_pref<3> per byte of stored tiles, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum of one launch at
# 2N=100,000, M=3: 19.00 MB read + 574.31 MB written for 635.79 MB of tiles).
# The kernel's reads (prefix sets, bucket index, keys) and writes (tiles) grow
# with the tiles it writes, so the bench scales it by the timed workload's
# tile bytes. It is reported only while the kernel sources are the ones it
# was measured on.
DOM_TRAFFIC_PER_TILE_BYTE = (18_997_504 + 574_313_984) / 635_785_216
DOM_TRAFFIC_SOURCES_SHA1 = "2fef57b62605552946187e6fbebff2dd5eb9c084"
DOM_SOURCES = ("k_dominance.cu", "emo_kernels.cuh", "emo_internal.cuh")


FP64_NOMINAL_TFLOPS = 1.25


def dom_sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in DOM_SOURCES:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2503_20286_gb300", "csrc", f),
                  "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def peel_read_bytes(emo, torch, Ft, F, n_keep: int) -> int:
    """Bytes the peel must read: every row of the fronts peeled before the last
    one (rank < l) is read once, 128 bytes per column block at or right of
    the row's block in lexicographic order (ranks from emo_nd_rank)."""
    rank, last = emo.emo_nd_rank(Ft, n_keep)
    torch.cuda.synchronize()
    r = rank.cpu().numpy()
    l = int(last.cpu().numpy().reshape(-1)[0])
    order = np.lexsort(tuple(F[:, k] for k in range(F.shape[1] - 1, -1, -1)))
    pos = np.empty(F.shape[0], dtype=np.int64)
    pos[order] = np.arange(F.shape[0])
    ncb = -(-F.shape[0] // 1024)
    return int(128 * np.sum(ncb - pos[r < l] // 1024))


def triangle_tile_bytes(n2: int) -> int:
    """Bytes of the stored triangle of D: 4 KB tiles (rb, cb) with cb >= rb / 32."""
    nrb, ncb = -(-n2 // 32), -(-n2 // 1024)
    s, t = divmod(nrb, 32)
    return (nrb * ncb - 32 * (s * (s - 1) // 2) - t * s) * 4096


def oneshot_timing(emo, torch, Ft, Rt, n_keep, seed, ws, flush, stream, steps):
    """The same selection with the one-shot niche selection (Algorithm S.4 +
    Update-Rank), device time per call (CUDA events, L2 flushed before each)."""
    surv = torch.empty(n_keep, dtype=torch.int32, device=Ft.device)
    for g in range(2):
        emo.emo_nsga3_select(Ft, Rt, n_keep, seed, g, survivors=surv, ws=ws, niche_mode=emo.EMO_NICHE_ONESHOT)
    emo.emo_set_stage_timing(True)
    ms, niche = [], []
    for k in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        emo.emo_nsga3_select(Ft, Rt, n_keep, seed, 2 + k, survivors=surv, ws=ws, niche_mode=emo.EMO_NICHE_ONESHOT)
        b.record(stream)
        niche.append(dict(emo.emo_stage_times()).get("niche", float("nan")))
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    emo.emo_set_stage_timing(False)
    if emo.emo_workspace_status(ws) != 0:
        raise SystemExit("one-shot selection failed on the device")
    t = statistics.mean(ms)
    return {"niche_mode": "one-shot (Algorithm S.4 + Update-Rank)", "steps": steps, "ms_per_step": t,
            "selections_per_s": 1e3 / t, "niche_ms": statistics.mean(niche)}


def hype_timing(emo, torch, Ft, F, n_keep, flush, stream, steps, n_samples: int = 10_000):
    """TensorHypE selection (Algorithms S.10, S.11) of the same population
    with n_samples Monte Carlo samples: device time per call (CUDA events,
    L2 flushed before each)."""
    U = np.random.Generator(np.random.Philox(7)).random((n_samples, F.shape[1])).astype(np.float32)
    v_ref = (F.max(axis=0) * np.float32(1.1)).astype(np.float32)
    Ut, vt = torch.from_numpy(U).to(Ft.device), torch.from_numpy(v_ref).to(Ft.device)
    nbytes = emo.emo_workspace_size(emo.EMO_OP_HYPE_SELECT, F.shape[0], F.shape[1], n_samples)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=Ft.device)
    surv = torch.empty(n_keep, dtype=torch.int32, device=Ft.device)
    for _ in range(2):
        emo.emo_hype_select(Ft, vt, Ut, n_keep, survivors=surv, ws=ws)
    emo.emo_set_stage_timing(True)
    ms, hype = [], []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        emo.emo_hype_select(Ft, vt, Ut, n_keep, survivors=surv, ws=ws)
        b.record(stream)
        hype.append({k: v for k, v in emo.emo_stage_times() if k.startswith("hype")})
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    emo.emo_set_stage_timing(False)
    if emo.emo_workspace_status(ws) != 0:
        raise SystemExit("HypE selection failed on the device")
    t = statistics.mean(ms)
    parts = {k: statistics.mean(h[k] for h in hype) for k in hype[0]}
    return {"selection": "TensorHypE (Algorithms S.10, S.11)", "samples": n_samples, "steps": steps,
            "ms_per_step": t, "selections_per_s": 1e3 / t, "hype_stage_ms": sum(parts.values()),
            "hype_parts_ms": parts}


def moead_inputs(h: int, m: int, d: int, t: int, seed: int):
    """A TensorMOEA/D selection problem: Das-Dennis weights (H = h), their t
    nearest neighbours, current and offspring populations on the sphere
    stand-in front (uniform decision vectors), z = minimum of the current
    objectives."""
    from paper_2503_20286_gb300 import workloads as wl
    W = wl.das_dennis(h, m)
    n = W.shape[0]
    I_nb = wl.moead_neighbours_fast(W, t)
    X = wl.decision_vectors(n, d, seed, stream=11)
    O = wl.decision_vectors(n, d, seed, stream=12)
    F1 = wl.objectives_from_decisions(X, m, "sphere")
    F2 = wl.objectives_from_decisions(O, m, "sphere")
    z = F1.min(axis=0).astype(np.float32)
    return X, F1, O, F2, z, W, I_nb


def moead_timing(emo, torch, dev, flush, stream, steps, h: int = 631, m: int = 3, d: int = 12, t: int = 20):
    """TensorMOEA/D selection (Algorithm S.8) of C(h+m-1, m-1) subproblems
    with t neighbours: device time per call (CUDA events, L2 flushed before
    each); the ideal point is reset before every call so each call does the
    same work."""
    X, F1, O, F2, z, W, I_nb = moead_inputs(h, m, d, t, seed=0x250320286)
    n = W.shape[0]
    T = {k: torch.from_numpy(v).to(dev) for k, v in
         dict(X=X, F1=F1, O=O, F2=F2, z=z, W=W, I=I_nb).items()}
    zt = T["z"].clone()
    Xn, Fn = torch.empty_like(T["X"]), torch.empty_like(T["F1"])
    win = torch.empty(n, dtype=torch.int32, device=dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    ws = torch.empty(emo.emo_workspace_size(emo.EMO_OP_MOEAD_SELECT, n, m, t), dtype=torch.uint8, device=dev)

    def call():
        zt.copy_(T["z"])
        emo.emo_moead_select(T["X"], T["F1"], T["O"], T["F2"], zt, T["W"], T["I"], 5.0, X_next=Xn, F_next=Fn,
                             winner=win, status=st, ws=ws, stream=stream)
    for _ in range(3):
        call()
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    if int(st.item()) != 0:
        raise RuntimeError(f"TensorMOEA/D selection status {int(st.item())} on the device")
    tm = statistics.mean(ms)
    # bytes the selection must move: the taken rows of X or O and X_next, F1, F2, W, F_next, I_nb
    nbytes = 2 * n * d * 4 + 4 * n * m * 4 + n * t * 4
    # FP64 operations the decisions need, counting a division or square root as one: per
    # subproblem ||w||, w / ||w|| and its own PBI value (12 m + 6); per (offspring, neighbour)
    # pair the offspring's PBI value with those reused (8 m + 4: one division, one square root)
    flops = n * (12 * m + 6) + n * t * (8 * m + 4)
    return {"selection": "TensorMOEA/D (Algorithm S.8), PBI theta = 5", "subproblems": n, "m": m, "d": d,
            "neighbours": t, "steps": steps, "ms_per_step": tm, "selections_per_s": 1e3 / tm,
            "replaced": int((win >= 0).sum().item()), "algorithmic_bytes": nbytes, "fp64_flops": flops,
            "roofline": {"bound": "fp64", "achieved": flops / (tm / 1e3) / 1e12, "peak": FP64_NOMINAL_TFLOPS,
                         "unit": "TFLOP/s", "frac": flops / (tm / 1e3) / 1e12 / FP64_NOMINAL_TFLOPS,
                         "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak)",
                         "hbm_gbs": nbytes / (tm / 1e3) / 1e9}}


def nd_rank_timing(emo, torch, dev, Ft, n_keep, flush, stream, steps):
    """Non-dominated sorting alone (emo_nd_rank): the benchmark population
    down to the last front the selection needs, and the 2N = 20,000 M = 3
    sphere population ranked completely. Device time per call (CUDA events,
    L2 flushed before each)."""
    from paper_2503_20286_gb300 import workloads as wl
    p1 = wl.config(1)
    F1 = torch.from_numpy(p1.F).to(dev)
    out = {}
    for name, F, keep in (("bench_population_to_last_front", Ft, n_keep), ("n2_20000_all_fronts", F1, 0)):
        n2, m = F.shape
        ws = torch.empty(emo.emo_workspace_size(emo.EMO_OP_ND_RANK, n2, m, 0), dtype=torch.uint8, device=dev)
        rank = torch.empty(n2, dtype=torch.int32, device=dev)
        last = torch.empty(1, dtype=torch.int32, device=dev)
        for _ in range(2):
            emo.emo_nd_rank(F, keep, rank=rank, last_rank=last, ws=ws, stream=stream)
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            emo.emo_nd_rank(F, keep, rank=rank, last_rank=last, ws=ws, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        t = statistics.mean(ms)
        out[name] = {"n2": n2, "m": m, "ms": t, "pairs_per_s": float(n2) * n2 / (t / 1e3),
                     "fronts_ranked": int(last.item()) + 1}
    return out


def batched_vs_plain(emo, torch, dev, rounds: int = 5):
    """64 uneven populations: one batched call replayed from a CUDA graph
    versus 64 plain calls on one stream (device time, CUDA events)."""
    from paper_2503_20286_gb300 import workloads as wl
    probs = wl.config(3)
    items, plain = [], []
    for p in probs:
        F, R = torch.from_numpy(p.F).to(dev), torch.from_numpy(p.R).to(dev)
        it = {"F": F, "R": R, "n_keep": p.n_keep, "seed": p.seed, "generation": p.generation,
              "survivors": torch.empty(p.n_keep, dtype=torch.int32, device=dev)}
        items.append(it)
        ws = torch.empty(emo.emo_workspace_size(emo.EMO_OP_NSGA3_SELECT, p.n2, p.m, p.n_r), dtype=torch.uint8,
                         device=dev)
        plain.append((it, ws, torch.empty(p.n_keep, dtype=torch.int32, device=dev)))
    bws = torch.empty(emo.emo_batch_workspace_size(items), dtype=torch.uint8, device=dev)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        emo.emo_nsga3_select_batch(items, ws=bws, stream=side)   # warm-up outside capture
    side.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        emo.emo_nsga3_select_batch(items, ws=bws, stream=side)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def plain_round():
        for it, ws, out in plain:
            emo.emo_nsga3_select(it["F"], it["R"], it["n_keep"], it["seed"], it["generation"], survivors=out, ws=ws)

    plain_round()
    graph.replay()
    torch.cuda.synchronize()
    ok = all(torch.equal(it["survivors"], out) for it, _, out in plain)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    for _ in range(rounds):
        graph.replay()
    e[1].record(stream)
    e[2].record(stream)
    for _ in range(rounds):
        plain_round()
    e[3].record(stream)
    torch.cuda.synchronize()
    b_ms, p_ms = e[0].elapsed_time(e[1]) / rounds, e[2].elapsed_time(e[3]) / rounds
    pairs = float(sum(p.n2 * p.n2 for p in probs))
    return {"populations": len(probs), "batched_ms": b_ms, "plain_ms": p_ms, "speedup": p_ms / b_ms,
            "batched_populations_per_s": len(probs) * 1e3 / b_ms, "batched_pairs_per_s": pairs * 1e3 / b_ms,
            "plain_populations_per_s": len(probs) * 1e3 / p_ms,
            "batched": "one emo_nsga3_select_batch call replayed from a CUDA graph",
            "plain": "64 emo_nsga3_select calls on one stream", "survivors_identical": bool(ok)}


def generation_loop(emo, torch, dev, flush, stream, gens: int = 20, n: int = N2 // 2, d: int = D_VARS):
    """The paper-scale NSGA-III run (Appendix S.I operators, Section VI):
    N = 200,000 decision vectors in [0, 1)^12 on the sphere-front stand-in,
    200,028 Das-Dennis directions (H = 631), 20 generations of random mating,
    SBX (eta 20, p 1), polynomial mutation (eta 20, p 1/D), evaluation and
    selection of 2N = 400,000 merged points, all in emo_nsga3_generation on
    the device. Per generation: device time of the whole generation and of
    its selection stages (CUDA events, L2 flushed before each); IGD of the
    population to the H = 631 sphere front before and after."""
    from paper_2503_20286_gb300 import workloads as wl
    seed = wl.BASE_SEED + 4
    R = torch.from_numpy(wl.das_dennis(H, M)).to(dev)
    front = torch.from_numpy(wl.reference_front(H, M, "sphere")).to(dev)
    X = torch.from_numpy(wl.decision_vectors(n, d, seed, stream=5)).to(dev)
    F = emo.emo_standin_objectives(X, M, emo.EMO_SHAPE_SPHERE)
    info = torch.zeros(8, dtype=torch.int32, device=dev)
    ws = torch.empty(emo.emo_generation_workspace_size(n, d, M, R.shape[0]), dtype=torch.uint8, device=dev)
    igd_ws = torch.empty(emo.emo_workspace_size(emo.EMO_OP_IGD, front.shape[0], M, 0), dtype=torch.uint8, device=dev)

    def igd():
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        v = emo.emo_igd(F, front, ws=igd_ws, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        return float(v.item()), a.elapsed_time(b)

    igd0, igd_ms = igd()
    emo.emo_set_stage_timing(True)
    gen_ms, sel_ms = [], []
    for g in range(gens):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        emo.emo_nsga3_generation(X, F, R, emo.EMO_SHAPE_SPHERE, seed, g, info=info, ws=ws, stream=stream)
        b.record(stream)
        sel_ms.append(sum(ms for _, ms in emo.emo_stage_times()))
        torch.cuda.synchronize()
        gen_ms.append(a.elapsed_time(b))
    emo.emo_set_stage_timing(False)
    if int(info[0].item()) != 0:
        raise RuntimeError(f"generation status {int(info[0].item())} on the device")
    igd1, _ = igd()
    return {"loop": "NSGA-III, 20 generations on the device (emo_nsga3_generation)", "n": n, "n2": 2 * n, "m": M,
            "d": d, "n_r": int(R.shape[0]), "sbx": {"eta": 20, "p": 1.0}, "pm": {"eta": 20, "p": 1.0 / d},
            "generations": gens, "generation_ms": gen_ms, "selection_ms": sel_ms,
            "generation_ms_mean": statistics.mean(gen_ms), "selection_ms_mean": statistics.mean(sel_ms),
            "generations_per_s": 1e3 / statistics.mean(gen_ms),
            "igd_initial": igd0, "igd_final": igd1, "igd_ms": igd_ms,
            "igd_front": f"Das-Dennis H={H} directions projected onto the unit sphere",
            "last_info": dict(zip(("status", "last_rank", "n_before", "n_last", "fallback_used", "n_recheck",
                                   "n_fronts", "n_levels"), info.cpu().tolist()))}


def dominance_call_timing(emo, torch, dev, flush, stream, steps):
    """emo_dominance (the first call of the boundary: the full matrix in the
    caller's order) at 2N = 100,000 and 400,000, M = 3: the direct
    pair-by-pair kernel and the prefix-set form (emo_dominance_ws). Bytes:
    the (2N)^2 / 8 written; device time per call (CUDA events, L2 flushed
    before each); both must give the same matrix."""
    from paper_2503_20286_gb300 import workloads as wl
    out = {}
    pk = peaks()
    for n2 in (100_000, N2):
        F = torch.from_numpy(wl.population(n2, M, D_VARS, "sphere", wl.BASE_SEED + 4)).to(dev)
        ld = (n2 + 31) // 32
        D = torch.empty((n2, ld), dtype=torch.int32, device=dev)
        c = torch.empty(n2, dtype=torch.int32, device=dev)
        ws = torch.empty(max(1, emo.emo_workspace_size(emo.EMO_OP_DOMINANCE_WS, n2, M, 0)), dtype=torch.uint8,
                         device=dev)
        res = {}
        for name, call in (("prefix_sets", lambda: emo.emo_dominance_ws(F, D=D, dom_count=c, ws=ws, stream=stream)),
                           ("direct", lambda: emo.emo_dominance(F, D=D, dom_count=c, stream=stream))):
            call()
            ms = []
            for _ in range(steps if (name == "prefix_sets" or n2 < N2) else 1):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                call()
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            t = statistics.median(ms)
            byt = n2 * ld * 4
            res[name] = {"ms": t, "GBps": byt / (t / 1e3) / 1e9, "frac_of_hbm": byt / (t / 1e3) / 1e9 / pk["hbm_gbs"]}
            if name == "prefix_sets":
                ref = (D.clone(), c.clone())
        res["identical"] = bool(torch.equal(ref[0], D) and torch.equal(ref[1], c))
        res["matrix_bytes"] = n2 * ld * 4
        out[f"n2_{n2}"] = res
        del D, ws, ref
        torch.cuda.empty_cache()
    return out


def batched_sharded(emo, torch, dev, world: int, rank: int, rounds: int = 5):
    """The 64-population batch spread over the ranks (shard_populations:
    longest first to the least-loaded rank, load (2N)^2), each rank's share
    one emo_nsga3_select_batch call replayed from a CUDA graph; no
    collective on the data path. Whole-job time = the slowest rank's."""
    import torch.distributed as dist
    from paper_2503_20286_gb300 import workloads as wl
    from paper_2503_20286_gb300.replicas import max_over_ranks, shard_populations
    probs = wl.config(3)
    mine = shard_populations([p.n2 for p in probs], world)[rank]
    items = []
    for i in mine:
        p = probs[i]
        items.append({"F": torch.from_numpy(p.F).to(dev), "R": torch.from_numpy(p.R).to(dev), "n_keep": p.n_keep,
                      "seed": p.seed, "generation": p.generation,
                      "survivors": torch.empty(p.n_keep, dtype=torch.int32, device=dev)})
    ms = 0.0
    if items:
        bws = torch.empty(emo.emo_batch_workspace_size(items), dtype=torch.uint8, device=dev)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            emo.emo_nsga3_select_batch(items, ws=bws, stream=side)
        side.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            emo.emo_nsga3_select_batch(items, ws=bws, stream=side)
        graph.replay()
        torch.cuda.synchronize()
        if emo.emo_workspace_status(bws) != 0:
            raise RuntimeError("batched selection failed on the device")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if items:
        stream = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(rounds):
            graph.replay()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / rounds
    if world > 1:
        dist.barrier()
    t = max_over_ranks(ms, dev)
    pairs = float(sum(p.n2 * p.n2 for p in probs))
    return {"populations": len(probs), "ranks": world, "populations_this_rank": len(mine), "ms": t,
            "populations_per_s": len(probs) * 1e3 / t, "pairs_per_s": pairs * 1e3 / t, "scaling": "strong",
            "split": "shard_populations (longest first, load (2N)^2), one batched graph replay per rank"}


def autotune_report(emo, torch, dev, flush, stream, steps):
    """Tuned against default launch shapes: workload 1 (2N = 20,000, M = 3:
    one selection, and non-dominated sorting of every front) and the
    64-population batch (one graph replay), timed before and after
    emo_autotune has tuned every (m, size) they contain. Tuning runs offline,
    outside every timed region; survivors must not change."""
    from paper_2503_20286_gb300 import workloads as wl
    p1 = wl.config(1)
    F1, R1 = torch.from_numpy(p1.F).to(dev), torch.from_numpy(p1.R).to(dev)
    probs = wl.config(3)
    items = [{"F": torch.from_numpy(p.F).to(dev), "R": torch.from_numpy(p.R).to(dev), "n_keep": p.n_keep,
              "seed": p.seed, "generation": p.generation,
              "survivors": torch.empty(p.n_keep, dtype=torch.int32, device=dev)} for p in probs]
    bws = torch.empty(emo.emo_batch_workspace_size(items), dtype=torch.uint8, device=dev)
    ws1 = torch.empty(emo.emo_workspace_size(emo.EMO_OP_NSGA3_SELECT, p1.n2, p1.m, p1.n_r), dtype=torch.uint8,
                      device=dev)
    wsr = torch.empty(emo.emo_workspace_size(emo.EMO_OP_ND_RANK, p1.n2, p1.m, 0), dtype=torch.uint8, device=dev)
    surv1 = torch.empty(p1.n_keep, dtype=torch.int32, device=dev)
    rank1 = torch.empty(p1.n2, dtype=torch.int32, device=dev)

    def timed(call):
        for g in range(2):
            call(g)
        ms = []
        for k in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call(2 + k)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    def measure():
        out = {"select_ms": timed(lambda g: emo.emo_nsga3_select(F1, R1, p1.n_keep, p1.seed, 0, survivors=surv1,
                                                                 ws=ws1, stream=stream)),
               "nd_rank_all_fronts_ms": timed(lambda g: emo.emo_nd_rank(F1, 0, rank=rank1, ws=wsr, stream=stream))}
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            emo.emo_nsga3_select_batch(items, ws=bws, stream=side)
        side.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            emo.emo_nsga3_select_batch(items, ws=bws, stream=side)
        torch.cuda.synchronize()
        out["batch_64_graph_ms"] = timed(lambda g: graph.replay())
        out["shape_workload_1"] = emo.emo_launch_shape(p1.m, p1.n2)
        return out, surv1.clone(), rank1.clone(), [it["survivors"].clone() for it in items]

    emo.emo_autotune_reset()
    default, s_d, r_d, b_d = measure()
    t0 = time.perf_counter()
    tuned_keys = sorted({(p1.m, p1.n2.bit_length())} | {(p.m, p.n2.bit_length()) for p in probs})
    done = set()
    for m, n2 in [(p1.m, p1.n2)] + [(p.m, p.n2) for p in probs]:
        if (m, n2.bit_length()) not in done:
            emo.emo_autotune(m, n2)
            done.add((m, n2.bit_length()))
    tune_s = time.perf_counter() - t0
    tuned, s_t, r_t, b_t = measure()
    emo.emo_autotune_reset()  # the rest of the bench runs with the default shapes
    same = bool(torch.equal(s_d, s_t) and torch.equal(r_d, r_t) and all(torch.equal(a, b) for a, b in zip(b_d, b_t)))
    return {"default": default, "tuned": tuned, "tuned_sizes": len(tuned_keys), "tune_s": tune_s,
            "speedup": {k: default[k] / tuned[k] for k in ("select_ms", "nd_rank_all_fronts_ms", "batch_64_graph_ms")},
            "survivors_and_ranks_identical": same,
            "tuner": "emo_autotune: dominance item size, peel CTAs per front, other cooperative CTAs, association "
                     "blocks per SM (coordinate search, best of three)"}


def _gpu_select_debug(emo, torch, dev, F, R, n_keep, seed, gen):
    """One selection through the C ABI with every intermediate returned."""
    n2, m = F.shape
    Ft, Rt = torch.from_numpy(F).to(dev), torch.from_numpy(R).to(dev)
    info = torch.zeros(8, dtype=torch.int32, device=dev)
    dbg = {"rank": torch.empty(n2, dtype=torch.int32, device=dev), "z": torch.empty(m, device=dev),
           "extreme": torch.empty(m, dtype=torch.int32, device=dev),
           "a": torch.empty(m, dtype=torch.float64, device=dev), "fnorm": torch.empty(n2 * m, device=dev),
           "pi": torch.empty(n2, dtype=torch.int32, device=dev),
           "dist": torch.empty(n2, dtype=torch.float64, device=dev)}
    surv = emo.emo_nsga3_select(Ft, Rt, n_keep, seed, gen, info=info, debug=dbg)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in dbg.items()}
    out["fnorm"] = out["fnorm"].reshape(n2, m)
    out["survivors"] = surv.cpu().numpy()
    out["info"] = dict(zip(("status", "last_rank", "n_before", "n_last", "fallback_used", "n_recheck", "n_fronts",
                            "n_levels"), info.cpu().tolist()))
    return out, Ft, Rt


def _gpu_select_ms(emo, torch, Ft, Rt, n_keep, seed, flush, stream, steps):
    surv = torch.empty(n_keep, dtype=torch.int32, device=Ft.device)
    nbytes = emo.emo_workspace_size(emo.EMO_OP_NSGA3_SELECT, Ft.shape[0], Ft.shape[1], Rt.shape[0])
    ws = torch.empty(nbytes, dtype=torch.uint8, device=Ft.device)
    for g in range(2):
        emo.emo_nsga3_select(Ft, Rt, n_keep, seed, g, survivors=surv, ws=ws)
    ms = []
    for k in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        emo.emo_nsga3_select(Ft, Rt, n_keep, seed, 2 + k, survivors=surv, ws=ws)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def _errors(g, S, fn64, z, a, pi, dist, rank, surv):
    """Per-output comparison of the GPU intermediates with FP64 values over S."""
    rel = np.abs(g["fnorm"][S].astype(np.float64) - fn64) / np.maximum(np.abs(fn64), 1e-300)
    rel[fn64 == 0] = np.abs(g["fnorm"][S][fn64 == 0])
    return {"survivors_equal": bool(np.array_equal(g["survivors"], surv)),
            "ranks_equal_on_S": bool(rank is None or np.array_equal(g["rank"][S], rank)),
            "z_equal": bool(np.array_equal(g["z"].astype(np.float64), z)),
            "intercepts_fp64_equal": bool(np.array_equal(g["a"], a)),
            "fnorm_fp32_max_rel_err": float(rel.max()) if rel.size else 0.0,
            "pi_mismatches": None if pi is None else int(np.sum(g["pi"][S] != pi)),
            "dist_fp64_max_abs_diff": None if dist is None else float(np.max(np.abs(g["dist"][S] - dist)))}


def cpu_baseline_leg(emo, torch, dev, flush, stream, steps, F4, R4, n_keep4, seed4, main_ms):
    """The oracle beside the GPU path: the FP64 CPU oracle timed on the host
    cores (1 thread on workloads 0 and 1, all cores on workloads 0-2; the
    2N = 400,000 workload from its committed fixture, written by the all-core
    oracle), and the GPU's outputs compared with it per output: survivors,
    ranks, z, FP64 intercepts, pi and FP64 distances exactly, normalised
    objectives as the largest float32 relative error, the oracle's near-tie
    count (two nearest lines within 1e-6 relative) and the GPU's FP64
    re-checks. GPU selections/s per workload (median of `steps`, CUDA events,
    L2 flushed before each)."""
    import hashlib
    import oracle
    from paper_2503_20286_gb300 import workloads as wl
    oracle.build()
    par = oracle.has_parallel()
    cores = oracle.threads(os.cpu_count() or 1) if par else 1
    report = {}
    for c in (0, 1, 2):
        p = wl.config(c)
        g, Ft, Rt = _gpu_select_debug(emo, torch, dev, p.F, p.R, p.n_keep, p.seed, p.generation)
        ms = _gpu_select_ms(emo, torch, Ft, Rt, p.n_keep, p.seed, flush, stream, steps)
        entry = {"workload": p.name, "gpu_ms": ms, "gpu_selections_per_s": 1e3 / ms,
                 "gpu_n_recheck": g["info"]["n_recheck"]}
        if c in (0, 1):
            t0 = time.perf_counter()
            oracle.nsga3_select(p.F, p.R, p.n_keep, p.seed, p.generation, trace=False)
            entry["oracle_1_thread_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        surv, t = oracle.nsga3_select(p.F, p.R, p.n_keep, p.seed, p.generation, parallel=par)
        entry[f"oracle_{cores}_threads_s"] = time.perf_counter() - t0
        S = np.flatnonzero(t["rank"] <= t["last_rank"])
        entry.update(_errors(g, S, t["fnorm"][S], t["z"], t["a"], t["pi"][S], t["dist"][S], t["rank"][S], surv))
        entry["oracle_near_ties"] = t["near_ties"]
        report[f"workload_{c}"] = entry
    path = os.path.join(ROOT, "tests", "golden", "config4_oracle.npz")
    if os.path.exists(path):
        gold = np.load(path)
        g, _, _ = _gpu_select_debug(emo, torch, dev, F4, R4, n_keep4, seed4, 0)
        mask = np.unpackbits(gold["survivor_mask"], count=F4.shape[0], bitorder="little").astype(bool)
        S = np.flatnonzero(gold["rank_u8"] != 255)
        fn64 = (F4[S].astype(np.float64) - gold["z"]) / gold["a"]
        entry = {"workload": "2N=400000 M=3 sphere H=631 (the timed population)", "gpu_ms": main_ms,
                 "gpu_selections_per_s": 1e3 / main_ms, "gpu_n_recheck": g["info"]["n_recheck"],
                 "oracle_fixture": "tests/golden/config4_oracle.npz",
                 f"oracle_{int(gold['oracle_threads'])}_threads_s_when_written": float(gold["oracle_seconds"])}
        entry.update(_errors(g, S, fn64, gold["z"], gold["a"], None, None,
                             gold["rank_u8"][S].astype(np.int32), np.flatnonzero(mask)))
        sha = lambda a: hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()  # noqa: E731
        entry["pi_equal_sha256"] = sha(g["pi"][S].astype("<i4")) == str(gold["pi_sha256"])
        entry["dist_fp64_equal_sha256"] = sha(g["dist"][S].astype("<f8")) == str(gold["dist_sha256"])
        entry["oracle_near_ties"] = int(gold["near_ties"])
        report["workload_4"] = entry
    return report, cores


def oracle_time(F, R, n_keep, seed, sample_n2: int):
    """FP64 CPU oracle on the first `sample_n2` points (same distribution)."""
    import oracle
    from paper_2503_20286_gb300 import workloads as wl
    oracle.build()
    Fs = np.ascontiguousarray(F[:sample_n2])
    Rs = wl.das_dennis(SAMPLE_H, M) if sample_n2 == SAMPLE_N2 else wl.das_dennis(
        wl.h_for_count(sample_n2 // 2, M), M)
    t0 = time.perf_counter()
    oracle.nsga3_select(Fs, Rs, sample_n2 // 2, seed, 0, trace=False)
    dt = time.perf_counter() - t0
    return dt, Rs.shape[0]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    F, R, n_keep, seed = workload(args.n2)
    ts = []
    for i in range(args.warmup + args.steps):
        dt, nr_s = oracle_time(F, R, n_keep, seed, SAMPLE_N2)
        if i >= args.warmup:
            ts.append(dt)
    t = statistics.mean(ts)
    value = SAMPLE_N2 ** 2 / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"NSGA-III selection, sample 2N={SAMPLE_N2} of the 2N={args.n2} M={M} "
                                   f"sphere population, {nr_s} directions", "n2": SAMPLE_N2, "m": M},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {SAMPLE_N2} points of the workload, {nr_s} Das-Dennis directions, "
                                       f"keep {SAMPLE_N2 // 2}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def profile_mode(args):
    """A few calls of one operation, for a profiler attached to this process:
    only the inputs, outputs and workspace are allocated, so that replays
    stay small; prints the stage times of the last call."""
    import torch
    from paper_2503_20286_gb300 import _binding as emo
    from paper_2503_20286_gb300 import build as emo_build
    from paper_2503_20286_gb300 import workloads as wl
    emo_build.build()
    dev = torch.device("cuda")
    n2, m, op = args.n2, args.profile_m, args.profile_op
    F = wl.population(n2, m, m + 9, "sphere", wl.BASE_SEED + 4)
    R = wl.das_dennis(H if (n2 == N2 and m == M) else wl.h_for_count(n2 // 2, m), m)
    Ft, Rt = torch.from_numpy(F).to(dev), torch.from_numpy(R).to(dev)
    emo.emo_set_stage_timing(True)
    out = {}
    if op == "select":
        ws = torch.empty(emo.emo_workspace_size(emo.EMO_OP_NSGA3_SELECT, n2, m, R.shape[0]), dtype=torch.uint8,
                         device=dev)
        surv = torch.empty(n2 // 2, dtype=torch.int32, device=dev)
        for c in range(args.profile_calls):
            emo.emo_nsga3_select(Ft, Rt, n2 // 2, 1, c, survivors=surv, ws=ws)
    elif op == "rank":
        ws = torch.empty(emo.emo_workspace_size(emo.EMO_OP_ND_RANK, n2, m, 0), dtype=torch.uint8, device=dev)
        for c in range(args.profile_calls):
            emo.emo_nd_rank(Ft, 0, ws=ws)
    elif op == "dominance":
        D = torch.empty((n2, (n2 + 31) // 32), dtype=torch.int32, device=dev)
        for c in range(args.profile_calls):
            emo.emo_dominance(Ft, D=D)
    elif op == "hype":
        U = np.random.Generator(np.random.Philox(7)).random((10_000, m)).astype(np.float32)
        v_ref = (F.max(axis=0) * np.float32(1.1)).astype(np.float32)
        Ut, vt = torch.from_numpy(U).to(dev), torch.from_numpy(v_ref).to(dev)
        ws = torch.empty(emo.emo_workspace_size(emo.EMO_OP_HYPE_SELECT, n2, m, 10_000), dtype=torch.uint8, device=dev)
        for c in range(args.profile_calls):
            emo.emo_hype_select(Ft, vt, Ut, n2 // 2, ws=ws)
    elif op == "moead":
        X, F1, O, F2, z, W, I_nb = moead_inputs(wl.h_for_count(n2 // 2, m), m, m + 9, 20, seed=0x250320286)
        T = {k: torch.from_numpy(v).to(dev) for k, v in dict(X=X, F1=F1, O=O, F2=F2, z=z, W=W, I=I_nb).items()}
        for c in range(args.profile_calls):
            emo.emo_moead_select(T["X"], T["F1"], T["O"], T["F2"], T["z"].clone(), T["W"], T["I"], 5.0)
        out["subproblems"] = int(W.shape[0])
    else:
        X = torch.from_numpy(wl.decision_vectors(n2 // 2, m + 9, wl.BASE_SEED + 4, stream=5)).to(dev)
        Fg = emo.emo_standin_objectives(X, m, emo.EMO_SHAPE_SPHERE)
        for c in range(args.profile_calls):
            emo.emo_nsga3_generation(X, Fg, Rt, emo.EMO_SHAPE_SPHERE, wl.BASE_SEED + 4, c)
    torch.cuda.synchronize()
    emo.emo_set_stage_timing(False)
    out.update({"profile_op": op, "n2": n2, "m": m, "n_r": int(R.shape[0]), "calls": args.profile_calls,
                "stage_ms": dict(emo.emo_stage_times()) if op not in ("dominance", "moead") else {}})
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_op:
        return profile_mode(args)

    import torch
    import torch.distributed as dist
    from paper_2503_20286_gb300 import build as emo_build
    from paper_2503_20286_gb300 import _binding as emo
    from paper_2503_20286_gb300.replicas import max_over_ranks

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or not os.path.exists(emo_build.LIB):
        emo_build.build()
    if world > 1:
        dist.barrier()
    emo.lib()

    F, R, n_keep, seed = workload(args.n2, seed_offset=rank)
    n2, n_r = F.shape[0], R.shape[0]
    Ft = torch.from_numpy(F).to(dev)
    Rt = torch.from_numpy(R).to(dev)
    surv = torch.empty(n_keep, dtype=torch.int32, device=dev)
    info = torch.zeros(8, dtype=torch.int32, device=dev)
    ws_bytes = emo.emo_workspace_size(emo.EMO_OP_NSGA3_SELECT, n2, M, n_r)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(gen):
        emo.emo_nsga3_select(Ft, Rt, n_keep, seed, gen, survivors=surv, info=info, ws=ws)

    for w in range(args.warmup):
        step(w)
    torch.cuda.synchronize()
    st = emo.emo_workspace_status(ws)
    if st != 0:
        raise SystemExit(f"selection failed on the device: status {st}")

    emo.emo_set_stage_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_ms: dict[str, list[float]] = {}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step(args.warmup + k)
        ev[k][1].record(stream)
        for name, ms in emo.emo_stage_times():
            stage_ms.setdefault(name, []).append(ms)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    emo.emo_set_stage_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dev)  # the whole job waits for the slowest rank
    st = emo.emo_workspace_status(ws)
    if st != 0:
        raise SystemExit(f"selection failed on the device: status {st}")
    info_h = info.cpu().tolist()

    # end to end through the C ABI with host buffers (copies inside the timed region)
    F_host = torch.from_numpy(F).pin_memory()
    R_host = torch.from_numpy(R).pin_memory()
    S_host = torch.empty(n_keep, dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    e_s, e_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e_s.record(stream)
    for k in range(e2e_steps):
        Ft.copy_(F_host, non_blocking=True)
        Rt.copy_(R_host, non_blocking=True)
        step(1000 + k)
        S_host.copy_(surv, non_blocking=True)
    e_e.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e_s.elapsed_time(e_e) / e2e_steps, dev)

    pairs = float(n2) * float(n2)
    ms_per_step = total_ms / args.steps
    value = world * pairs * args.steps / (total_ms / 1e3)
    pk = peaks()
    dom_ms = statistics.mean(stage_ms.get("dominance", [float("nan")]))
    # dominance roofline: the kernel must write the triangle of D as 4 KB
    # tiles; achieved = tile bytes / kernel time against measured HBM copy BW
    tile_bytes = triangle_tile_bytes(n2)
    achieved = tile_bytes / (dom_ms / 1e3) / 1e9
    # peel roofline: the rows of the fronts before the last, read once from HBM
    peel_ms = statistics.mean(stage_ms.get("peel", [float("nan")]))
    peel_bytes = peel_read_bytes(emo, torch, Ft, F, n_keep)
    peel_roofline = {"bound": "hbm", "kernel": "k_peel", "achieved": peel_bytes / (peel_ms / 1e3) / 1e9,
                     "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": peel_bytes / (peel_ms / 1e3) / 1e9 / pk["hbm_gbs"], "algorithmic_bytes": peel_bytes}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"NSGA-III selection 2N={n2} M={M} n_r={n_r} keep {n_keep}, sphere-front "
                               f"stand-in D={D_VARS}", "n2": n2, "m": M, "n_r": n_r, "n_keep": n_keep,
                   "l2": f"flushed ({FLUSH_BYTES >> 20} MB write) before every timed step",
                   "parallelism": f"replicas x{world} (independent populations)"},
        "selections_per_s": world * 1e3 / ms_per_step,
        "dominance_pairs_per_s_kernel": pairs / (dom_ms / 1e3),
        "stage_ms": {k: statistics.mean(v) for k, v in stage_ms.items()},
        "roofline": {"bound": "hbm", "kernel": f"k_dom_pref<{M}>", "achieved": achieved,
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                     "traffic": (DOM_TRAFFIC_PER_TILE_BYTE * tile_bytes
                                 if M == 3 and dom_sources_sha1() == DOM_TRAFFIC_SOURCES_SHA1 else None),
                     "traffic_source": "ncu dram bytes at 2N=100k scaled by tile bytes",
                     "algorithmic_bytes": tile_bytes,
                     "peak_source": f"{pk['source']} HBM copy bandwidth"},
        "peel_roofline": peel_roofline,
        "e2e": {"value": world * pairs / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(F.nbytes + R.nbytes), "d2h_bytes_per_step": int(n_keep * 4)},
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "clocks": clk,
        "info": dict(zip(("status", "last_rank", "n_before", "n_last", "fallback_used", "n_recheck",
                          "n_fronts", "n_levels"), info_h)),
    }
    if rank == 0 and world == 1:
        line["oneshot"] = oneshot_timing(emo, torch, Ft, Rt, n_keep, seed, ws, flush, stream, max(3, args.steps // 2))
        del ws  # the HypE workspace replaces it
        line["hype"] = hype_timing(emo, torch, Ft, F, n_keep, flush, stream, max(3, args.steps // 2))
        try:
            line["nd_rank"] = nd_rank_timing(emo, torch, dev, Ft, n_keep, flush, stream, max(3, args.steps // 2))
        except Exception as e:  # reported in the line; the selection numbers above stand
            line["nd_rank"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            line["moead"] = moead_timing(emo, torch, dev, flush, stream, max(3, args.steps // 2))
        except Exception as e:  # reported in the line; the selection numbers above stand
            line["moead"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            line["emo_dominance"] = dominance_call_timing(emo, torch, dev, flush, stream, max(3, args.steps // 2))
        except Exception as e:  # reported in the line; the selection numbers above stand
            line["emo_dominance"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            line["generation_loop"] = generation_loop(emo, torch, dev, flush, stream)
        except Exception as e:  # reported in the line; the selection numbers above stand
            line["generation_loop"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and world == 1 and not args.no_batch:
        line["batched_vs_plain"] = batched_vs_plain(emo, torch, dev)
    if not args.no_batch:
        line["batched_sharded"] = batched_sharded(emo, torch, dev, world, rank)
    if rank == 0 and world == 1 and not args.no_batch:
        try:
            line["autotune"] = autotune_report(emo, torch, dev, flush, stream, max(5, args.steps))
        except Exception as e:  # reported in the line; the selection numbers above stand
            line["autotune"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, nr_s = oracle_time(F, R, n_keep, seed, SAMPLE_N2)
        line["cpu_baseline"] = {"value": SAMPLE_N2 ** 2 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {SAMPLE_N2} points of the workload, {nr_s} Das-Dennis "
                                          f"directions, keep {SAMPLE_N2 // 2}; {dt:.1f} s"}
        if not args.no_parity:
            rep, cores = cpu_baseline_leg(emo, torch, dev, flush, stream, max(3, args.steps), F, R, n_keep, seed,
                                          ms_per_step)
            line["cpu_baseline"]["host_cores"] = cores
            line["parity"] = rep
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
