"""Run a few selections on one synthetic population (for profilers).

python -m paper_2503_20286_gb300.profile_run --n2 100000 --m 3 --calls 2

Prints the per-stage device times of the last call (CUDA events recorded by
the library between its stages). Nothing else is allocated besides the
inputs, outputs and the workspace, which keeps profiler replays small.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import _binding as emo
from . import build as emo_build
from . import workloads as wl


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n2", type=int, default=100_000)
    ap.add_argument("--m", type=int, default=3)
    ap.add_argument("--shape", default="sphere")
    ap.add_argument("--calls", type=int, default=2)
    ap.add_argument("--op", choices=["select", "rank", "dominance"], default="select")
    args = ap.parse_args()
    emo_build.build()
    dev = torch.device("cuda")
    F = wl.population(args.n2, args.m, args.m + 9, args.shape, wl.BASE_SEED + 4)
    R = wl.das_dennis(wl.h_for_count(args.n2 // 2, args.m), args.m)
    Ft, Rt = torch.from_numpy(F).to(dev), torch.from_numpy(R).to(dev)
    n_keep = args.n2 // 2
    emo.emo_set_stage_timing(True)
    if args.op == "select":
        ws = torch.empty(emo.emo_workspace_size(emo.EMO_OP_NSGA3_SELECT, args.n2, args.m, R.shape[0]),
                         dtype=torch.uint8, device=dev)
        surv = torch.empty(n_keep, dtype=torch.int32, device=dev)
        for c in range(args.calls):
            emo.emo_nsga3_select(Ft, Rt, n_keep, 1, c, survivors=surv, ws=ws)
    elif args.op == "rank":
        ws = torch.empty(emo.emo_workspace_size(emo.EMO_OP_ND_RANK, args.n2, args.m, 0), dtype=torch.uint8,
                         device=dev)
        for c in range(args.calls):
            emo.emo_nd_rank(Ft, 0, ws=ws)
    else:
        for c in range(args.calls):
            emo.emo_dominance(Ft)
    torch.cuda.synchronize()
    print(json.dumps({"n2": args.n2, "m": args.m, "n_r": int(R.shape[0]), "op": args.op,
                      "stage_ms": dict(emo.emo_stage_times())}))


if __name__ == "__main__":
    main()
