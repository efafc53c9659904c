"""Write the oracle fixture of the 2N = 400,000 selection workload
(M = 3, sphere-shaped front, 200,028 Das-Dennis directions, keep 200,000).

Calls only the oracle (its all-core build, whose results equal the
single-threaded build's) and the seeded workload generators; no value comes
from the CUDA path. The full arrays are too large to store, so the fixture
keeps what is small exactly and the rest as SHA-256 digests plus a sample:

* the SHA-256 of the float32 inputs F and R (the test checks that it feeds
  the same arrays);
* the survivors as a bit mask over the 2N points (exact);
* the ranks of S = {rank <= l} as uint8 (255 outside S; exact);
* z, the extreme points, the intercepts a (FP64 bits), l, |P|, |L|, the
  fallback flag, the niching levels and the oracle's near-tie count;
* SHA-256 digests of pi and of the FP64 distances over S (index order), of
  rho, each also in 64 chunks of S so that a mismatch can be located;
* every 61st point of S with its pi and distance, stored exactly.

Run: python tests/golden/make_config4_golden.py  (about 20 GB of memory for
Deb's domination sets; minutes on a few cores).
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2503_20286_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(HERE, "config4_oracle.npz")
CHUNKS = 64
SAMPLE_STEP = 61


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def chunk_digests(a: np.ndarray) -> np.ndarray:
    return np.array([sha(c) for c in np.array_split(a, CHUNKS)])


def main():
    p = wl.config(4)
    t0 = time.time()
    surv, t = oracle.nsga3_select(p.F, p.R, p.n_keep, p.seed, p.generation, parallel=True)
    secs = time.time() - t0
    n2 = p.n2
    l = t["last_rank"]
    S = np.flatnonzero(t["rank"] <= l)
    rank_u8 = np.full(n2, 255, np.uint8)
    rank_u8[S] = t["rank"][S].astype(np.uint8)
    mask = np.zeros(n2, bool)
    mask[surv] = True
    pi_S = t["pi"][S].astype("<i4")
    dist_S = t["dist"][S].astype("<f8")
    sample = S[::SAMPLE_STEP]
    np.savez_compressed(
        OUT,
        workload=np.array(p.name), n2=n2, m=p.m, n_r=p.n_r, n_keep=p.n_keep, seed=np.uint64(p.seed),
        generation=p.generation,
        F_sha256=np.array(sha(p.F.astype("<f4"))), R_sha256=np.array(sha(p.R.astype("<f4"))),
        survivor_mask=np.packbits(mask, bitorder="little"),
        rank_u8=rank_u8,
        z=t["z"], extreme=t["extreme"], a=t["a"],
        last_rank=l, n_before=t["n_before"], n_last=t["n_last"], fallback=t["fallback"],
        n_levels=t["n_levels"], near_ties=t["near_ties"],
        pi_sha256=np.array(sha(pi_S)), dist_sha256=np.array(sha(dist_S)),
        rho_sha256=np.array(sha(t["rho"].astype("<i4"))),
        pi_chunk_sha256=chunk_digests(pi_S), dist_chunk_sha256=chunk_digests(dist_S),
        sample_index=sample.astype(np.int32), sample_pi=t["pi"][sample].astype(np.int32),
        sample_dist=t["dist"][sample],
        oracle_seconds=secs, oracle_threads=oracle.threads())
    print(f"wrote {OUT}: l={l} |P|={t['n_before']} |L|={t['n_last']} near_ties={t['near_ties']} "
          f"levels={t['n_levels']} in {secs:.0f} s on {oracle.threads()} threads")


if __name__ == "__main__":
    main()
