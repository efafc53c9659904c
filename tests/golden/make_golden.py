"""Write the oracle regression fixtures under tests/golden/.

Calls only the oracle (oracle/) and the seeded workload generators; no
value comes from the CUDA path. Run: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2503_20286_gb300 import workloads as wl  # noqa: E402


def main():
    p = wl.config(0)
    surv, t = oracle.nsga3_select(p.F, p.R, p.n_keep, p.seed, p.generation)
    with open(os.path.join(HERE, "config0_oracle.txt"), "w") as fh:
        fh.write("# NSGA-III environmental selection (Algorithm S.1 with S.5), oracle output\n")
        fh.write(f"# workload: {p.name}, n_keep={p.n_keep}, seed={p.seed}, generation={p.generation}\n")
        fh.write(f"last_rank: {t['last_rank']}\n")
        fh.write(f"n_before: {t['n_before']}\n")
        fh.write(f"n_last: {t['n_last']}\n")
        fh.write(f"fallback: {t['fallback']}\n")
        fh.write("rank: " + " ".join(map(str, t["rank"].tolist())) + "\n")
        fh.write("survivors: " + " ".join(map(str, surv.tolist())) + "\n")


if __name__ == "__main__":
    main()
