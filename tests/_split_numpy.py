"""Test-only arithmetic for the split exchange on CPU ranks: the same three
steps as the library's kernels (column share of the dominance matrix and
its counts, one peeling step, selection), written with the oracle and
numpy. Lets gloo ranks on the CPU run paper_2503_20286_gb300.split."""
import numpy as np
import torch

import oracle


class NumpyOps:
    n2 = 0

    def dominance_cols(self, F, lo, hi):
        D = oracle.dominance_bits(F.numpy())
        bits = np.unpackbits(D.view(np.uint8), bitorder="little", axis=1)[:, lo:hi]
        return torch.from_numpy(bits.astype(np.int32)), torch.from_numpy(bits.sum(axis=0).astype(np.int32))

    def front_counts(self, D, ncols, members, counts):
        d = D[members.long()].sum(dim=0).to(torch.int32)
        counts -= d
        return ((d > 0) & (counts == 0)).to(torch.uint8)

    def select_ranked(self, F, R, n_keep, seed, generation, ranks):
        surv, _ = oracle.nsga3_select(F.numpy(), R.numpy(), n_keep, seed, generation, trace=False)
        return torch.from_numpy(surv), None
