"""Test-only arithmetic for the split exchange on CPU ranks: the same four
steps as the library's kernels (column share of the dominance matrix and
its counts, one peeling step, the association of a column range, the
niching from the gathered association), written with the oracle and numpy.
Lets gloo ranks on the CPU run paper_2503_20286_gb300.split; the niching
step checks that the exchange delivered the oracle's niche counts and front
l."""
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

    def associate_range(self, F, R, n_keep, ranks, lo, hi):
        """pi, dist of the range and the niche counts of its points of P,
        from the oracle's trace (normalisation and association draw nothing
        random)."""
        self._F, self._R = F.numpy(), R.numpy()
        _, t = oracle.nsga3_select(self._F, self._R, n_keep, 0, 0)
        r = ranks.numpy()
        l = t["last_rank"]
        assert np.array_equal(np.where(t["rank"] <= l, t["rank"], r), r)
        pi = t["pi"][lo:hi].astype(np.int32)
        P = np.nonzero(r[lo:hi] < l)[0]
        rho = np.bincount(pi[P], minlength=R.shape[0]).astype(np.int32)
        return torch.from_numpy(pi), torch.from_numpy(t["dist"][lo:hi].copy()), torch.from_numpy(rho)

    def niche_given(self, n2, n_r, n_keep, seed, generation, ranks, rho, last, last_pi, last_d):
        """The gathered association must be the oracle's (summed niche
        counts of P; front l ascending with its references and distances);
        the survivors are then the oracle's."""
        surv, t = oracle.nsga3_select(self._F, self._R, n_keep, seed, generation)
        L = np.nonzero(t["rank"] == t["last_rank"])[0]
        assert np.array_equal(rho.numpy(), t["rho"])
        assert np.array_equal(last.numpy(), L)
        assert np.array_equal(last_pi.numpy(), t["pi"][L])
        assert np.array_equal(last_d.numpy(), t["dist"][L])
        return torch.from_numpy(surv), None
