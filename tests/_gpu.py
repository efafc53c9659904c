"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
the oracle on the same seeded float32 inputs."""
import numpy as np
import torch

import oracle
from paper_2503_20286_gb300 import _binding as emo

DEBUG_FIELDS = ("rank", "z", "extreme", "a", "fnorm", "pi", "dist", "rho", "picked")


def gpu_select(F, R, n_keep, seed, gen=0, debug=True, mode=0):
    dev = torch.device("cuda")
    Ft = torch.from_numpy(np.ascontiguousarray(F, np.float32)).to(dev)
    Rt = torch.from_numpy(np.ascontiguousarray(R, np.float32)).to(dev)
    n2, m = F.shape
    n_r = R.shape[0]
    info = torch.full((8,), -7, dtype=torch.int32, device=dev)
    dbg = None
    if debug:
        dbg = {"rank": torch.empty(n2, dtype=torch.int32, device=dev),
               "z": torch.empty(m, dtype=torch.float32, device=dev),
               "extreme": torch.empty(m, dtype=torch.int32, device=dev),
               "a": torch.empty(m, dtype=torch.float64, device=dev),
               "fnorm": torch.empty(n2 * m, dtype=torch.float32, device=dev),
               "pi": torch.empty(n2, dtype=torch.int32, device=dev),
               "dist": torch.empty(n2, dtype=torch.float64, device=dev),
               "rho": torch.empty(n_r, dtype=torch.int32, device=dev),
               "picked": torch.empty(n2, dtype=torch.uint8, device=dev)}
    surv = emo.emo_nsga3_select(Ft, Rt, n_keep, seed, gen, info=info, debug=dbg, niche_mode=mode)
    torch.cuda.synchronize()
    inf = dict(zip(("status", "last_rank", "n_before", "n_last", "fallback_used", "n_recheck", "n_fronts",
                    "n_levels"), info.cpu().tolist()))
    out = {k: v.cpu().numpy() for k, v in (dbg or {}).items()}
    if "fnorm" in out:
        out["fnorm"] = out["fnorm"].reshape(n2, m)
    return surv.cpu().numpy(), inf, out


def compare_select(F, R, n_keep, seed, gen=0, check_debug=True, mode=0):
    """Bit-exact survivors and intermediates against the oracle (niche mode
    0: Algorithm S.1 levels, 1: one-shot Algorithm S.4 + S.6)."""
    s_or, t = oracle.nsga3_select(F, R, n_keep, seed, gen, mode=mode)
    s_gpu, info, g = gpu_select(F, R, n_keep, seed, gen, debug=check_debug, mode=mode)
    assert info["status"] == 0, info
    assert info["last_rank"] == t["last_rank"]
    assert info["n_before"] == t["n_before"] and info["n_last"] == t["n_last"]
    if mode == 0 and t["n_last"] > n_keep - t["n_before"]:
        # niching levels of Algorithm S.1 (served one at a time or in bulk); when
        # the whole last front survives no level is run on the device
        assert info["n_levels"] == t["n_levels"], (info["n_levels"], t["n_levels"])
    if check_debug:
        l = t["last_rank"]
        S = t["rank"] <= l
        assert np.array_equal(g["rank"][S], t["rank"][S])
        assert np.all(g["rank"][~S] == emo.EMO_NOT_RANKED)
        assert np.array_equal(g["z"].astype(np.float64), t["z"])
        assert np.array_equal(g["extreme"], t["extreme"])
        assert info["fallback_used"] == t["fallback"]
        assert np.array_equal(g["a"], t["a"]), (g["a"], t["a"])
        # normalised objectives: float32 on the GPU vs float64, 1e-5 relative
        np.testing.assert_allclose(g["fnorm"][S], t["fnorm"][S], rtol=1e-5, atol=1e-30)
        assert np.all(np.isnan(g["fnorm"][~S]))
        assert np.array_equal(g["pi"], t["pi"]), np.flatnonzero(g["pi"] != t["pi"])[:10]
        assert np.array_equal(g["dist"][S], t["dist"][S])
        assert np.array_equal(g["rho"], t["rho"])
        assert np.array_equal(g["picked"], t["picked"])
    assert np.array_equal(s_gpu, s_or), (np.setdiff1d(s_gpu, s_or)[:10], np.setdiff1d(s_or, s_gpu)[:10])
    return info, t


def gpu_rank(F, n_keep=0):
    dev = torch.device("cuda")
    Ft = torch.from_numpy(np.ascontiguousarray(F, np.float32)).to(dev)
    rank, last = emo.emo_nd_rank(Ft, n_keep)
    torch.cuda.synchronize()
    return rank.cpu().numpy(), int(last.cpu().item())


def gpu_dominance(F, ld=None):
    dev = torch.device("cuda")
    Ft = torch.from_numpy(np.ascontiguousarray(F, np.float32)).to(dev)
    n2 = F.shape[0]
    D = None
    if ld is not None:
        D = torch.full((n2, ld), -1, dtype=torch.int32, device=dev)
    D, c = emo.emo_dominance(Ft, D=D)
    torch.cuda.synchronize()
    return D.cpu().numpy().view(np.uint32), c.cpu().numpy()
