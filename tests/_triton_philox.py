"""Triton's library Philox-4x32-10, run by its CPU interpreter (test helper)."""
import os

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402
from triton.language.random import philox_impl  # noqa: E402


@triton.jit
def _kern(c_ptr, k_ptr, o_ptr, n: tl.constexpr):
    i = tl.arange(0, n)
    o0, o1, o2, o3 = philox_impl(tl.load(c_ptr + 4 * i), tl.load(c_ptr + 4 * i + 1),
                                 tl.load(c_ptr + 4 * i + 2), tl.load(c_ptr + 4 * i + 3),
                                 tl.load(k_ptr + 2 * i), tl.load(k_ptr + 2 * i + 1))
    tl.store(o_ptr + 4 * i, o0)
    tl.store(o_ptr + 4 * i + 1, o1)
    tl.store(o_ptr + 4 * i + 2, o2)
    tl.store(o_ptr + 4 * i + 3, o3)


def philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """ctr [n,4] uint32, key [n,2] uint32 -> [n,4] uint32 (n a power of two)."""
    n = ctr.shape[0]
    out = torch.zeros(4 * n, dtype=torch.uint32)
    _kern[(1,)](torch.from_numpy(np.ascontiguousarray(ctr, np.uint32).reshape(-1).copy()),
                torch.from_numpy(np.ascontiguousarray(key, np.uint32).reshape(-1).copy()), out, n)
    return out.numpy().reshape(n, 4)
