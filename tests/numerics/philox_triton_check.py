"""Philox4x32-10 through Triton's own implementation, run by Triton's CPU
interpreter: reads counter words (n x 4) and key words (n x 2) as uint32
from the .npy files named on the command line and writes the generator's
output words (n x 4) to the third.  Test infrastructure only: an
implementation of the generator that shares nothing with the oracle, used
to pin the oracle's bit pattern on a machine without a GPU.
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402
from triton.language.random import philox_impl  # noqa: E402


@triton.jit
def _philox_rows(C, K, O, n, BLOCK: tl.constexpr):
    i = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    m = i < n
    c0 = tl.load(C + 4 * i + 0, mask=m)
    c1 = tl.load(C + 4 * i + 1, mask=m)
    c2 = tl.load(C + 4 * i + 2, mask=m)
    c3 = tl.load(C + 4 * i + 3, mask=m)
    k0 = tl.load(K + 2 * i + 0, mask=m)
    k1 = tl.load(K + 2 * i + 1, mask=m)
    o0, o1, o2, o3 = philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(O + 4 * i + 0, o0, mask=m)
    tl.store(O + 4 * i + 1, o1, mask=m)
    tl.store(O + 4 * i + 2, o2, mask=m)
    tl.store(O + 4 * i + 3, o3, mask=m)


def main(ctr_path, key_path, out_path):
    ctr = np.ascontiguousarray(np.load(ctr_path).astype(np.uint32))
    key = np.ascontiguousarray(np.load(key_path).astype(np.uint32))
    n = ctr.shape[0]
    as_u32 = lambda a: torch.from_numpy(a.view(np.int32).copy()).view(torch.uint32)
    out = torch.zeros((n, 4), dtype=torch.uint32)
    block = 256
    _philox_rows[((n + block - 1) // block,)](as_u32(ctr), as_u32(key), out, n, BLOCK=block)
    np.save(out_path, out.view(torch.int32).numpy().view(np.uint32))


if __name__ == "__main__":
    main(*sys.argv[1:4])
