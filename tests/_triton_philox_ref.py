"""Philox4x32-10 reference outputs from Triton's library implementation.

Run as a separate process with TRITON_INTERPRET=1 so that Triton's CPU
interpreter executes ``tl.philox`` without a GPU.  Reads a JSON object
{"seeds": [...], "ctr": [[c0, c1, c2, c3], ...]} from argv[1] and prints the
four output words per (seed, ctr) pair as JSON.  Used only to pin the oracle.
"""
import json
import os
import sys

os.environ.setdefault("TRITON_INTERPRET", "1")

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(c_ptr, out_ptr, seed, N: tl.constexpr):
    offs = tl.arange(0, N)
    c0 = tl.load(c_ptr + offs * 4 + 0)
    c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2)
    c3 = tl.load(c_ptr + offs * 4 + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + offs * 4 + 0, a)
    tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c)
    tl.store(out_ptr + offs * 4 + 3, d)


def main():
    req = json.loads(sys.argv[1])
    ctr = np.asarray(req["ctr"], dtype=np.uint64).astype(np.uint32)
    n = ctr.shape[0]
    result = []
    for seed in req["seeds"]:
        out = torch.zeros(n * 4, dtype=torch.int32)
        cin = torch.from_numpy(ctr.view(np.int32).reshape(-1).copy())
        _philox_kernel[(1,)](cin, out, int(seed), N=n)
        result.append(out.numpy().view(np.uint32).reshape(n, 4).tolist())
    print(json.dumps(result))


if __name__ == "__main__":
    main()
