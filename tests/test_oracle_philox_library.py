"""Pin of the oracle's Philox4x32-10 (oracle/perturb.py) against an independent implementation.

The generator of the drawn perturbations is Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011):
ten rounds of two 32x32->64-bit products with the Weyl key schedule.  Both the oracle and the
CUDA kernel restate that definition, so a shared misreading (a multiplier, the word order of a
round, the key increment) would pass every distributional pin and every GPU parity test.  Here
the oracle is compared word for word with Triton's `tl.philox` (Triton's own library code, key =
(seed mod 2^32, seed div 2^32), 10 rounds), executed on the CPU by Triton's interpreter in a
child process, on random counters and on counters and keys at the ends of the 32-bit range.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle.perturb import philox4x32_10

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(seed, c0p, c1p, c2p, c3p, o0, o1, o2, o3, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i))
    tl.store(o0 + i, a); tl.store(o1 + i, b); tl.store(o2 + i, c); tl.store(o3 + i, d)

req = json.loads(sys.stdin.read())
res = []
for seed, ctr in req:
    ctr = np.asarray(ctr, dtype=np.uint64).astype(np.uint32)
    n = ctr.shape[0]
    cs = [torch.from_numpy(np.ascontiguousarray(ctr[:, j]).view(np.int32)) for j in range(4)]
    outs = [torch.zeros(n, dtype=torch.int32) for _ in range(4)]
    k[(1,)](seed, *cs, *outs, N=n)
    res.append(np.stack([o.numpy().view(np.uint32) for o in outs], -1).astype(np.int64).tolist())
print(json.dumps(res))
"""


def _triton_philox(cases):
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", CHILD], input=json.dumps(cases), capture_output=True, text=True,
                       env=env, timeout=600, cwd=ROOT)
    if r.returncode != 0:
        pytest.fail("triton interpreter failed:\n" + r.stderr[-2000:])
    return [np.asarray(x, dtype=np.uint64).astype(np.uint32) for x in json.loads(r.stdout.strip().splitlines()[-1])]


def test_philox_matches_triton_library():
    pytest.importorskip("triton")
    rng = np.random.default_rng(20261203)
    top = 2 ** 32 - 1
    cases = []
    # seeds: small, both key words used, the largest key words Triton's int64 seed can carry
    seeds = [0, 1, 0x0123456789ABCDEF, 0x7FFFFFFFFFFFFFFF, int(rng.integers(0, 2 ** 63))]
    for seed in seeds:
        ctr = rng.integers(0, 2 ** 32, size=(16, 4), dtype=np.uint64)
        ctr[0] = 0
        ctr[1] = top
        ctr[2] = [top, 0, top, 0]
        ctr[3] = [0, 1, 2, 3]
        cases.append((seed, ctr.tolist()))
    got = _triton_philox(cases)
    for (seed, ctr), g in zip(cases, got):
        c = np.asarray(ctr, dtype=np.uint64).astype(np.uint32)
        key = np.broadcast_to(np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32), (c.shape[0], 2))
        ref = philox4x32_10(c, key)
        assert np.array_equal(ref, g), (hex(seed), ref[:2], g[:2])
