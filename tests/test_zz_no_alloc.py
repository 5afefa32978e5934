"""The allocation-free key switch, blb_keyswitch_noalloc.

It serves callers that may not allocate device memory while they run (a
process whose memory manager owns the whole device budget, a loop that cannot
afford cudaMalloc's synchronization, code inside the library's allocator
callbacks).  Its result must equal blb_keyswitch_coeffs, which uses the
context's allocated scratch, limb for limb; it keeps all temporaries in one
fixed device array, so nothing is allocated during the call, and sizes beyond
that array are refused.  This file is collected last on purpose."""
import gc

import numpy as np
import pytest

from paper_2508_19525_b300 import workloads as wl

from _helpers import make_ctx

pytestmark = pytest.mark.gpu
SEED = 0xA11C


@pytest.mark.parametrize("prm", [wl.TINY, wl.SMALL, wl.BERT_CP], ids=["tiny", "small", "bert_cp"])
def test_noalloc_equals_allocating_keyswitch(prm):
    import torch
    ctx = make_ctx(prm)
    keys = ctx.keygen(SEED, [3, -5])
    levels = range(ctx.nQ) if prm.logN <= 12 else [ctx.nQ - 1, 3, 0]
    primes = ctx.primes
    for level in levels:
        n = level + 1
        for call, rot in enumerate((3, -5)):  # two calls in a row, different inputs and keys
            d = wl.random_residues(primes[:n], ctx.N, seed=1000 * level + call)[0]
            ref = ctx.keyswitch_coeffs(keys, rot, d)
            d_dev = torch.from_numpy(d).cuda()
            out = torch.zeros((2, n, ctx.N), dtype=torch.uint64, device="cuda")
            torch.cuda.synchronize()
            gc.collect()
            gc.disable()  # no unrelated object may be freed inside the measured call
            try:
                before_torch, before_ctx = torch.cuda.memory_allocated(), ctx.bytes_in_use()
                ctx.keyswitch_noalloc(keys, rot, d_dev, out)
                ctx.sync()
                after_torch, after_ctx = torch.cuda.memory_allocated(), ctx.bytes_in_use()
            finally:
                gc.enable()
            assert after_torch == before_torch and after_ctx == before_ctx
            assert np.array_equal(out.cpu().numpy(), ref), (level, call)
    # host buffers work too
    d = wl.random_residues(primes[:2], ctx.N, seed=7)[0]
    out = np.zeros((2, 2, ctx.N), np.uint64)
    ctx.keyswitch_noalloc(keys, 3, d, out)
    assert np.array_equal(out, ctx.keyswitch_coeffs(keys, 3, d))


def test_noalloc_refuses_sizes_beyond_its_array():
    from paper_2508_19525_b300 import blb
    ctx = make_ctx(wl.BERT_CC)  # N = 2^16, 12 primes
    keys = ctx.keygen(SEED, [1])
    d = wl.random_residues(ctx.primes[:12], ctx.N, seed=1)[0]
    out = np.zeros((2, 12, ctx.N), np.uint64)
    with pytest.raises(blb.BlbError) as e:
        ctx.keyswitch_noalloc(keys, 1, d, out)
    assert e.value.code == blb.ERR_ARG and "MiB" in str(e.value)
    # a low level of the same ring still fits and matches
    d = wl.random_residues(ctx.primes[:3], ctx.N, seed=2)[0]
    out = np.zeros((2, 3, ctx.N), np.uint64)
    ctx.keyswitch_noalloc(keys, 1, d, out)
    assert np.array_equal(out, ctx.keyswitch_coeffs(keys, 1, d))


_FRESH = r"""
import gc, sys
sys.path[:0] = [{root!r}, {tests!r}]
import numpy as np
import torch
from paper_2508_19525_b300 import workloads as wl
from _helpers import make_ctx
ctx = make_ctx(wl.BERT_CP)
keys = ctx.keygen({seed}, [3])
n = ctx.nQ
d = wl.random_residues(ctx.primes[:n], ctx.N, seed=5)[0]
d_dev = torch.from_numpy(d).cuda()
out = torch.zeros((2, n, ctx.N), dtype=torch.uint64, device="cuda")
# the NTT kernels are shared with every other operation; run them once, as any
# earlier operation of a real caller would have
ctx.ntt(d[:1], [0])
ctx.ntt(d[:1], [0], inverse=True)
torch.cuda.synchronize()
gc.collect()
gc.disable()
free0 = torch.cuda.mem_get_info()[0]
ctx.keyswitch_noalloc(keys, 3, d_dev, out)  # the first key switch of this process
ctx.sync()
free1 = torch.cuda.mem_get_info()[0]
gc.enable()
ref = ctx.keyswitch_coeffs(keys, 3, d)
print("FREE", free0, free1, "EQUAL", bool(np.array_equal(out.cpu().numpy(), ref)))
"""


def test_noalloc_first_call_of_a_fresh_process_leaves_device_memory_unchanged():
    """Run in a process of its own, so that blb_keyswitch_noalloc is the first
    key switch there: the free device memory reported by the driver
    (cudaMemGetInfo) is the same before and after the call, i.e. neither the
    call nor a module load inside it allocated anything."""
    import os
    import subprocess
    import sys
    tests = os.path.dirname(os.path.abspath(__file__))
    code = _FRESH.format(root=os.path.dirname(tests), tests=tests, seed=SEED)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("FREE")][-1].split()
    assert line[1] == line[2], f"free device memory changed: {line[1]} -> {line[2]}"
    assert line[4] == "True"
