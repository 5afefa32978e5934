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
