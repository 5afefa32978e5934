"""Failure detection of the bounded device waits (no GPU fault involved).

The plaintext-product pipelines of matmul_cp (the mma.sync kernel of single
sequences and the tcgen05 kernel of batches) wait on shared-memory barriers
that their copy stage and operand builders complete.  With the copy stage told to
withhold its copies (a condition that nothing else completes) and a 1 ms wait
limit, every consumer's wait runs out: the kernel ends early, the copies it had
in flight (none here) are drained, and blb_ctx_sync reports BLB_ERR_TIMEOUT
once.  The context stays usable: the same product with normal settings then
equals the oracle limb for limb."""
import time

import numpy as np
import pytest

from paper_2508_19525_b300 import workloads as wl

from _helpers import cp_rotations, make_ctx, make_oracle, oracle_galois, pack_cols

pytestmark = pytest.mark.gpu
SEED = 0x7173


def test_expired_wait_reports_timeout_and_the_context_recovers():
    from paper_2508_19525_b300 import blb
    prm, m, d, d_out, b1 = wl.SMALL, 64, 80, 40, 4
    o, ctx = make_oracle(prm), make_ctx(prm)
    k = o.N // 2 // m
    level = o.nQ - 1
    rots = cp_rotations(m, b1, k // b1)
    keys = ctx.keygen(SEED, rots)
    X, W = wl.cp_operands(m, d, d_out, seed=3)
    zs = pack_cols(X, m, k, (d + k - 1) // k)
    cts = [ctx.encrypt(keys, ctx.encode(z, level), nonce=c) for c, z in enumerate(zs)]
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)
    ctx.sync()

    ctx.set_wait_limit(1_000_000)  # 1 ms
    ctx.test_withhold_copies(True)
    t0 = time.time()
    ctx.matmul_cp_plan(keys, plan, cts)
    with pytest.raises(blb.BlbError) as e:
        ctx.sync()
    assert e.value.code == blb.ERR_TIMEOUT
    assert time.time() - t0 < 30
    ctx.sync()  # reported once, then cleared

    ctx.test_withhold_copies(False)
    ctx.set_wait_limit(0)  # back to the 2 s default
    Y = ctx.matmul_cp_plan(keys, plan, cts)
    ctx.sync()
    sk = o.keygen_secret(SEED)
    ref_in = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, c) for c, z in enumerate(zs)])
    ref = o.matmul_cp(ref_in, m, d, W, d_out, b1, oracle_galois(o, sk, SEED, rots))
    for e_, y in enumerate(Y):
        assert np.array_equal(ctx.ct_export(y), ref[e_]), e_


def test_expired_wait_in_the_batched_tcgen05_product():
    """The same for a batch of two sequences (the tcgen05 kernel): the withheld
    copies make its waits run out, the tensor memory is freed, the next sync
    reports BLB_ERR_TIMEOUT, and the batch then equals the per-sequence
    products."""
    from paper_2508_19525_b300 import blb
    prm, m, d, d_out, b1 = wl.SMALL, 64, 80, 40, 4
    ctx = make_ctx(prm)
    k = ctx.N // 2 // m
    level = ctx.nQ - 1
    keys = ctx.keygen(SEED, cp_rotations(m, b1, k // b1))
    W = wl.cp_operands(m, d, d_out, seed=5)[1]
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)
    seqs = []
    for s_ in range(2):
        X = wl.cp_operands(m, d, d_out, seed=20 + s_)[0]
        seqs.append([ctx.encrypt(keys, ctx.encode(z, level), 10 * s_ + c)
                     for c, z in enumerate(pack_cols(X, m, k, (d + k - 1) // k))])
    ctx.sync()
    ctx.set_batch_mac(2)  # the tcgen05 kernel
    ctx.set_wait_limit(1_000_000)
    ctx.test_withhold_copies(True)
    ctx.matmul_cp_batch(keys, plan, seqs)
    with pytest.raises(blb.BlbError) as e:
        ctx.sync()
    assert e.value.code == blb.ERR_TIMEOUT
    ctx.test_withhold_copies(False)
    ctx.set_wait_limit(0)
    batched = ctx.matmul_cp_batch(keys, plan, seqs)
    ctx.sync()
    for s_, X in enumerate(seqs):
        for a, b in zip(batched[s_], ctx.matmul_cp_plan(keys, plan, X)):
            assert np.array_equal(ctx.ct_export(a), ctx.ct_export(b)), s_
