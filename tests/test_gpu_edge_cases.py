"""Edge cases of the product path, limb for limb against the oracle: the
degenerate baby-step / giant-step splits of the diagonal method (App. C.1):
b1 = 1 (giant steps only) and b1 = k (baby steps only, no giant-step key
switching); one column per ciphertext (k = 1: no rotation at all); a single
input and output column (d = d_out = 1); an all-zero weight matrix; the lowest
level that can still rescale (level 1, output at level 0); an empty encoding;
and empty or mismatched inputs, which the boundary refuses (BLB_ERR_ARG /
BLB_ERR_LEVEL) without touching the device."""
import numpy as np
import pytest

from paper_2508_19525_b300 import workloads as wl

from _helpers import cp_rotations, make_ctx, make_oracle, oracle_galois, pack_cols, unpack_cols

pytestmark = pytest.mark.gpu
SEED = 0xED6E


CASES = [
    # params, m, d, d_out, b1, level (None: the top level), all-zero W
    (wl.SMALL, 64, 80, 40, 1, None, False),     # k = 32, b1 = 1: G = 32 giant steps only
    (wl.SMALL, 64, 80, 40, 32, None, False),    # b1 = k: G = 1, baby steps only
    (wl.SMALL, 2048, 3, 2, 1, None, False),     # k = 1: three inputs, two outputs, no rotation
    (wl.SMALL, 32, 1, 1, 8, None, False),       # a single input and output column
    (wl.SMALL, 64, 80, 40, 4, None, True),      # W = 0
    (wl.SMALL, 64, 80, 40, 4, 1, False),        # level 1 -> output at level 0
]


@pytest.mark.parametrize("prm,m,d,d_out,b1,level,zero_w", CASES)
def test_matmul_cp_edge_cases_match_the_oracle(prm, m, d, d_out, b1, level, zero_w):
    o, ctx = make_oracle(prm), make_ctx(prm)
    k = o.N // 2 // m
    G = k // b1
    level = o.nQ - 1 if level is None else level
    X, W = wl.cp_operands(m, d, d_out, seed=m + d + b1)
    if zero_w:
        W = np.zeros_like(W)
    nX = (d + k - 1) // k
    rots = cp_rotations(m, b1, G)
    if k == 1:
        assert rots == []
    sk = o.keygen_secret(SEED)
    keys = ctx.keygen(SEED, rots)
    zs = pack_cols(X, m, k, nX)
    cts = [ctx.encrypt(keys, ctx.encode(z, level), nonce=c) for c, z in enumerate(zs)]
    ref_in = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, c) for c, z in enumerate(zs)])
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)
    info = plan.info()
    assert (info["nX"], info["b1"], info["G"]) == (nX, b1, G)
    Y = ctx.matmul_cp_plan(keys, plan, cts)
    ref = o.matmul_cp(ref_in, m, d, W, d_out, b1, oracle_galois(o, sk, SEED, rots))
    assert len(Y) == len(ref) == (d_out + k - 1) // k
    slots = []
    for e, y in enumerate(Y):
        assert y.level == level - 1
        assert np.array_equal(ctx.ct_export(y), ref[e]), e
        slots.append(ctx.decrypt(keys, y, coeffs=False)[1])
    assert np.abs(unpack_cols(slots, m, k, d_out) - X @ W).max() <= 1e-4


def test_empty_encoding_is_the_zero_plaintext():
    prm = wl.SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    level = o.nQ - 1
    pt = ctx.encode(np.zeros(0), level)
    got = ctx.pt_export(pt, level)
    assert np.array_equal(got, o.encode(np.zeros(o.N // 2), level, prm.scale))
    assert not got.any()


def test_empty_and_mismatched_inputs_are_refused():
    from paper_2508_19525_b300 import blb
    prm, m, d, d_out, b1 = wl.SMALL, 64, 80, 40, 4
    ctx = make_ctx(prm)
    k = ctx.N // 2 // m
    level = ctx.nQ - 1
    keys = ctx.keygen(SEED, cp_rotations(m, b1, k // b1))
    X, W = wl.cp_operands(m, d, d_out, seed=3)
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)
    cts = [ctx.encrypt(keys, ctx.encode(z, level), c) for c, z in enumerate(pack_cols(X, m, k, 3))]
    for bad in ([], cts[:2]):  # no inputs; one input fewer than the plan's nX
        with pytest.raises(blb.BlbError) as e:
            ctx.matmul_cp_plan(keys, plan, bad)
        assert e.value.code == blb.ERR_ARG
    with pytest.raises(blb.BlbError) as e:  # an empty batch
        ctx.matmul_cp_batch(keys, plan, [])
    assert e.value.code == blb.ERR_ARG
    low = [ctx.encrypt(keys, ctx.encode(z, level - 1), c) for c, z in enumerate(pack_cols(X, m, k, 3))]
    with pytest.raises(blb.BlbError) as e:  # inputs at another level than the plan's
        ctx.matmul_cp_plan(keys, plan, low)
    assert e.value.code == blb.ERR_LEVEL
    with pytest.raises(blb.BlbError) as e:  # b1 must divide k
        ctx.cp_plan(m, d, W, d_out, level, 3)
    assert e.value.code == blb.ERR_ARG
    # the context is still usable: the product equals a fresh one
    Y = ctx.matmul_cp_plan(keys, plan, cts)
    Y2 = ctx.matmul_cp_plan(keys, plan, cts)
    assert all(np.array_equal(ctx.ct_export(a), ctx.ct_export(b)) for a, b in zip(Y, Y2))
