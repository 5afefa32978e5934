"""GPU matmul_cc (Sec. 5.1, App. C.1) against the oracle, bit-exact on every
RNS limb, and at the BERT-base attention size (N = 2^16, 12 primes, 12 heads
in groups of 8 and 4, L = 128, head dim 64) against FP64 within 1e-4."""
import numpy as np
import pytest

import cc_schedule as cs
import oracle
from paper_2508_19525_b300 import workloads as wl

from _helpers import make_ctx, make_oracle

pytestmark = pytest.mark.gpu
SEED = 0xCC


def operands(kind, L, Hg, R, seed):
    Q, K, V, P = wl.attention_operands(L, Hg, R, seed=seed)
    if kind == "qk":
        return Q, np.transpose(K, (0, 2, 1))
    return P, np.concatenate([V, np.zeros((Hg, L, L - V.shape[2]))], axis=2)


def gpu_cc(ctx, keys, plan, A, B, L, Hg, level, scale):
    info = plan.info()
    Kc, n_c = info["Kc"], info["n_c"]
    Az = cs.pack(A, L, Hg, Kc, n_c, rows=False)
    Bz = cs.pack(B, L, Hg, Kc, n_c, rows=True)
    Ac = [ctx.encrypt(keys, ctx.encode(z, level, scale), c) for c, z in enumerate(Az)]
    Bc = [ctx.encrypt(keys, ctx.encode(z, level, scale), 100 + c) for c, z in enumerate(Bz)]
    C = ctx.matmul_cc_plan(keys, plan, Ac, Bc)
    zs = np.stack([ctx.decrypt(keys, c, coeffs=False)[1] for c in C])
    return C, cs.unpack_diagonals(zs, L, Hg, Kc), Az, Bz


@pytest.mark.parametrize("kind,R,b1s1,b1s2", [("qk", 16, 4, 8), ("qk", 32, 2, 4), ("pv", 16, 4, 8)])
def test_matmul_cc_parity_with_oracle(kind, R, b1s1, b1s2):
    prm = wl.SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    L, Hg = 32, 4
    level = o.nQ - 1
    A, B = operands(kind, L, Hg, R, seed=R)
    plan = ctx.cc_plan(L, Hg, R if kind == "qk" else L, level, b1s1, b1s2)
    rots = plan.rotations()
    keys = ctx.keygen(SEED, rots, relin=True)
    C, got, Az, Bz = gpu_cc(ctx, keys, plan, A, B, L, Hg, level, prm.scale)
    # the same inputs through the oracle
    sk = o.keygen_secret(SEED)
    Ao = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, c) for c, z in enumerate(Az)])
    Bo = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 100 + c) for c, z in enumerate(Bz)])
    gal = {o.galois_elt(r): o.keygen_galois(SEED, sk, o.galois_elt(r)) for r in rots}
    ref = o.matmul_cc(Ao, Bo, L, Hg, b1s1, b1s2, gal, o.keygen_relin(SEED, sk))
    assert len(C) == ref.shape[0]
    for j, c in enumerate(C):
        assert c.level == level - 4
        assert np.array_equal(ctx.ct_export(c), ref[j]), j
    err = np.abs(got - np.einsum("hik,hkj->hij", A, B))
    assert err.max() <= 1e-4


def test_matmul_cc_bert_base_attention_size():
    prm = wl.BERT_CC
    ctx = make_ctx(prm)
    L, Dh, level = 128, 64, ctx.nQ - 1
    plans = {Hg: (ctx.cc_plan(L, Hg, Dh, level), ctx.cc_plan(L, Hg, L, level)) for Hg in (8, 4)}
    rots = sorted({r for pq, pv in plans.values() for r in pq.rotations() + pv.rotations()})
    keys = ctx.keygen(SEED, rots, relin=True)
    for Hg, (pq, pv) in plans.items():
        for kind, plan in (("qk", pq), ("pv", pv)):
            A, B = operands(kind, L, Hg, Dh, seed=Hg)
            _, got, _, _ = gpu_cc(ctx, keys, plan, A, B, L, Hg, level, prm.scale)
            err = np.abs(got - np.einsum("hik,hkj->hij", A, B))
            assert err.max() <= 1e-4, (kind, Hg, err.max())
