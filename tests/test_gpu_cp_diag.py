"""GPU diagonal-input matmul_cp (App. C.2): limb-for-limb parity with the oracle,
and the BERT-base attention chain Softmax x V_h (matmul_cc, 12 heads as groups of
8 and 4, L = 128, head dim 64, N = 2^16) -> merge of complementary diagonals ->
Concat(Att_h) W_O, against FP64 within 1e-4."""
import numpy as np
import pytest

import cc_schedule as cs
import oracle
from paper_2508_19525_b300 import workloads as wl

from _helpers import make_ctx, make_oracle
from test_oracle_cp_diag import cp_rots, dense_diagonals, unpack_spatial

pytestmark = pytest.mark.gpu
SEED = 0xD1A7


def test_diag_cp_parity_with_oracle():
    prm = wl.SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    s, L, Dh, groups, d_out, b1 = o.N // 2, 32, 16, [4, 4], 64, 8
    k, H = s // L, sum(groups)
    rng = np.random.default_rng(3)
    Att = rng.uniform(-1, 1, (H, L, Dh))
    W = rng.uniform(-1, 1, (H * Dh, d_out))
    level = o.nQ - 1
    rots = cp_rots(L, k, b1)
    keys = ctx.keygen(SEED, rots)
    sk = o.keygen_secret(SEED)
    zs, h0 = [], 0
    for Hg in groups:
        Kc = s // (L * Hg)
        zs += list(dense_diagonals(Att[h0:h0 + Hg], L, Hg, Kc, Dh))
        h0 += Hg
    X = [ctx.encrypt(keys, ctx.encode(z, level), c) for c, z in enumerate(zs)]
    Xo = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, c) for c, z in enumerate(zs)])
    plan = ctx.cp_plan_diag(L, groups, Dh, W, d_out, level, b1)
    assert plan.info()["nX"] == len(zs)
    Y = ctx.matmul_cp_plan(keys, plan, X)
    gal = {o.galois_elt(r): o.keygen_galois(SEED, sk, o.galois_elt(r)) for r in rots}
    ref = o.matmul_cp_diag(Xo, L, groups, Dh, W, d_out, b1, gal)
    assert len(Y) == len(ref)
    for e, y in enumerate(Y):
        assert np.array_equal(ctx.ct_export(y), ref[e]), e
    slots = [ctx.decrypt(keys, y, coeffs=False)[1] for y in Y]
    E = np.concatenate([Att[h] for h in range(H)], axis=1) @ W
    assert np.abs(unpack_spatial(slots, L, k, d_out) - E).max() <= 1e-4


def test_bert_base_attention_chain_to_output_projection():
    prm = wl.BERT_CC
    ctx = make_ctx(prm)
    s, L, Dh, H = ctx.N // 2, 128, 64, 12
    groups = [8, 4]
    level = ctx.nQ - 1
    k = s // L
    plans = {Hg: ctx.cc_plan(L, Hg, L, level) for Hg in groups}
    _, _, V, P = wl.attention_operands(L, H, Dh, seed=11)
    Wo = wl.uniform((H * Dh, H * Dh), seed=12)
    cc_out_level = level - 4
    diag = ctx.cp_plan_diag(L, groups, Dh, Wo, H * Dh, cc_out_level)
    info = diag.info()
    rots = sorted({r for p in plans.values() for r in p.rotations()} |
                  {b * L for b in range(1, info["b1"])} | {g * info["b1"] * L for g in range(1, info["G"])})
    keys = ctx.keygen(SEED, rots, relin=True)
    merged, h0 = [], 0
    for Hg in groups:
        pl = plans[Hg]
        pi = pl.info()
        A = P[h0:h0 + Hg]
        B = np.concatenate([V[h0:h0 + Hg], np.zeros((Hg, L, L - Dh))], axis=2)
        Az = cs.pack(A, L, Hg, pi["Kc"], pi["n_c"], rows=False)
        Bz = cs.pack(B, L, Hg, pi["Kc"], pi["n_c"], rows=True)
        Ac = [ctx.encrypt(keys, ctx.encode(z, level), 10 * h0 + c) for c, z in enumerate(Az)]
        Bc = [ctx.encrypt(keys, ctx.encode(z, level), 10 * h0 + 5 + c) for c, z in enumerate(Bz)]
        C = ctx.matmul_cc_plan(keys, pl, Ac, Bc)
        half = Dh // pi["Kc"]
        merged += [ctx.add(C[j], C[j + half]) for j in range(half)]
        h0 += Hg
    E_ct = ctx.matmul_cp_plan(keys, diag, merged)
    slots = [ctx.decrypt(keys, y, coeffs=False)[1] for y in E_ct]
    Att = np.einsum("hik,hkj->hij", P, V)
    E = np.concatenate([Att[h] for h in range(H)], axis=1) @ Wo
    err = np.abs(unpack_spatial(slots, L, k, H * Dh) - E).max()
    assert err <= 1e-4, err
