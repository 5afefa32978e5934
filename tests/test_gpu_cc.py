"""GPU matmul_cc (Sec. 5.1, App. C.1) against the oracle, bit-exact on every
RNS limb (also with steps 1-2 in chunks), and at the BERT-base attention size
(N = 2^16, 12 primes, 12 heads in groups of 8 and 4, L = 128, head dim 64) and
a BERT-large one (16 heads, L = 256) against FP64 within 1e-4."""
import numpy as np
import pytest

import cc_schedule as cs
import oracle
from paper_2508_19525_b300 import workloads as wl

from _helpers import assert_limbs_consistent, make_ctx, make_oracle

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
    zs = []
    for c in C:
        coeffs, z = ctx.decrypt(keys, c)
        assert_limbs_consistent(coeffs, ctx.primes)  # every limb, not only the decoded q_0
        zs.append(z)
    return C, cs.unpack_diagonals(np.stack(zs), L, Hg, Kc), Az, Bz


@pytest.mark.parametrize("kind,R,b1s1,b1s2,L,Hg,chunks", [
    ("qk", 16, 4, 8, 32, 4, (0, 0)), ("qk", 32, 2, 4, 32, 4, (0, 0)), ("pv", 16, 4, 8, 32, 4, (0, 0)),
    ("pv", 16, 4, 8, 32, 4, (1, 5)),      # one input ciphertext per pass, ragged diagonal chunks
    ("qk", 16, 2, 4, 64, 2, (0, 24)),     # Kc = 16, four output ciphertexts
    ("qk", 32, 4, 4, 32, 2, (0, 0))])     # Kc = L: one output, all-ones step-3 masks
def test_matmul_cc_parity_with_oracle(kind, R, b1s1, b1s2, L, Hg, chunks):
    prm = wl.SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    level = o.nQ - 1
    A, B = operands(kind, L, Hg, R, seed=R)
    plan = ctx.cc_plan(L, Hg, R if kind == "qk" else L, level, b1s1, b1s2, *chunks)
    info = plan.info()
    if chunks[0]:
        assert info["c_chunk"] == chunks[0] < info["n_c"]
    if chunks[1]:
        assert info["t_chunk"] == chunks[1]
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


def test_matmul_cc_bert_large_long_sequence():
    """BERT-large attention shape, 16 heads in one group at L = 256 (Kc = 8):
    Q K^T (8 input ciphertexts per operand for head dim 64) and P V (32, steps
    1-2 in chunks under an 8 GiB workspace budget) against FP64."""
    prm = wl.BERT_CC
    ctx = make_ctx(prm)
    L, Dh, Hg, level = 256, 64, 16, ctx.nQ - 1
    pq, pv = ctx.cc_plan(L, Hg, Dh, level), ctx.cc_plan(L, Hg, L, level, workspace_bytes=8 << 30)
    info = pv.info()
    assert info["Kc"] == 8 and info["n_c"] == 32
    assert 1 < info["c_chunk"] < info["n_c"]
    rots = sorted(set(pq.rotations()) | set(pv.rotations()))
    keys = ctx.keygen(SEED, rots, relin=True)
    for kind, plan in (("qk", pq), ("pv", pv)):
        A, B = operands(kind, L, Hg, Dh, seed=3)
        _, got, _, _ = gpu_cc(ctx, keys, plan, A, B, L, Hg, level, prm.scale)
        err = np.abs(got - np.einsum("hik,hkj->hij", A, B))
        assert err.max() <= 1e-4, (kind, err.max())


def test_cc_plan_masks_at_512_tokens():
    """At L = 512 (16 heads, Kc = 4) the plan stores 2 Kc step-1 masks, 2 L
    step-2 masks and at most 2 Kc distinct step-3 masks (of L^2/Kc)."""
    prm = wl.BERT_CC
    ctx = make_ctx(prm)
    L, Hg, level = 512, 16, ctx.nQ - 1
    plan = ctx.cc_plan(L, Hg, L, level)
    info = plan.info()
    Kc, N = info["Kc"], ctx.N
    assert Kc == 4
    limbs = 2 * Kc * (level + 1) + 2 * L * level
    assert (limbs * N * 8) < info["mask_bytes"] <= (limbs + 2 * Kc * (level - 2)) * N * 8


def test_matmul_cc_captured_graph_replays_the_product():
    """P V at N = 2^12 (two input ciphertexts, steps 1-2 in chunks of one)
    captured as one CUDA graph: a replay gives the eager limbs, and after new
    operands are copied into the captured inputs a replay gives the eager
    limbs for those."""
    import torch
    from paper_2508_19525_b300 import blb
    prm = wl.SMALL
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, prm.dnum, prm.scale, stream=torch.cuda.Stream())
    L, Hg, R = 32, 4, 32
    level = ctx.nQ - 1
    plan = ctx.cc_plan(L, Hg, R, level, 4, 8, 1, 0)
    keys = ctx.keygen(SEED, plan.rotations(), relin=True)
    info = plan.info()
    Kc, n_c = info["Kc"], info["n_c"]

    def encrypt(seed, base):
        A, B = operands("pv", L, Hg, 16, seed=seed)
        Az, Bz = cs.pack(A, L, Hg, Kc, n_c, rows=False), cs.pack(B, L, Hg, Kc, n_c, rows=True)
        return ([ctx.encrypt(keys, ctx.encode(z, level, prm.scale), base + c) for c, z in enumerate(Az)],
                [ctx.encrypt(keys, ctx.encode(z, level, prm.scale), base + 50 + c) for c, z in enumerate(Bz)],
                np.einsum("hik,hkj->hij", A, B))

    Ac, Bc, _ = encrypt(1, 0)
    An, Bn, want = encrypt(2, 200)
    graph, Cg = ctx.capture(lambda: ctx.matmul_cc_plan(keys, plan, Ac, Bc))
    graph.replay()
    torch.cuda.synchronize()
    eager = ctx.matmul_cc_plan(keys, plan, Ac, Bc)
    for a, b in zip(Cg, eager):
        assert np.array_equal(ctx.ct_export(a), ctx.ct_export(b))
    for dst, src in zip(Ac + Bc, An + Bn):
        ctx.ct_copy(dst, src)
    graph.replay()
    torch.cuda.synchronize()
    eager2 = ctx.matmul_cc_plan(keys, plan, An, Bn)
    for a, b in zip(Cg, eager2):
        assert np.array_equal(ctx.ct_export(a), ctx.ct_export(b))
    zs = np.stack([ctx.decrypt(keys, c, coeffs=False)[1] for c in Cg])
    assert np.abs(cs.unpack_diagonals(zs, L, Hg, Kc) - want).max() <= 1e-4
