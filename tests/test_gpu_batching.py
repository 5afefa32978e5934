"""Batching on the GPU.  Token-chunked matmul_cp: uneven-length sequences cut
into m-row chunks; the batched product equals the per-chunk product limb for
limb and every token's output is X W within 1e-4; the autotuner returns a
measured (b1, chunks per call) choice whose results decode to the same
product.  Packed matmul_cc: several sequences of one padded length in one
product as the heads of one group, limb for limb against the oracle and each
sequence within 1e-4 of its own FP64 products."""
import numpy as np
import pytest

from paper_2508_19525_b300 import batching as bt
from paper_2508_19525_b300 import layer as ly
from paper_2508_19525_b300 import workloads as wl

from _helpers import make_ctx, make_oracle

pytestmark = pytest.mark.gpu
SEED = 0xBA7C


def test_batched_chunks_equal_plain_and_fp64():
    prm = wl.SMALL
    ctx = make_ctx(prm)
    m, d, d_out = 8, 64, 96
    s = ctx.N // 2
    k = s // m
    lengths = [3, 17, 9, 30, 1, 12]
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (sum(lengths), d))
    W = rng.uniform(-1, 1, (d, d_out))
    level = ctx.nQ - 1
    n_cts = -(-d // k)
    cands = (8, 16)
    keys = ctx.keygen(SEED, sorted({r for b1 in cands for r in bt.cp_rotations(m, k, b1)}))
    Z = bt.pack_chunks(X, m, k, n_cts)
    chunks = [ctx.encrypt_batch(keys, ctx.encode_batch(Z[c], level), [100 * c + i for i in range(n_cts)])
              for c in range(len(Z))]
    (b1, group), timings = bt.autotune(ctx, keys, m, d, W, d_out, level, chunks, cands, (1, 2, 4))
    assert b1 in cands and group in (1, 2, 4) and len(timings) == 6 and all(t > 0 for t in timings.values())
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)
    batched = bt.run_batched(ctx, keys, plan, chunks, 4)
    plain = [ctx.matmul_cp_plan(keys, plan, ch) for ch in chunks]
    for c in range(len(chunks)):
        for yb, yp in zip(batched[c], plain[c]):
            assert np.array_equal(ctx.ct_export(yb), ctx.ct_export(yp)), c
    Y = np.concatenate([bt.unpack_chunk([ctx.decrypt(keys, y, coeffs=False)[1] for y in batched[c]], m, k, d_out)
                        for c in range(len(chunks))])[:len(X)]
    assert np.abs(Y - X @ W).max() < 1e-4


def test_captured_graph_replays_the_batched_product():
    """The batched product over all chunks captured once: a replay gives the
    eager result limb for limb, and after new inputs are copied into the same
    ciphertexts a replay gives the eager result for those."""
    import torch
    from paper_2508_19525_b300 import blb
    prm = wl.SMALL
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, prm.dnum, prm.scale, stream=torch.cuda.Stream())
    m, d, d_out, b1 = 8, 64, 96, 8
    s = ctx.N // 2
    k = s // m
    level = ctx.nQ - 1
    keys = ctx.keygen(SEED, bt.cp_rotations(m, k, b1))
    rng = np.random.default_rng(9)
    W = rng.uniform(-1, 1, (d, d_out))
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)

    def encrypt(X, base):
        Z = bt.pack_chunks(X, m, k, 1)
        return [ctx.encrypt_batch(keys, ctx.encode_batch(Z[c], level), [base + c]) for c in range(len(Z))]

    X1, X2 = rng.uniform(-1, 1, (40, d)), rng.uniform(-1, 1, (40, d))
    chunks, new = encrypt(X1, 0), encrypt(X2, 100)
    graph, Yg = ctx.capture(lambda: bt.run_batched(ctx, keys, plan, chunks, 2))
    graph.replay()
    torch.cuda.synchronize()
    eager = bt.run_batched(ctx, keys, plan, chunks, 2)
    for a, b in zip(Yg, eager):
        for ya, yb in zip(a, b):
            assert np.array_equal(ctx.ct_export(ya), ctx.ct_export(yb))
    for dst, src in zip(chunks, new):
        ctx.ct_copy(dst[0], src[0])
    graph.replay()
    torch.cuda.synchronize()
    eager2 = bt.run_batched(ctx, keys, plan, new, 2)
    for a, b in zip(Yg, eager2):
        for ya, yb in zip(a, b):
            assert np.array_equal(ctx.ct_export(ya), ctx.ct_export(yb))
    got = np.concatenate([bt.unpack_chunk([ctx.decrypt(keys, y, coeffs=False)[1] for y in Yg[c]], m, k, d_out)
                          for c in range(len(Yg))])[:40]
    assert np.abs(got - X2 @ W).max() < 1e-4


def _seq_operands(kind, L, heads, R, length, seed):
    """One sequence's operands at padded length L: rows and columns past its
    length are zero (P renormalised over its first `length` rows' entries)."""
    Q, K, V, P = wl.attention_operands(L, heads, R, seed=seed)
    for M in (Q, K, V):
        M[:, length:] = 0.0
    if kind == "qk":
        return Q, np.transpose(K, (0, 2, 1))
    P[:, length:, :] = 0.0
    P[:, :, length:] = 0.0
    P[:, :length] /= P[:, :length].sum(axis=2, keepdims=True)
    return P, np.concatenate([V, np.zeros((heads, L, L - R))], axis=2)


@pytest.mark.parametrize("kind,L,heads,R,lengths", [
    ("qk", 32, 4, 16, (20, 32)),              # two sequences: Hg = 8, Kc = 8
    ("pv", 32, 4, 8, (32, 7, 19, 26)),        # four: Hg = 16, Kc = 4
    ("qk", 16, 4, 8, (16,) * 16 + (3,) * 16),  # thirty-two: Hg = 128, Kc = 1 (one block per head)
])
def test_cc_sequences_packed_as_heads_match_oracle_and_each_sequence(kind, L, heads, R, lengths):
    """Several sequences of one client, of one padded length, in one matmul_cc
    product as S x heads heads of one group (cc_pack_groups): every limb equals
    the oracle's product of the same packed operands, and each sequence's
    heads decrypt to that sequence's own products within 1e-4."""
    prm = wl.SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    S = len(lengths)
    Hg = S * heads
    level = o.nQ - 1
    assert bt.cc_pack_groups([L] * S, heads, ctx.N // 2) == [(L, list(range(S)))]
    ops = [_seq_operands(kind, L, heads, R, n, seed=31 + j) for j, n in enumerate(lengths)]
    A = bt.stack_heads([a for a, _ in ops])
    B = bt.stack_heads([b for _, b in ops])
    plan = ctx.cc_plan(L, Hg, R if kind == "qk" else L, level)
    info = plan.info()
    Kc, n_c = info["Kc"], info["n_c"]
    assert Kc == ctx.N // 2 // (L * Hg)
    rots = plan.rotations()
    keys = ctx.keygen(SEED, rots, relin=True)
    Az = ly.pack_heads(A, L, Hg, Kc, n_c, rows=False)
    Bz = ly.pack_heads(B, L, Hg, Kc, n_c, rows=True)
    Ac = [ctx.encrypt(keys, ctx.encode(z, level, prm.scale), c) for c, z in enumerate(Az)]
    Bc = [ctx.encrypt(keys, ctx.encode(z, level, prm.scale), 500 + c) for c, z in enumerate(Bz)]
    C = ctx.matmul_cc_plan(keys, plan, Ac, Bc)
    sk = o.keygen_secret(SEED)
    Ao = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, c) for c, z in enumerate(Az)])
    Bo = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 500 + c) for c, z in enumerate(Bz)])
    gal = {o.galois_elt(r): o.keygen_galois(SEED, sk, o.galois_elt(r)) for r in rots}
    ref = o.matmul_cc(Ao, Bo, L, Hg, info["b1s1"], info["b1s2"], gal, o.keygen_relin(SEED, sk))
    assert len(C) == ref.shape[0] == L // Kc
    for j, c in enumerate(C):
        assert np.array_equal(ctx.ct_export(c), ref[j]), j
    Z = np.stack([ctx.decrypt(keys, c, coeffs=False)[1] for c in C])
    got = bt.split_heads(ly.unpack_diagonals(Z, L, Hg, Kc), S)
    for j, (a, b) in enumerate(ops):
        assert np.abs(got[j] - np.einsum("hik,hkj->hij", a, b)).max() <= 1e-4, j
