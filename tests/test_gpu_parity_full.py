"""GPU against the oracle, limb for limb, at the term counts and head shapes the
benchmarked workloads run, on the smallest ring that holds them (N = 2^12,
primes 60 + 4 x 40, special primes 2 x 60, dnum 3):

* matmul_cp (Sec. 4.2.1 / 5.2, BSGS of App. C.1) with 96 terms per output and
  giant step (nX = 6 inputs x b1 = 16, the BERT-base step's contraction),
  64 terms (one input x b1 = 64, the BERT-large chunk products' contraction)
  and 192 terms (two 128-term segments of the tensor-core MAC), each with a
  ragged last output ciphertext; and batches of 9 sequences at 96 terms (one
  8-sequence launch and one single-sequence launch), the first and last
  sequence against the oracle and all of them against one call per sequence;
* matmul_cc (Sec. 5.1) at L = 128 with head groups of 8 and 16 (Kc = 2 and 1),
  Q K^T-shaped and, for 8 heads, Softmax x V-shaped (64 input ciphertexts per
  operand, steps 1-2 in ragged chunks of input ciphertexts).
"""
import numpy as np
import pytest

import cc_schedule as cs
from paper_2508_19525_b300 import workloads as wl

from _helpers import (assert_limbs_consistent, cp_rotations, make_ctx, make_oracle, oracle_galois, pack_cols,
                      unpack_cols)

pytestmark = pytest.mark.gpu
SEED = 0xF1


def _cp_case(m, d, d_out, b1, n_seq=1):
    prm = wl.SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    k = o.N // 2 // m
    G = k // b1
    level = o.nQ - 1
    nX = (d + k - 1) // k
    rots = cp_rotations(m, b1, G)
    sk = o.keygen_secret(SEED)
    keys = ctx.keygen(SEED, rots)
    W = wl.cp_operands(m, d, d_out, seed=d + d_out)[1]
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)
    info = plan.info()
    assert (info["nX"], info["b1"], info["G"]) == (nX, b1, G)
    seqs = []
    for s in range(n_seq):
        X = wl.cp_operands(m, d, d_out, seed=100 + s)[0]
        zs = pack_cols(X, m, k, nX)
        cts = [ctx.encrypt(keys, ctx.encode(z, level), nonce=1000 * s + c) for c, z in enumerate(zs)]
        seqs.append((X, zs, cts))
    return prm, o, ctx, sk, keys, plan, W, seqs, (k, level, nX, rots)


def _oracle_cp(o, prm, sk, zs, s, m, d, W, d_out, b1, level, gal):
    ref_in = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 1000 * s + c) for c, z in enumerate(zs)])
    return ref_in, o.matmul_cp(ref_in, m, d, W, d_out, b1, gal)


@pytest.mark.parametrize("m,d,d_out,b1", [
    (16, 768, 200, 16),     # 96 terms (6 x 16), two outputs, the second ragged
    (2, 1024, 1500, 64),    # 64 terms (1 x 64), two outputs, the second ragged
    (16, 1536, 100, 16),    # 192 terms: two segments of 8 term tiles
])
def test_matmul_cp_full_term_counts_match_the_oracle(m, d, d_out, b1):
    prm, o, ctx, sk, keys, plan, W, seqs, (k, level, nX, rots) = _cp_case(m, d, d_out, b1)
    X, zs, cts = seqs[0]
    gal = oracle_galois(o, sk, SEED, rots)
    ref_in, ref = _oracle_cp(o, prm, sk, zs, 0, m, d, W, d_out, b1, level, gal)
    for c in range(nX):
        assert np.array_equal(ctx.ct_export(cts[c]), ref_in[c])
    Y = ctx.matmul_cp_plan(keys, plan, cts)
    assert len(Y) == len(ref) == (d_out + k - 1) // k
    slots = []
    for e, y in enumerate(Y):
        assert np.array_equal(ctx.ct_export(y), ref[e]), e
        coeffs, z = ctx.decrypt(keys, y)
        assert_limbs_consistent(coeffs, o.primes)
        slots.append(z)
    assert np.abs(unpack_cols(slots, m, k, d_out) - X @ W).max() <= 1e-4


def test_matmul_cp_batch_of_nine_at_96_terms_matches_the_oracle():
    m, d, d_out, b1 = 16, 768, 200, 16
    prm, o, ctx, sk, keys, plan, W, seqs, (k, level, nX, rots) = _cp_case(m, d, d_out, b1, n_seq=9)
    batched = ctx.matmul_cp_batch(keys, plan, [cts for _, _, cts in seqs])
    assert len(batched) == 9
    for s, (X, zs, cts) in enumerate(seqs):
        single = ctx.matmul_cp_plan(keys, plan, cts)
        for a, b in zip(batched[s], single):
            assert np.array_equal(ctx.ct_export(a), ctx.ct_export(b)), s
    gal = oracle_galois(o, sk, SEED, rots)
    for s in (0, 8):  # first sequence of the 8-sequence launch, and the ninth alone
        X, zs, _ = seqs[s]
        _, ref = _oracle_cp(o, prm, sk, zs, s, m, d, W, d_out, b1, level, gal)
        for e, y in enumerate(batched[s]):
            assert np.array_equal(ctx.ct_export(y), ref[e]), (s, e)
        got = unpack_cols([ctx.decrypt(keys, y, coeffs=False)[1] for y in batched[s]], m, k, d_out)
        assert np.abs(got - X @ W).max() <= 1e-4
    # both kernels of batched plaintext products (mma.sync and tcgen05) give these limbs
    for kind in (1, 2):
        ctx.set_batch_mac(kind)
        again = ctx.matmul_cp_batch(keys, plan, [cts for _, _, cts in seqs])
        for s in range(9):
            for a, b in zip(again[s], batched[s]):
                assert np.array_equal(ctx.ct_export(a), ctx.ct_export(b)), (kind, s)
    ctx.set_batch_mac(0)


@pytest.mark.parametrize("kind,L,Hg,R,b1s1,b1s2,c_chunk", [
    ("qk", 128, 8, 8, 2, 8, 0),      # Kc = 2, 4 input ciphertexts, 64 outputs
    ("qk", 128, 16, 2, 1, 16, 0),    # Kc = 1, 2 input ciphertexts, 128 outputs
    ("pv", 128, 8, 128, 1, 8, 5),    # Softmax x V: 64 input ciphertexts in chunks of 5
])
def test_matmul_cc_at_128_tokens_matches_the_oracle(kind, L, Hg, R, b1s1, b1s2, c_chunk):
    prm = wl.SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    level = o.nQ - 1
    Q, K, V, P = wl.attention_operands(L, Hg, 64 if kind == "pv" else R, seed=L + Hg + R)
    if kind == "qk":
        A, B = Q[:, :, :R], np.transpose(K[:, :, :R], (0, 2, 1))
    else:
        A, B = P, np.concatenate([V, np.zeros((Hg, L, L - V.shape[2]))], axis=2)
    plan = ctx.cc_plan(L, Hg, R, level, b1s1, b1s2, c_chunk, 0)
    info = plan.info()
    Kc, n_c = info["Kc"], info["n_c"]
    assert Kc == o.N // 2 // (L * Hg) and n_c == -(-R // Kc)
    if c_chunk:
        assert info["c_chunk"] == c_chunk and n_c % c_chunk
    rots = plan.rotations()
    keys = ctx.keygen(SEED, rots, relin=True)
    Az = cs.pack(A, L, Hg, Kc, n_c, rows=False)
    Bz = cs.pack(B, L, Hg, Kc, n_c, rows=True)
    Ac = [ctx.encrypt(keys, ctx.encode(z, level), c) for c, z in enumerate(Az)]
    Bc = [ctx.encrypt(keys, ctx.encode(z, level), 500 + c) for c, z in enumerate(Bz)]
    C = ctx.matmul_cc_plan(keys, plan, Ac, Bc)
    sk = o.keygen_secret(SEED)
    Ao = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, c) for c, z in enumerate(Az)])
    Bo = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 500 + c) for c, z in enumerate(Bz)])
    gal = {o.galois_elt(r): o.keygen_galois(SEED, sk, o.galois_elt(r)) for r in rots}
    ref = o.matmul_cc(Ao, Bo, L, Hg, b1s1, b1s2, gal, o.keygen_relin(SEED, sk))
    assert len(C) == ref.shape[0] == L // Kc
    for j, c in enumerate(C):
        assert np.array_equal(ctx.ct_export(c), ref[j]), j
    zs = np.stack([ctx.decrypt(keys, c, coeffs=False)[1] for c in C])
    err = np.abs(cs.unpack_diagonals(zs, L, Hg, Kc) - np.einsum("hik,hkj->hij", A, B))
    assert err.max() <= 1e-4
