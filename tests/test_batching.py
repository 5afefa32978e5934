"""Host logic of the batching: the token-chunked layout of uneven-length
sequences for matmul_cp (layout and spatial-first packing round trips), and
the packing of several sequences of one padded length into one matmul_cc head
group (grouping rules, and the schedule's algebra on plaintext slots)."""
import numpy as np
import pytest

import cc_schedule as cs
from paper_2508_19525_b300 import batching as bt


def test_layout_and_packing_round_trip():
    rng = np.random.default_rng(1)
    lengths = [3, 17, 9, 30, 1]
    m, k, d = 8, 16, 40
    n_cts = -(-d // k)
    T = sum(lengths)
    X = rng.uniform(-1, 1, (T, d))
    starts, n_chunks = bt.chunk_layout(lengths, m)
    assert list(starts) == [0, 3, 20, 29, 59] and n_chunks == -(-T // m)
    Z = bt.pack_chunks(X, m, k, n_cts)
    assert Z.shape == (n_chunks, n_cts, m * k)
    Xp = np.zeros((n_chunks * m, d))
    Xp[:T] = X
    for c in range(n_chunks):
        assert np.array_equal(bt.unpack_chunk(Z[c], m, k, d), Xp[c * m:(c + 1) * m])
    # column j of a chunk occupies slots [j m, (j+1) m) of ciphertext j // k
    c, j = 2, 21
    assert np.array_equal(Z[c, j // k, (j % k) * m:(j % k + 1) * m], Xp[c * m:(c + 1) * m, j])


def test_rotation_sets():
    m, k = 32, 1024
    for b1 in (16, 32, 64):
        rots = bt.cp_rotations(m, k, b1)
        assert len(rots) == (b1 - 1) + (k // b1 - 1)
        assert all(r % m == 0 and 0 < r < m * k for r in rots)


def test_cc_pack_groups_cover_every_sequence_once():
    rng = np.random.default_rng(7)
    lengths = rng.integers(16, 513, 32)
    pads = [max(64, 1 << int(np.ceil(np.log2(x)))) for x in lengths]
    slots, heads = 32768, 16
    for max_pack in (None, 1, 2, 4):
        groups = bt.cc_pack_groups(pads, heads, slots, max_pack)
        seen = sorted(i for _, idx in groups for i in idx)
        assert seen == list(range(len(pads)))
        for Lp, idx in groups:
            S = len(idx)
            assert S & (S - 1) == 0 and all(pads[i] == Lp for i in idx)
            assert slots % (Lp * S * heads) == 0           # Kc >= 1
            assert max_pack is None or S <= max_pack
        if max_pack == 1:
            assert len(groups) == len(pads)
    # greedy: 5 sequences of 64 tokens at s = 32768 (up to 32 per product) -> 4 + 1
    assert [len(i) for _, i in bt.cc_pack_groups([64] * 5, 16, 32768)] == [4, 1]
    # at 512 tokens Kc = 32768 / (512 S 16) >= 1 allows at most 4
    assert [len(i) for _, i in bt.cc_pack_groups([512] * 9, 16, 32768)] == [4, 4, 1]
    with pytest.raises(ValueError):
        bt.cc_pack_groups([64], 12, 32768)


@pytest.mark.parametrize("s,L,heads,S,R", [(256, 16, 4, 2, 8), (256, 16, 4, 4, 16), (128, 8, 2, 8, 8),
                                         (512, 16, 4, 2, 16)])
def test_cc_sequences_packed_as_heads_give_each_sequence_its_product(s, L, heads, S, R):
    """The schedule on plaintext slots (no encryption): S sequences' heads
    stacked into one head group of S x heads multiply exactly as each sequence
    alone, down to Kc = 1 (s = L S heads)."""
    Hg = S * heads
    Kc = s // (L * Hg)
    rng = np.random.default_rng(L + S)
    A = [rng.uniform(-1, 1, (heads, L, R)) for _ in range(S)]
    B = [rng.uniform(-1, 1, (heads, R, L)) for _ in range(S)]
    n_c = -(-R // Kc)
    Az = cs.pack(bt.stack_heads(A), L, Hg, Kc, n_c, rows=False)
    Bz = cs.pack(bt.stack_heads(B), L, Hg, Kc, n_c, rows=True)
    C, _ = cs.simulate(Az, Bz, L, Hg, 1, 1 if L < 4 else 2)
    got = bt.split_heads(cs.unpack_diagonals(C, L, Hg, Kc), S)
    for j in range(S):
        assert np.allclose(got[j], np.einsum("hik,hkj->hij", A[j], B[j]), atol=1e-12)


def test_rotation_count_per_token_falls_with_rows_per_ciphertext():
    """The rotation count of one m-row product: baby steps per input
    ciphertext plus giant steps per output ciphertext, checked against a
    direct count of the BSGS schedule's rotations (every nonzero baby-step
    rotation of every input, every nonzero giant-step rotation of every
    output); per token it falls as m grows for the BERT-large products."""
    slots = 32768
    for d, d_out in ((1024, 3072), (1024, 4096), (4096, 1024), (768, 2304)):
        per_token = []
        for m in (32, 64, 128, 256):
            k = slots // m
            nX, nY = -(-d // k), -(-d_out // k)
            cands = bt.cp_b1_candidates(m, d, d_out, slots)
            assert cands == sorted(cands) and all(k % b == 0 and b < k for b in cands)
            best = min(range(1, k.bit_length()), key=lambda i: bt.cp_rotation_count(m, d, d_out, slots, 1 << i))
            assert (1 << best) in cands
            for b1 in cands:
                G = k // b1
                direct = sum(1 for _ in range(nX) for b in range(b1) if b) + \
                    sum(1 for _ in range(nY) for g in range(G) if g)
                assert bt.cp_rotation_count(m, d, d_out, slots, b1) == direct
                assert set(bt.cp_rotations(m, k, b1)) == {b * m for b in range(1, b1)} | {g * b1 * m for g in range(1, G)}
            per_token.append(min(bt.cp_rotation_count(m, d, d_out, slots, b) for b in cands) / m)
        assert all(a > b for a, b in zip(per_token, per_token[1:])), per_token
