"""Rotation and ct-ct multiplication counts of the matmul_cc schedule at the
paper's shapes (Table complexity_compare: BERT-large, s = 16384 slots, 16 heads
of dimension 64 at 128 tokens; Table exp_micro: the same and GPT2-base, 12
heads at 64 tokens, as head groups of 8 and 4).

The schedule runs on plaintext slot vectors at those exact sizes (every
rotation is counted by the simulator), must reproduce every head's product,
and its counts must equal the closed form the oracle implements.  The
ct-ct multiplication counts equal the paper's (1024 and 2048 at BERT-large);
the rotation counts are below the paper's printed ones (640, 1056, 488): the
paper gives totals without a breakdown, and this reading hoists nothing into
the count but folds step 2's giant-step rotations into step 3's one rotation
per diagonal (App. C.1)."""
import numpy as np
import pytest

import cc_schedule as cs
import oracle

PAPER = {"bert_large_qk": (640, 1024), "bert_large_sv": (1056, 2048), "gpt2_qk": (488, None), "gpt2_sv": (488, None)}


def _best_split(n_c, L, Kc):
    lib = oracle.lib()
    return min((lib.orc_cc_num_rotations(n_c, L, Kc, b1, b2), b1, b2)
               for b1 in range(1, Kc + 1) if Kc % b1 == 0 for b2 in range(1, L + 1) if L % b2 == 0)


@pytest.mark.parametrize("name,L,groups,R", [
    ("bert_large_qk", 128, (16,), 64),
    ("bert_large_sv", 128, (16,), 128),
    ("gpt2_qk", 64, (8, 4), 64),
    ("gpt2_sv", 64, (8, 4), 64),
])
def test_counts_at_the_papers_shapes(name, L, groups, R):
    s = 16384
    rng = np.random.default_rng(L + R)
    rot_total = mult_total = 0
    for Hg in groups:
        Kc = s // (L * Hg)
        n_c = -(-R // Kc)
        nrot, b1s1, b1s2 = _best_split(n_c, L, Kc)
        A = rng.uniform(-1, 1, size=(Hg, L, R))
        B = rng.uniform(-1, 1, size=(Hg, R, L))
        C, sim_rot = cs.simulate(cs.pack(A, L, Hg, Kc, n_c, rows=False), cs.pack(B, L, Hg, Kc, n_c, rows=True),
                                 L, Hg, b1s1, b1s2)
        assert np.abs(cs.unpack_diagonals(C, L, Hg, Kc) - np.einsum("hik,hkj->hij", A, B)).max() < 1e-10
        assert sim_rot == nrot
        rot_total += nrot
        mult_total += n_c * L  # step 2: one tensor product per (input ciphertext, diagonal)
    paper_rot, paper_mult = PAPER[name]
    print(f"{name}: {rot_total} rotations (paper {paper_rot}), {mult_total} ct-ct products (paper {paper_mult})")
    assert rot_total <= paper_rot
    if paper_mult is not None:
        assert mult_total == paper_mult
