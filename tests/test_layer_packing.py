"""Block 1 of the hybrid layer as one HE block (Sec. 5.1, multi-head packing):
with W_Q and W_K's columns in the head-packed order, the spatial-first output
ciphertexts of the QKV product are exactly matmul_cc's head-packed operands
(Q as spatial-first A, K^T as reduce-first B), at the test shape and at
BERT-base (12 heads as groups of 8 and 4)."""
import numpy as np
import pytest

from paper_2508_19525_b300 import layer as ly


@pytest.mark.parametrize("L,d,H,Dh,groups,s", [(32, 128, 8, 16, (8,), 2048), (128, 768, 12, 64, (8, 4), 16384)])
def test_reordered_weights_give_the_head_packing(L, d, H, Dh, groups, s):
    k = s // L
    rng = np.random.default_rng(1)
    X, Wq, Wk = rng.uniform(-1, 1, (L, d)), rng.uniform(-1, 1, (d, d)), rng.uniform(-1, 1, (d, d))
    perm = ly.head_permutation(groups, Dh, k)
    assert sorted(perm) == list(range(d))
    Zq, Zk = ly.pack_columns(X @ Wq[:, perm], L, k), ly.pack_columns(X @ Wk[:, perm], L, k)
    Qh = (X @ Wq).reshape(L, H, Dh).transpose(1, 0, 2)
    Kh = (X @ Wk).reshape(L, H, Dh).transpose(1, 0, 2)
    e0 = h0 = 0
    for Hg in groups:
        Kc = k // Hg
        n_c = Dh // Kc
        assert np.array_equal(Zq[e0:e0 + n_c], ly.pack_heads(Qh[h0:h0 + Hg], L, Hg, Kc, n_c, rows=False))
        assert np.array_equal(Zk[e0:e0 + n_c], ly.pack_heads(Kh[h0:h0 + Hg].transpose(0, 2, 1), L, Hg, Kc, n_c,
                                                             rows=True))
        e0 += n_c
        h0 += Hg
    assert e0 * k == d
