"""Host logic of the token-chunked batching (uneven-length sequences cut into
m-row chunks for matmul_cp): layout and spatial-first packing round trips."""
import numpy as np

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
