"""Pins for the oracle's protocols: matmul_cp (diagonal method + BSGS, App. C.1)
against the FP64 matrix product, and the CKKS-to-MPC masking of Alg. 1 against
exact share reconstruction and uniformity (Thm. 1), with MP2ML's encoded mask
(Sec. 6.2, Fig. 4) as the negative case."""
import numpy as np
import pytest

import oracle
from paper_2508_19525_b300 import workloads as wl


def make(prm):
    return oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum)


def pack_cols(X, m, k, n_cts):
    """Spatial-first packing (Sec. 4.2.1): ct c holds X[i, c k + b] at slot i + m b."""
    out = []
    d = X.shape[1]
    for c in range(n_cts):
        z = np.zeros(m * k)
        for b in range(k):
            col = c * k + b
            if col < d:
                z[b * m:(b + 1) * m] = X[:, col]
        out.append(z)
    return out


def unpack_cols(zs, m, k, d_out):
    Y = np.zeros((m, d_out))
    for e, z in enumerate(zs):
        for b in range(k):
            col = e * k + b
            if col < d_out:
                Y[:, col] = z[b * m:(b + 1) * m]
    return Y


def cp_keys(o, s, seed, m, b1, G):
    rots = [b * m for b in range(1, b1)] + [g * b1 * m for g in range(1, G)]
    return {o.galois_elt(r): o.keygen_galois(seed, s, o.galois_elt(r)) for r in rots}


@pytest.mark.parametrize("case", [
    # (params, m, d, d_out, b1): cfg-1 shape, multi-ct with a ragged tail
    (wl.TINY, 32, 64, 64, 8),
    (wl.SMALL, 64, 80, 40, 4),
])
def test_matmul_cp_decrypts_to_fp64_product(case):
    prm, m, d, d_out, b1 = case
    o = make(prm)
    s_ = o.N // 2
    k = s_ // m
    G = k // b1
    level = o.nQ - 1
    X, W = wl.cp_operands(m, d, d_out, seed=5)
    sk = o.keygen_secret(0)
    nX = (d + k - 1) // k
    cts = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), 0, c)
                    for c, z in enumerate(pack_cols(X, m, k, nX))])
    keys = cp_keys(o, sk, 0, m, b1, G)
    Y = o.matmul_cp(cts, m, d, W, d_out, b1, keys)
    nY = (d_out + k - 1) // k
    assert Y.shape == (nY, 2, level, o.N)
    zs = [o.decode(o.centered(o.decrypt(sk, y)[0]), prm.scale) for y in Y]
    got = unpack_cols(zs, m, k, d_out)
    ref = X @ W
    err = np.abs(got - ref)
    assert err.max() <= 1e-4
    assert np.mean(err ** 2) < 1e-11
    # unused slots (columns beyond d_out) decrypt to ~0
    if nY * k > d_out:
        last = zs[-1][(d_out - (nY - 1) * k) * m:]
        assert np.abs(last).max() < 1e-6


def test_matmul_cp_output_subset_matches_full():
    o = make(wl.TINY)
    m, d, d_out, b1 = 32, 64, 64, 8
    k = o.N // 2 // m
    X, W = wl.cp_operands(m, d, d_out, seed=9)
    sk = o.keygen_secret(1)
    cts = np.stack([o.encrypt(sk, o.encode(pack_cols(X, m, k, 1)[0], 2, 2.0 ** 40), 1, 0)])
    keys = cp_keys(o, sk, 1, m, b1, k // b1)
    full = o.matmul_cp(cts, m, d, W, d_out, b1, keys)
    sub = o.matmul_cp(cts, m, d, W, d_out, b1, keys, out_idx=[0])
    assert np.array_equal(full[0], sub[0])


def test_cp_rotation_count_formula():
    o = make(wl.TINY)
    # BERT-base QKV at N=2^15: 6 input cts, 18 outputs, b1=16, G=8 -> 216
    assert o.cp_num_rotations(6, 18, 16, 8) == 216
    assert o.cp_num_rotations(6, 6, 16, 8) == 132
    assert o.cp_num_rotations(1, 1, 8, 8) == 14


def test_matmul_cp_missing_key_is_an_error():
    o = make(wl.TINY)
    m = 32
    sk = o.keygen_secret(1)
    cts = np.stack([o.encrypt(sk, o.encode(np.zeros(4), 2, 2.0 ** 40), 1, 0)])
    with pytest.raises(ValueError):
        o.matmul_cp(cts, m, 64, np.zeros((64, 64)), 64, 8, {})


# --------------------------------------------------------------------------- he2mpc
def test_he2mpc_shares_reconstruct_exactly():
    o = make(wl.SMALL)
    sk = o.keygen_secret(4)
    z = wl.slot_vector(o.N // 2, seed=4)
    ct = o.encrypt(sk, o.encode(z, 4, 2.0 ** 40), 4, 3)
    masked, u1 = o.he2mpc(ct, seed=4, nonce=99)
    u0 = o.decrypt(sk, masked)[0]
    q0 = o.primes[0]
    unmasked = o.decrypt(sk, ct)[0]
    assert np.array_equal((u0.astype(object) + u1.astype(object)) % q0, unmasked.astype(object))
    # the mask is the MASK-purpose uniform draw
    r = oracle.sample_uniform(o.N, q0, 4, 99, oracle.MASK)
    assert np.array_equal(u1, (np.uint64(q0) - r) % np.uint64(q0))
    # decoded reconstruction is the message
    rec = o.centered((u0.astype(object) + u1.astype(object)) % q0)
    assert np.max(np.abs(o.decode(rec.astype(np.int64), 2.0 ** 40) - z)) < 1e-6


def test_he2mpc_client_share_is_uniform():
    """Thm. 1: P0's share Encode(x) + e + r mod q0 is uniform whatever x is."""
    o = make(wl.TINY)
    sk = o.keygen_secret(8)
    z = np.full(o.N // 2, 0.9)  # a message far from zero
    ct = o.encrypt(sk, o.encode(z, 2, 2.0 ** 40), 8, 0)
    q0 = o.primes[0]
    shares = []
    for nonce in range(16):
        masked, _ = o.he2mpc(ct, seed=8, nonce=nonce)
        shares.append(o.decrypt(sk, masked)[0])
    u = np.concatenate(shares).astype(np.float64) / q0
    nb = 64
    hist = np.bincount((u * nb).astype(int), minlength=nb)
    n = len(u)
    chi2 = np.sum((hist - n / nb) ** 2 / (n / nb))
    assert chi2 < 130  # 63 dof, p ~ 1e-6
    # and unmasked decryptions are not uniform at all
    dec = o.decrypt(sk, ct)[0].astype(np.float64) / q0
    assert np.mean((dec > 0.01) & (dec < 0.99)) < 0.01


def test_mp2ml_encoded_mask_is_concentrated():
    """Sec. 6.2 / Fig. 4 (N = 8192, q ~ 2^60): Encode(Delta^-1 r) for uniform
    r in Z_q^{N/2}.  Each non-constant coefficient is (2/N) Re sum_j r_j w_j
    with |w_j| = 1, so its standard deviation is q / sqrt(12 N) (closed form);
    practically all coefficients lie in +-q/sqrt(N), a 2/sqrt(N) ~ 2% sliver of
    Z_q, whereas a uniform residue has spread q/sqrt(12).  The mask therefore
    leaves the high bits of a message visible."""
    o = oracle.Oracle(13, (60,), (60,), 1)
    q = o.primes[0]
    N = o.N
    rng = np.random.default_rng(0)
    r = rng.integers(0, q, size=N // 2, dtype=np.uint64).astype(np.float64)
    delta = 2.0 ** 40
    coef = o.encode_int(r / delta, delta).astype(np.float64)
    assert abs(coef[0] - np.mean(r)) < q / np.sqrt(N)  # the constant term carries the mean of r
    c = coef[1:]
    assert abs(np.std(c) / (q / np.sqrt(12 * N)) - 1) < 0.03
    assert np.mean(np.abs(c) <= q / np.sqrt(N)) > 0.999
    # a uniform share would put only ~2/sqrt(N) of its mass in that band
    u = rng.integers(0, q, size=N, dtype=np.uint64).astype(np.float64)
    u = np.where(u > q / 2, u - q, u)
    assert np.mean(np.abs(u) <= q / np.sqrt(N)) < 0.05


def test_matmul_cp_phases_equal_the_one_call_product():
    """orc_matmul_cp's two phases (baby steps; outputs from pre-encoded
    plaintext diagonals) give the one-call product's limbs, for a subset of
    outputs in any order."""
    prm = wl.SMALL
    o = oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum)
    m, d, d_out, b1 = 64, 80, 100, 4
    k = o.N // 2 // m
    G, level = k // b1, o.nQ - 1
    sk = o.keygen_secret(4)
    rots = [b * m for b in range(1, b1)] + [g * b1 * m for g in range(1, G)]
    gal = {o.galois_elt(r): o.keygen_galois(4, sk, o.galois_elt(r)) for r in rots}
    X, W = wl.cp_operands(m, d, d_out, seed=8)
    nX = (d + k - 1) // k
    Z = np.zeros((nX, o.N // 2))
    for c in range(nX):
        for b in range(k):
            if c * k + b < d:
                Z[c, b * m:(b + 1) * m] = X[:, c * k + b]
    cts = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), 4, c) for c, z in enumerate(Z)])
    ref = o.matmul_cp(cts, m, d, W, d_out, b1, gal)
    baby = o.cp_baby_steps(cts, m, b1, gal)
    pts = o.cp_encode_diagonals(level, m, d, W, d_out, b1, [1, 0])
    Y = o.cp_outputs(baby, m, b1, pts, gal)
    assert np.array_equal(Y[0], ref[1]) and np.array_equal(Y[1], ref[0])
    # and the finest phases: one inner sum per giant step, then the giant-step
    # rotations summed with one ModDown, then the rescale
    T = [o.cp_inner_sum(baby, pts[0, g]) for g in range(G)]
    acc = o.rotate_sum(T[0], np.stack(T[1:]), [g * b1 * m for g in range(1, G)],
                       [gal[o.galois_elt(g * b1 * m)] for g in range(1, G)])
    assert np.array_equal(o.rescale(acc), ref[1])
