"""Pins for the oracle's rotate-and-sum packing (Sec. 4.2.1) and the HE steps
of the secure LayerNorm before rsqrt (Alg. LayerNorm lines 1-6): decrypted
results against block sums, broadcasts, row means and row variances computed
by numpy in FP64, at N = 2^12 with spatial-first packing (block b of a
ciphertext = slots [b L, (b+1) L))."""
import numpy as np
import pytest

import oracle
from paper_2508_19525_b300 import workloads as wl

SEED = 0x5A5A


@pytest.fixture(scope="module")
def env():
    prm = wl.SMALL
    o = oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum)
    sk = o.keygen_secret(SEED)
    return prm, o, sk


def keys_for(o, sk, rots):
    return [o.keygen_galois(SEED, sk, o.galois_elt(r)) for r in rots]


def dec(o, sk, ct, scale):
    return o.decode(o.centered(o.decrypt(sk, ct)[0]), scale)


def blocks(z, L):
    return z.reshape(-1, L)


@pytest.mark.parametrize("L,D", [(32, 64), (16, 8), (64, 2)])
def test_sum_with_mask(env, L, D):
    prm, o, sk = env
    s = o.N // 2
    k = s // L
    rng = np.random.default_rng(L + D)
    z = np.zeros(s)
    z[:L * D] = rng.uniform(-1, 1, L * D)       # D blocks of data, the rest zero
    level = o.nQ - 1
    ct = o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 1)
    out = o.rs_packing(ct, L, D, 0, True, keys_for(o, sk, [L << i for i in range(int(np.log2(D)))]))
    assert out.shape[1] == level                 # one rescale
    got = blocks(dec(o, sk, out, prm.scale), L)
    ref = blocks(z, L)[:D].sum(axis=0)
    assert np.abs(got[0] - ref).max() < 1e-4
    assert np.abs(got[1:]).max() < 1e-4          # the mask clears every other block
    assert k >= D


def test_sum_without_mask_leaves_the_total_in_every_block(env):
    prm, o, sk = env
    s, L = o.N // 2, 32
    k = s // L
    rng = np.random.default_rng(2)
    z = rng.uniform(-1, 1, s)
    level = o.nQ - 1
    ct = o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 2)
    out = o.rs_packing(ct, L, k, 0, False, keys_for(o, sk, [L << i for i in range(int(np.log2(k)))]))
    got = blocks(dec(o, sk, out, prm.scale), L)
    total = blocks(z, L).sum(axis=0)
    assert np.abs(got - total[None, :]).max() < 1e-4


@pytest.mark.parametrize("D", [4, 64])
def test_broadcast(env, D):
    prm, o, sk = env
    s, L = o.N // 2, 32
    rng = np.random.default_rng(D)
    z = np.zeros(s)
    z[:L] = rng.uniform(-1, 1, L)
    level = o.nQ - 1
    ct = o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 3)
    out = o.rs_packing(ct, L, D, 1, False, keys_for(o, sk, [-(L << i) for i in range(int(np.log2(D)))]))
    got = blocks(dec(o, sk, out, prm.scale), L)
    assert np.abs(got[:D] - z[:L][None, :]).max() < 1e-4
    assert np.abs(got[D:]).max(initial=0) < 1e-4   # blocks past D stay empty


def test_rs_packing_rejects_bad_shapes(env):
    prm, o, sk = env
    ct = np.zeros((2, o.nQ, o.N), np.uint64)
    with pytest.raises(ValueError):
        o.rs_packing(ct, 32, 3, 0, False, [])      # D not a power of two
    with pytest.raises(ValueError):
        o.rs_packing(ct, 32, 4, 1, True, [ct, ct])  # the mask belongs to the sum


def layernorm_inputs(o, sk, prm, L, D, seed):
    s = o.N // 2
    k = s // L
    nc = -(-D // k)
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (L, D)) + rng.uniform(-0.5, 0.5, (L, 1))
    level = o.nQ - 1
    cts = []
    for c in range(nc):
        z = np.zeros(s)
        for b in range(k):
            col = c * k + b
            if col < D:
                z[b * L:(b + 1) * L] = X[:, col]
        cts.append(o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 10 + c))
    return X, np.stack(cts), k, nc


@pytest.mark.parametrize("L,D", [(32, 96), (64, 32)])
def test_layernorm_head(env, L, D):
    prm, o, sk = env
    X, cts, k, nc = layernorm_inputs(o, sk, prm, L, D, seed=L + D)
    gks = keys_for(o, sk, [L << i for i in range(int(np.log2(k)))])
    X_mu, var = o.layernorm_head(cts, L, D, gks, o.keygen_relin(SEED, sk))
    level = o.nQ - 1
    assert X_mu.shape == (nc, 2, level, o.N) and var.shape == (2, level - 2, o.N)
    mean = X.mean(axis=1, keepdims=True)
    for c in range(nc):
        got = blocks(dec(o, sk, X_mu[c], prm.scale), L)
        for b in range(k):
            col = c * k + b
            ref = X[:, col] - mean[:, 0] if col < D else -mean[:, 0]
            assert np.abs(got[b] - ref).max() < 1e-4, (c, b)
    scale_var = prm.scale * prm.scale / o.primes[level - 1]
    v = blocks(dec(o, sk, var, scale_var), L)
    # zero-padded columns of the last ciphertext contribute mean^2 each to the sum
    pad = nc * k - D
    ref_var = (((X - mean) ** 2).sum(axis=1) + pad * mean[:, 0] ** 2) / D
    assert np.abs(v - ref_var[None, :]).max() < 1e-4
