"""GPU rotate-and-sum packing (Sec. 4.2.1) and the LayerNorm head (Alg.
LayerNorm lines 1-6) against the oracle limb for limb at N = 2^12 (batched
over ciphertexts and sequences), and at the BERT-base shape (N = 2^15,
L = 128 tokens, D = 768 in 6 ciphertexts of 128 columns) against numpy's row
means and variances."""
import numpy as np
import pytest

import oracle
from paper_2508_19525_b300 import workloads as wl

from _helpers import make_ctx, make_oracle

pytestmark = pytest.mark.gpu
SEED = 0x5A5B


def blocks(z, L):
    return z.reshape(-1, L)


@pytest.mark.parametrize("L,D,direction,mask", [(32, 64, 0, True), (32, 64, 0, False), (16, 4, 1, False),
                                                (64, 32, 0, True), (32, 1, 0, False)])
def test_rotate_sum_parity(L, D, direction, mask):
    prm = wl.SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    s = o.N // 2
    rots = [(-1 if direction else 1) * (L << i) for i in range(int(np.log2(D)))]
    keys = ctx.keygen(SEED, rots)
    sk = o.keygen_secret(SEED)
    gks = [o.keygen_galois(SEED, sk, o.galois_elt(r)) for r in rots]
    rng = np.random.default_rng(L * D + direction)
    level = o.nQ - 1
    Z = rng.uniform(-1, 1, (3, s))
    if direction:
        Z[:, L:] = 0.0
    cts = [ctx.encrypt(keys, ctx.encode(z, level), 20 + i) for i, z in enumerate(Z)]
    out = ctx.rotate_sum_packing(keys, cts, L, D, direction, mask)
    assert len(out) == 3
    for i, z in enumerate(Z):
        ref = o.rs_packing(o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 20 + i), L, D, direction, mask, gks)
        assert np.array_equal(ctx.ct_export(out[i]), ref), i
    got = blocks(ctx.decrypt(keys, out[0], coeffs=False)[1], L)
    b = blocks(Z[0], L)
    k = s // L
    if direction == 0:
        want = np.stack([sum(b[(j + t) % k] for t in range(D)) for j in range(k)])
        if mask:
            want[1:] = 0.0
    else:
        want = np.stack([sum(b[(j - t) % k] for t in range(D)) for j in range(k)])
    assert np.abs(got - want).max() < 1e-4


def layernorm_cts(ctx, keys, X, L, k, level, nonce):
    L_, D = X.shape
    nc = -(-D // k)
    Z = np.zeros((nc, ctx.N // 2))
    for c in range(nc):
        for b in range(k):
            col = c * k + b
            if col < D:
                Z[c, b * L:(b + 1) * L] = X[:, col]
    return ctx.encrypt_batch(keys, ctx.encode_batch(Z, level), [nonce + c for c in range(nc)]), Z


def test_layernorm_head_parity():
    prm = wl.SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    s, L, D = o.N // 2, 32, 96
    k = s // L
    nc = -(-D // k)
    rots = [L << i for i in range(int(np.log2(k)))]
    keys = ctx.keygen(SEED, rots, relin=True)
    sk = o.keygen_secret(SEED)
    gks = [o.keygen_galois(SEED, sk, o.galois_elt(r)) for r in rots]
    rk = o.keygen_relin(SEED, sk)
    level = o.nQ - 1
    rng = np.random.default_rng(5)
    Xs = [rng.uniform(-1, 1, (L, D)) + rng.uniform(-0.5, 0.5, (L, 1)) for _ in range(2)]
    cts, Zs = [], []
    for j, X in enumerate(Xs):
        c, Z = layernorm_cts(ctx, keys, X, L, k, level, 100 * j)
        cts += c
        Zs.append(Z)
    X_mu, var = ctx.layernorm_head(keys, cts, L, D, nc)
    assert len(X_mu) == 2 * nc and len(var) == 2
    for j in range(2):
        ref_in = np.stack([o.encrypt(sk, o.encode(Zs[j][c], level, prm.scale), SEED, 100 * j + c) for c in range(nc)])
        rx, rv = o.layernorm_head(ref_in, L, D, gks, rk)
        for c in range(nc):
            assert np.array_equal(ctx.ct_export(X_mu[j * nc + c]), rx[c]), (j, c)
        assert np.array_equal(ctx.ct_export(var[j]), rv), j


def test_bert_base_layernorm_head():
    prm = wl.BERT_CP
    ctx = make_ctx(prm)
    s, L, D = ctx.N // 2, 128, 768
    k = s // L
    nc = D // k
    rots = [L << i for i in range(int(np.log2(k)))]
    keys = ctx.keygen(SEED, rots, relin=True)
    level = ctx.nQ - 1
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, (L, D)) + rng.uniform(-0.5, 0.5, (L, 1))
    cts, _ = layernorm_cts(ctx, keys, X, L, k, level, 0)
    X_mu, var = ctx.layernorm_head(keys, cts, L, D, nc)
    mean = X.mean(axis=1, keepdims=True)
    for c in range(nc):
        got = blocks(ctx.decrypt(keys, X_mu[c], coeffs=False)[1], L)
        assert np.abs(got - (X[:, c * k:(c + 1) * k] - mean).T).max() < 1e-4
    v = blocks(ctx.decrypt(keys, var[0], coeffs=False)[1], L)
    assert np.abs(v - X.var(axis=1)[None, :]).max() < 1e-4
