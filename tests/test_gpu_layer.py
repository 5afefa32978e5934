"""The hybrid encoder layer (five fused HE blocks with CKKS <-> MPC conversions
at every boundary, MPC simulated) against the FP64 layer with the same
approximations, at a reduced shape; block 1 (QKV with head-packed W_Q / W_K
columns, then Q K^T on its output ciphertexts) and the HE part of the
softmax-exponential block (sub, scalar multiply with an aligned scale,
constant add, six squarings) limb for limb against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2508_19525_b300 import layer as ly
from paper_2508_19525_b300 import workloads as wl

from _helpers import assert_limbs_consistent, make_ctx, make_oracle

pytestmark = pytest.mark.gpu
SEED = 0x1A7E
P_SMALL = wl.HEParams(12, (60,) + (40,) * 7, (60,) * 3, 3)
P_BIG = wl.HEParams(13, (60,) + (40,) * 11, (60,) * 3, 4)


def test_layer_matches_fp64():
    ctx, big = make_ctx(P_SMALL), make_ctx(P_BIG)
    lay = ly.BertLayer(ctx, big, L=32, d=128, H=8, Dh=16, f=256, groups=(8,), seed=3, b1=8)
    rs, rb = lay.rotations()
    keys, keysb = ctx.keygen(SEED, rs, relin=True), big.keygen(SEED + 1, rb, relin=True)
    X = np.random.default_rng(5).uniform(-1, 1, (32, 128))
    Y, he, conv = lay.forward(X, keys, keysb, ly.Mpc(9))
    ref = lay.reference(X)
    assert Y.shape == ref.shape
    # every value crosses six CKKS <-> MPC boundaries as 2^-13 fixed point
    # (half a unit, 6.1e-5, per rounding), and the LayerNorm tails divide by
    # sigma (about 0.5 here); 2e-3 = 16 units of 2^-13 (measured: 5.8e-4)
    assert np.abs(Y - ref).max() < 2e-3, np.abs(Y - ref).max()
    assert set(he) == set(conv) and len(he) == 6


def test_exp_block_parity_with_oracle():
    prm = P_SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    keys = ctx.keygen(SEED, [], relin=True)
    sk = o.keygen_secret(SEED)
    rk = o.keygen_relin(SEED, sk)
    level = o.nQ - 1
    rng = np.random.default_rng(2)
    s_, m_ = rng.uniform(-6, 0, o.N // 2), np.zeros(o.N // 2)
    cs = [ctx.encrypt(keys, ctx.encode(v, level), 10 + i) for i, v in enumerate((s_, m_))]
    os_ = [o.encrypt(sk, o.encode(v, level, prm.scale), SEED, 10 + i) for i, v in enumerate((s_, m_))]
    # GPU
    x = ctx.mul_const(ctx.sub(cs[0], cs[1]), 1.0 / 64.0)
    x = ctx.add_plain(x, ctx.encode(np.ones(o.N // 2), x.level, x.scale))
    for _ in range(6):
        x = ctx.rescale(ctx.mul(keys, x, x))
    # oracle, the same steps
    d = (os_[0].astype(object) - os_[1].astype(object))
    for i in range(level + 1):
        d[:, i] %= o.primes[i]
    d = d.astype(np.uint64)
    sc = prm.scale
    s_c = sc * o.primes[level] / sc
    y = o.rescale(o.mul_plain(d, o.encode(np.full(o.N // 2, 1.0 / 64.0), level, s_c)))
    lv = level - 1
    one = o.encode(np.ones(o.N // 2), lv, sc)
    y[0] = (y[0].astype(object) + one.astype(object)) % np.array(o.primes[:lv + 1], dtype=object)[:, None]
    y = y.astype(np.uint64)
    for _ in range(6):
        y = o.rescale(o.relinearize(o.tensor(y, y), rk))
    assert np.array_equal(ctx.ct_export(x), y)
    got = ctx.decrypt(keys, x, coeffs=False)[1]
    assert np.abs(got - (1 + s_ / 64) ** 64).max() < 1e-4


def test_block1_parity_with_oracle():
    """QKV (matmul_cp with the reordered W_Q / W_K columns) and Q K^T
    (matmul_cc on the QKV output ciphertexts) as one HE block: every output
    limb equals the oracle's run of the same two products, and the scores
    decrypt to the FP64 Q K^T within 1e-4."""
    ctx, big = make_ctx(P_SMALL), make_ctx(P_BIG)
    lay = ly.BertLayer(ctx, big, L=32, d=128, H=8, Dh=16, f=256, groups=(8,), seed=3, b1=8)
    L, d, k, top = lay.L, lay.d, lay.k, lay.top
    rs, _ = lay.rotations()
    keys = ctx.keygen(SEED, rs, relin=True)
    X = np.random.default_rng(6).uniform(-1, 1, (L, d))
    Z = ly.pack_columns(X, L, k)
    Xc = [ctx.encrypt(keys, ctx.encode(z, top), 40 + c) for c, z in enumerate(Z)]
    Y, Cs = lay.he_block1(keys, Xc)
    o = make_oracle(P_SMALL)
    sk = o.keygen_secret(SEED)
    Xo = np.stack([o.encrypt(sk, o.encode(z, top, P_SMALL.scale), SEED, 40 + c) for c, z in enumerate(Z)])
    gal = {o.galois_elt(r): o.keygen_galois(SEED, sk, o.galois_elt(r)) for r in rs}
    info = lay.p_qkv.info()
    Yo = o.matmul_cp(Xo, L, d, lay.Wqkv_he, 3 * d, info["b1"], gal)
    assert len(Y) == len(Yo)
    for e, y in enumerate(Y):
        assert np.array_equal(ctx.ct_export(y), Yo[e]), e
    nq, e0, h0 = d // k, 0, 0
    Q = (X @ lay.Wqkv[:, :d]).reshape(L, lay.H, lay.Dh).transpose(1, 0, 2)
    K = (X @ lay.Wqkv[:, d:2 * d]).reshape(L, lay.H, lay.Dh).transpose(1, 0, 2)
    for Hg, C in zip(lay.groups, Cs):
        ci = lay.cc_qk[Hg].info()
        n_c = ci["n_c"]
        Co = o.matmul_cc(Yo[e0:e0 + n_c], Yo[nq + e0:nq + e0 + n_c], L, Hg, ci["b1s1"], ci["b1s2"], gal,
                         o.keygen_relin(SEED, sk))
        assert len(C) == Co.shape[0]
        zs = []
        for j, c in enumerate(C):
            assert np.array_equal(ctx.ct_export(c), Co[j]), (Hg, j)
            coeffs, z = ctx.decrypt(keys, c)
            assert_limbs_consistent(coeffs, ctx.primes)
            zs.append(z)
        S = ly.unpack_diagonals(np.stack(zs), L, Hg, ci["Kc"])
        ref = np.einsum("hik,hjk->hij", Q[h0:h0 + Hg], K[h0:h0 + Hg])
        assert np.abs(S - ref).max() <= 1e-4
        e0 += n_c
        h0 += Hg
