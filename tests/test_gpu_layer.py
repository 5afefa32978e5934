"""The hybrid encoder layer (five fused HE blocks with CKKS <-> MPC conversions
at every boundary, MPC simulated) against the FP64 layer with the same
approximations, at a reduced shape; and the HE part of the softmax-exponential
block (sub, scalar multiply with an aligned scale, constant add, six
squarings) limb for limb against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2508_19525_b300 import layer as ly
from paper_2508_19525_b300 import workloads as wl

from _helpers import make_ctx, make_oracle

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
    assert np.abs(Y - ref).max() < 3e-2, np.abs(Y - ref).max()
    assert set(he) == set(conv) and len(he) == 7


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
