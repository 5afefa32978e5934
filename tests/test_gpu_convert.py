"""GPU local steps of the CKKS <-> MPC conversions (Alg. 1 steps 3-4, Alg. 2,
App. C.3) against the oracle, element by element: the simulated wrap-bit
shares, the decoding of shares (C2M) and the encoding of shares with ring to
field (M2C), at N = 2^12 (two CTA tiles per FFT pass) and N = 2^15 (the
BERT-base matmul_cp parameters), batched, with ragged slot counts, host and
device buffers, and the whole protocol: masking -> decryption -> C2M, then
M2C -> encryption -> addition."""
import numpy as np
import pytest

import oracle
from paper_2508_19525_b300 import workloads as wl

from _helpers import make_ctx, make_oracle

pytestmark = pytest.mark.gpu
L_MPC, SF = 43, 13
SEED = 0xC0417


def signed(v, bits):
    v %= 1 << bits
    return v - (1 << bits) if v >> (bits - 1) else v


def split_mod(rng, vals, q):
    t0 = rng.integers(0, q, len(vals), dtype=np.uint64)
    t1 = np.array([(int(v) - int(a)) % q for v, a in zip(vals, t0)], np.uint64)
    return t0, t1


@pytest.fixture(scope="module", params=["small", "bert"])
def setup(request):
    prm = wl.SMALL if request.param == "small" else wl.BERT_CP
    return prm, make_oracle(prm), make_ctx(prm)


def c2m_inputs(o, rng, count, scale):
    N, q = o.N, o.primes[0]
    T0, T1 = [], []
    for k in range(count):
        z = rng.uniform(-6, 6, N // 2)
        m = o.encode_int(z, scale)
        t0, t1 = split_mod(rng, [int(v) % q for v in m], q)
        T0.append(t0)
        T1.append(t1)
    return np.stack(T0), np.stack(T1)


def test_wrap_sims_match_oracle(setup):
    prm, o, ctx = setup
    N, q = o.N, o.primes[0]
    rng = np.random.default_rng(1)
    t0 = rng.integers(0, q, (2, N), dtype=np.uint64)
    t1 = rng.integers(0, q, (2, N), dtype=np.uint64)
    w0, w1 = ctx.f2r_wrap_sim(t0, t1, SEED, [5, 9])
    for k, nonce in enumerate((5, 9)):
        r0, r1 = oracle.f2r_wrap_sim(q, t0[k], t1[k], SEED, nonce)
        assert np.array_equal(w0[k], r0) and np.array_equal(w1[k], r1)
    n = N // 2 - 3
    x0 = rng.integers(0, 1 << L_MPC, (3, n), dtype=np.uint64)
    x1 = rng.integers(0, 1 << L_MPC, (3, n), dtype=np.uint64)
    v0, v1 = ctx.ext_wrap_sim(x0, x1, n, L_MPC, SEED, [1, 2, 3])
    for k in range(3):
        r0, r1 = oracle.ext_wrap_sim(L_MPC, x0[k], x1[k], SEED, k + 1)
        assert np.array_equal(v0[k], r0) and np.array_equal(v1[k], r1)


@pytest.mark.parametrize("scale", [2.0**40, 2.0**40 * 1.37])
def test_c2m_local_parity(setup, scale):
    prm, o, ctx = setup
    rng = np.random.default_rng(int(scale) % 1000)
    count = 3
    T0, T1 = c2m_inputs(o, rng, count, scale)
    W0, W1 = ctx.f2r_wrap_sim(T0, T1, SEED, list(range(count)))
    outs = [ctx.c2m_local(b, T, W, scale, L_MPC, SF) for b, T, W in ((0, T0, W0), (1, T1, W1))]
    for k in range(count):
        for b, T, W in ((0, T0, W0), (1, T1, W1)):
            ref = o.c2m_local(b, T[k], W[k], scale, L_MPC, SF)
            assert np.array_equal(outs[b][k], ref), (k, b)
    # the reconstruction is the decoding within one unit of 2^-sf
    q = o.primes[0]
    m = o.centered(((T0[0].astype(object) + T1[0].astype(object)) % q).astype(np.uint64))
    x = np.array([signed(int(a) + int(b), L_MPC) for a, b in zip(outs[0][0], outs[1][0])]) / 2**SF
    assert np.abs(x - o.decode(m, scale)).max() < 2.0**-SF + 2.0**-17


@pytest.mark.parametrize("ragged", [0, 7])
def test_m2c_local_parity(setup, ragged):
    prm, o, ctx = setup
    s = o.N // 2
    n = s - ragged
    count = 2
    level = o.nQ - 1 - (ragged % 2)
    rng = np.random.default_rng(n)
    xi = np.round(rng.uniform(-8, 8, (count, n)) * 2**SF).astype(np.int64)
    X0 = rng.integers(0, 1 << L_MPC, (count, n), dtype=np.uint64)
    X1 = np.array([[(int(v) - int(a)) % (1 << L_MPC) for v, a in zip(xi[k], X0[k])] for k in range(count)],
                  np.uint64)
    W0, W1 = ctx.ext_wrap_sim(X0, X1, n, L_MPC, SEED, [7, 8])
    for scale in (prm.scale, prm.scale * 1.37):
        outs = [ctx.m2c_local(b, X, W, n, level, scale, L_MPC, SF) for b, X, W in ((0, X0, W0), (1, X1, W1))]
        for k in range(count):
            for b, X, W in ((0, X0, W0), (1, X1, W1)):
                ref = o.m2c_local(b, X[k], W[k], level, scale, L_MPC, SF)
                assert np.array_equal(outs[b][k], ref), (k, b, scale)


def test_device_buffers_and_empty_inputs(setup):
    import torch
    prm, o, ctx = setup
    N, q = o.N, o.primes[0]
    rng = np.random.default_rng(3)
    T0, T1 = c2m_inputs(o, rng, 2, prm.scale)
    W0h, W1h = ctx.f2r_wrap_sim(T0, T1, SEED, [1, 2])
    dev = lambda a: torch.from_numpy(a.view(np.int64)).cuda()
    T0d, T1d = dev(T0), dev(T1)
    W0d = torch.zeros((2, N, 2), dtype=torch.int64, device="cuda")
    W1d = torch.zeros_like(W0d)
    ctx.f2r_wrap_sim(T0d, T1d, SEED, [1, 2], W0d, W1d)
    out_d = torch.zeros((2, N // 2), dtype=torch.int64, device="cuda")
    ctx.c2m_local(0, T0d, W0d, prm.scale, L_MPC, SF, out=out_d)
    ctx.sync()
    assert np.array_equal(W0d.cpu().numpy().view(np.uint64), W0h)
    assert np.array_equal(out_d.cpu().numpy().view(np.uint64), ctx.c2m_local(0, T0, W0h, prm.scale, L_MPC, SF))
    # no slots: both parties encode zero, exactly
    z = ctx.m2c_local(0, np.zeros(0, np.uint64), np.zeros((0, 2), np.uint64), 0, 1, prm.scale, L_MPC, SF)
    assert not z.any()
    # argument errors are refused before any launch
    from paper_2508_19525_b300.blb import BlbError
    with pytest.raises(BlbError):
        ctx.c2m_local(0, T0, W0h, prm.scale, 70, SF)
    with pytest.raises(BlbError):
        ctx.c2m_local(2, T0, W0h, prm.scale, L_MPC, SF)
    misaligned = torch.zeros(2 * N * 2 + 1, dtype=torch.int64, device="cuda")[1:]
    with pytest.raises(BlbError):
        ctx.c2m_local(0, T0d, misaligned, prm.scale, L_MPC, SF)


def test_protocol_round_trip_matches_oracle():
    """Alg. 1 then Alg. 2 on the GPU, every intermediate equal to the oracle's."""
    prm = wl.SMALL
    o, ctx = make_oracle(prm), make_ctx(prm)
    N, s, q = o.N, o.N // 2, o.primes[0]
    level = o.nQ - 1
    keys = ctx.keygen(SEED, [])
    sk = o.keygen_secret(SEED)
    rng = np.random.default_rng(4)
    Z = rng.uniform(-5, 5, (2, s))
    cts = ctx.encrypt_batch(keys, ctx.encode_batch(Z, level), [11, 12])
    masked, p1 = ctx.he2mpc_batch(keys, cts, [21, 22])
    p0 = ctx.decrypt_batch(keys, masked)[0][:, 0, :]
    W0, W1 = ctx.f2r_wrap_sim(p0, p1, SEED, [31, 32])
    y0 = ctx.c2m_local(0, p0, W0, prm.scale, L_MPC, SF)
    y1 = ctx.c2m_local(1, p1, W1, prm.scale, L_MPC, SF)
    lv = 2
    V0, V1 = ctx.ext_wrap_sim(y0, y1, s, L_MPC, SEED, [41, 42])
    m0 = ctx.m2c_local(0, y0, V0, s, lv, prm.scale, L_MPC, SF)
    m1 = ctx.m2c_local(1, y1, V1, s, lv, prm.scale, L_MPC, SF)
    outs = []
    for k in range(2):
        ct0 = ctx.encrypt(keys, ctx.pt_import(m0[k], lv), 51 + k)     # P0 encrypts its share
        outs.append(ctx.add_plain(ct0, ctx.pt_import(m1[k], lv)))    # P1 adds its own
    for k in range(2):
        # the same chain on the oracle
        ct = o.encrypt(sk, o.encode(Z[k], level, prm.scale), SEED, 11 + k)
        mk, sh = o.he2mpc(ct, SEED, 21 + k)
        d0 = o.decrypt(sk, mk)[0]
        assert np.array_equal(d0, p0[k]) and np.array_equal(sh, p1[k])
        r0, r1 = oracle.f2r_wrap_sim(q, d0, sh, SEED, 31 + k)
        a0 = o.c2m_local(0, d0, r0, prm.scale, L_MPC, SF)
        a1 = o.c2m_local(1, sh, r1, prm.scale, L_MPC, SF)
        assert np.array_equal(a0, y0[k]) and np.array_equal(a1, y1[k])
        xi = np.array([signed(int(a) + int(b), L_MPC) for a, b in zip(a0, a1)])
        assert np.abs(xi / 2**SF - Z[k]).max() < 2.0**-SF + 2.0**-17
        v0, v1 = oracle.ext_wrap_sim(L_MPC, a0, a1, SEED, 41 + k)
        e0 = o.m2c_local(0, a0, v0, lv, prm.scale, L_MPC, SF)
        e1 = o.m2c_local(1, a1, v1, lv, prm.scale, L_MPC, SF)
        assert np.array_equal(e0, m0[k]) and np.array_equal(e1, m1[k])
        ref = o.encrypt(sk, e0, SEED, 51 + k)
        for i in range(lv + 1):
            ref[0, i] = (ref[0, i].astype(object) + e1[i].astype(object)) % o.primes[i]
        assert np.array_equal(ctx.ct_export(outs[k]), ref)
        dec = ctx.decrypt(keys, outs[k], coeffs=False)[1]
        assert np.abs(dec - xi / 2**SF).max() < 2.0**-17
