"""Pins for the oracle's local steps of the conversions between CKKS and additive
shares (Alg. 1 steps 3-4, Alg. 2, App. C.3), checked against what the
mathematics fixes rather than against the oracle's own formulas:

* probabilistic truncation: floor(m / 2^k) + u, u in {0, 1} with
  Pr[u = 1] = (m mod 2^k) / 2^k (the functionality App. C.3 states), and the
  overflow failure rate |m| / 2^128;
* field to ring, signed extension, ring to field: the two local results sum to
  the centered message exactly (brute force over random and edge-case shares);
* decoding of shares: the reconstruction lies within one unit of 2^-sf of the
  FP64 decoding (and of the O(N^2) definition at N = 32), unbiased on average;
* encoding of shares: the reconstructed coefficients are those of
  round(Delta pi^-1(x)) up to the fixed point's resolution, consistent across
  the primes of the level, and decode back to x;
* the whole protocol: encrypt -> mask -> decrypt -> F2R -> decode shares, then
  extend -> encode shares -> R2F -> encrypt + add -> decrypt.
"""
import numpy as np
import pytest

import oracle
from paper_2508_19525_b300 import workloads as wl

R = 1 << 128
L_MPC, SF = 43, 13  # the MPC ring width and fixed-point scale of Sec. 7.1


def signed(v, bits=128):
    v %= 1 << bits
    return v - (1 << bits) if v >> (bits - 1) else v


def words(vals):
    return oracle.u128_words(vals)


def split(rng, vals, mod):
    """Uniform additive shares of the integers vals mod `mod` (Python ints)."""
    s0 = [int.from_bytes(rng.bytes(16), "little") % mod for _ in vals]
    s1 = [(v - a) % mod for v, a in zip(vals, s0)]
    return s0, s1


def small_oracle():
    prm = wl.SMALL
    return oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum)


# ---- probabilistic truncation ------------------------------------------------
@pytest.mark.parametrize("k", [1, 13, 30, 57])
def test_truncation_is_floor_plus_a_bernoulli(k):
    rng = np.random.default_rng(k)
    ps = [int(v) for v in rng.integers(-2**62, 2**62, 300)] + [0, 1, -1, (1 << k) - 1, -(1 << k), 1 << k]
    ps += [signed(int.from_bytes(rng.bytes(12), "little"), 96) for _ in range(100)]
    s0, s1 = split(rng, ps, R)
    t0 = oracle.words_u128(oracle.share_trunc(0, words(s0), k))
    t1 = oracle.words_u128(oracle.share_trunc(1, words(s1), k))
    for p, a, b in zip(ps, t0, t1):
        u = signed(a + b) - (p >> k)          # p >> k is floor(p / 2^k)
        assert u in (0, 1), (p, u)


def test_truncation_rounding_probability():
    """Pr[u = 1] = (m mod 2^k) / 2^k: over many random splits of one m."""
    rng = np.random.default_rng(5)
    k, trials = 8, 4000
    for r in (0, 37, 128, 250):
        p = 12345 * (1 << k) + r
        s0, s1 = split(rng, [p] * trials, R)
        t0 = oracle.words_u128(oracle.share_trunc(0, words(s0), k))
        t1 = oracle.words_u128(oracle.share_trunc(1, words(s1), k))
        u = np.array([signed(a + b) - (p >> k) for a, b in zip(t0, t1)])
        assert set(np.unique(u)) <= {0, 1}
        f, pr = u.mean(), r / (1 << k)
        assert abs(f - pr) <= 5 * np.sqrt(pr * (1 - pr) / trials) + 1e-9, (r, f, pr)


def test_truncation_failure_rate_is_m_over_ring():
    """The shares overflow (and the result is off by about 2^(128-k)) with
    probability |m| / 2^128: 1/4 for |m| = 2^126."""
    rng = np.random.default_rng(6)
    k, trials = 20, 4000
    for p in (1 << 126, -(1 << 126)):
        s0, s1 = split(rng, [p] * trials, R)
        t0 = oracle.words_u128(oracle.share_trunc(0, words(s0), k))
        t1 = oracle.words_u128(oracle.share_trunc(1, words(s1), k))
        bad = np.mean([signed(a + b) - (p >> k) not in (0, 1) for a, b in zip(t0, t1)])
        assert abs(bad - 0.25) <= 5 * np.sqrt(0.25 * 0.75 / trials), bad


# ---- field to ring, extension, ring to field ------------------------------------
def test_field_to_ring_is_exact():
    o = small_oracle()
    q = o.primes[0]
    h = (q - 1) // 2
    rng = np.random.default_rng(7)
    t0 = [int(v) for v in rng.integers(0, q, 400, dtype=np.uint64)]
    t1 = [int(v) for v in rng.integers(0, q, 400, dtype=np.uint64)]
    # edge cases around the wrap: (t0 + h mod q) + t1 in {q - 1, q, q + 1}, 0, 2q - 2
    for tgt in (q - 1, q, q + 1):
        a = int(rng.integers(1, q - 1))
        t0.append((a - h) % q)
        t1.append((tgt - a) % q)
    t0 += [(0 - h) % q, q - 1, 0]
    t1 += [0, q - 1, 0]
    w0, w1 = oracle.f2r_wrap_sim(q, np.array(t0, np.uint64), np.array(t1, np.uint64), 11, 2)
    U0 = oracle.words_u128(oracle.f2r_local(0, q, np.array(t0, np.uint64), w0))
    U1 = oracle.words_u128(oracle.f2r_local(1, q, np.array(t1, np.uint64), w1))
    for a, b, x, y in zip(t0, t1, U0, U1):
        m = (a + b) % q
        m = m - q if m > h else m
        assert signed(x + y) == m
    # the wrap-bit shares are uniform-looking: P0's share alone reveals nothing
    assert len({int(v) for v in w0[:, 1]}) > 390


@pytest.mark.parametrize("l", [L_MPC, 20, 62])
def test_signed_extension_is_exact(l):
    rng = np.random.default_rng(l)
    M = 1 << l
    x0 = [int(v) for v in rng.integers(0, M, 400, dtype=np.uint64)]
    x1 = [int(v) for v in rng.integers(0, M, 400, dtype=np.uint64)]
    for tgt in (M - 1, M, M + 1, 0, M // 2, M // 2 - 1):
        a = int(rng.integers(1, M - 1))
        x0.append((a - M // 2) % M)
        x1.append((tgt - a) % M)
    w0, w1 = oracle.ext_wrap_sim(l, np.array(x0, np.uint64), np.array(x1, np.uint64), 3, 9)
    X0 = oracle.words_u128(oracle.ext_local(0, l, np.array(x0, np.uint64), w0))
    X1 = oracle.words_u128(oracle.ext_local(1, l, np.array(x1, np.uint64), w1))
    for a, b, x, y in zip(x0, x1, X0, X1):
        assert signed(x + y) == signed(a + b, l)


def test_ring_to_field():
    o = small_oracle()
    level = o.nQ - 1
    rng = np.random.default_rng(8)
    ms = [int(v) for v in rng.integers(-2**61, 2**61, 200)] + [0, 1, -1]
    cases = [split(rng, ms, R)]
    # shares bounded like the output of a truncation, and two zero shares
    b0 = [signed(int.from_bytes(rng.bytes(12), "little"), 96) for _ in ms]
    cases.append((b0, [m - a for m, a in zip(ms, b0)]))
    cases.append(([0] * len(ms), list(ms)))
    for s0, s1 in cases:
        r0 = o.r2f_local(0, words(s0), level)
        r1 = o.r2f_local(1, words(s1), level)
        for i in range(level + 1):
            q = o.primes[i]
            got = (r0[i].astype(object) + r1[i].astype(object)) % q
            assert list(got) == [m % q for m in ms]
    # the failure case: signed shares that overflow when added (s0 = 2^127 - 1,
    # s1 = m - s0 wraps to a positive value for m < 0)
    m = -5
    s0 = (1 << 127) - 1
    r = (o.r2f_local(0, words([s0]), 0)[0, 0] + o.r2f_local(1, words([m - s0]), 0)[0, 0]) % o.primes[0]
    assert int(r) == (m + R) % o.primes[0] != m % o.primes[0]


# ---- decoding of shares (C2M) -----------------------------------------------------
def c2m_reconstruct(o, m, scale, seed):
    """Share the coefficients m (signed ints) mod q_0, run both parties' local
    steps, return the reconstructed fixed-point slots as floats."""
    q = o.primes[0]
    rng = np.random.default_rng(seed)
    t0, t1 = split(rng, [int(v) for v in m], q)
    t0, t1 = np.array(t0, np.uint64), np.array(t1, np.uint64)
    w0, w1 = oracle.f2r_wrap_sim(q, t0, t1, seed, 1)
    o0 = o.c2m_local(0, t0, w0, scale, L_MPC, SF)
    o1 = o.c2m_local(1, t1, w1, scale, L_MPC, SF)
    assert int(o0.max()) < 1 << L_MPC and int(o1.max()) < 1 << L_MPC
    return np.array([signed(int(a) + int(b), L_MPC) for a, b in zip(o0, o1)], float) / 2**SF


@pytest.mark.parametrize("scale", [2.0**40, 2.0**40 * 1.37, 2.0**30, 2.0**50])
def test_c2m_decoding_within_one_unit(scale):
    o = small_oracle()
    rng = np.random.default_rng(int(np.log2(scale) * 10))
    z = rng.uniform(-6, 6, o.N // 2)
    m = o.encode_int(z, scale)
    ref = o.decode(m, scale)
    x = c2m_reconstruct(o, m, scale, 21)
    err = x - ref
    assert np.abs(err).max() < 2.0**-SF + 2.0**-17
    assert abs(err.mean()) < 0.05 * 2.0**-SF      # probabilistic rounding: no bias


def test_c2m_against_the_definition_at_n32():
    """z_j = (1/Delta) sum_t m_t zeta^(t 5^j), evaluated term by term."""
    o = oracle.Oracle(5, (50, 40), (60,), 2)
    N, s = o.N, o.N // 2
    rng = np.random.default_rng(4)
    scale = 2.0**36
    m = rng.integers(-2**38, 2**38, N)
    zeta = np.exp(1j * np.pi / N)
    z = np.array([sum(int(m[t]) * zeta**(t * pow(5, j, 2 * N)) for t in range(N)).real / scale for j in range(s)])
    x = c2m_reconstruct(o, m, scale, 5)
    assert np.abs(x - z).max() < 2.0**-SF + 2.0**-17


def test_c2m_degenerate_inputs():
    o = small_oracle()
    N = o.N
    zero = c2m_reconstruct(o, np.zeros(N, np.int64), 2.0**40, 3)
    assert np.abs(zero).max() <= 2.0**-SF
    # a constant polynomial m_0 = c: every slot decodes to c / Delta
    m = np.zeros(N, np.int64)
    m[0] = 3 << 40
    x = c2m_reconstruct(o, m, 2.0**40, 4)
    assert np.abs(x - 3.0).max() < 2.0**-SF + 2.0**-17


# ---- encoding of shares (M2C) -----------------------------------------------------
def m2c_reconstruct(o, xi, level, scale, seed):
    """Share the fixed-point slots xi (signed ints at 2^-sf) mod 2^l, run both
    parties' local steps, return the residues of the sum per prime."""
    rng = np.random.default_rng(seed)
    x0, x1 = split(rng, [int(v) for v in xi], 1 << L_MPC)
    x0, x1 = np.array(x0, np.uint64), np.array(x1, np.uint64)
    w0, w1 = oracle.ext_wrap_sim(L_MPC, x0, x1, seed, 2)
    r0 = o.m2c_local(0, x0, w0, level, scale, L_MPC, SF)
    r1 = o.m2c_local(1, x1, w1, level, scale, L_MPC, SF)
    return [(r0[i].astype(object) + r1[i].astype(object)) % o.primes[i] for i in range(level + 1)]


@pytest.mark.parametrize("scale,n", [(2.0**40, None), (2.0**40 * 1.37, None), (2.0**30, 1000), (2.0**58, 7)])
def test_m2c_encoding(scale, n):
    o = small_oracle()
    s = o.N // 2
    n = s if n is None else n
    level = o.nQ - 1
    rng = np.random.default_rng(n)
    xi = np.round(rng.uniform(-8, 8, n) * 2**SF).astype(np.int64)
    x = xi / 2**SF
    res = m2c_reconstruct(o, xi, level, scale, 17)
    mc = o.centered(np.array(res[0], np.uint64))
    for i in range(1, level + 1):               # one integer behind every prime
        assert list(res[i]) == [int(v) % o.primes[i] for v in mc]
    ref = o.encode_int(x, scale)
    assert np.abs(mc - ref).max() <= scale * 2.0**-(oracle.FX_P - 2)
    z = o.decode(mc, scale)
    assert np.abs(z[:n] - x).max() < 2.0**-17
    assert np.abs(z[n:]).max(initial=0) < 2.0**-17


def test_m2c_zero_shares_encode_zero():
    o = small_oracle()
    res = m2c_reconstruct(o, np.zeros(o.N // 2, np.int64), 1, 2.0**40, 8)
    assert all(int(v) == 0 for r in res for v in r)


# ---- the protocol end to end (Alg. 1 then Alg. 2) --------------------------------
def test_c2m_then_m2c_round_trip():
    o = small_oracle()
    prm = wl.SMALL
    N, s = o.N, o.N // 2
    seed = 0xC2
    sk = o.keygen_secret(seed)
    level = o.nQ - 1
    rng = np.random.default_rng(12)
    z = rng.uniform(-5, 5, s)
    ct = o.encrypt(sk, o.encode(z, level, prm.scale), seed, 1)
    # Alg. 1: P1 masks, P0 decrypts; both convert to shares of the slots
    masked, p1 = o.he2mpc(ct, seed, 2)
    p0 = o.decrypt(sk, masked)[0]
    q = o.primes[0]
    w0, w1 = oracle.f2r_wrap_sim(q, p0, p1, seed, 3)
    y0 = o.c2m_local(0, p0, w0, prm.scale, L_MPC, SF)
    y1 = o.c2m_local(1, p1, w1, prm.scale, L_MPC, SF)
    xi = np.array([signed(int(a) + int(b), L_MPC) for a, b in zip(y0, y1)])
    assert np.abs(xi / 2**SF - z).max() < 2.0**-SF + 2.0**-17
    # Alg. 2: back to a ciphertext at level 1 with the same scale
    lv = 1
    v0, v1 = oracle.ext_wrap_sim(L_MPC, y0, y1, seed, 4)
    m0 = o.m2c_local(0, y0, v0, lv, prm.scale, L_MPC, SF)
    m1 = o.m2c_local(1, y1, v1, lv, prm.scale, L_MPC, SF)
    ct2 = o.encrypt(sk, m0, seed, 5)            # P0 encrypts its share
    for i in range(lv + 1):                     # P1 adds its share
        ct2[0, i] = (ct2[0, i].astype(object) + m1[i].astype(object)) % o.primes[i]
    dec = o.decode(o.centered(o.decrypt(sk, ct2)[0]), prm.scale)
    assert np.abs(dec - xi / 2**SF).max() < 2.0**-17
