"""Pins for the oracle's ring layer: primes, NTT, RNS products, Philox sampling.

Each check compares the oracle with something it does not share code with:
sympy's primality test, the O(N^2) definition of the transform, Python
big-integer arithmetic, published Philox known-answer vectors, cuRAND's CPU
generator, and distribution statistics computed with the decimal module.
"""
import ctypes
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest
import sympy

import oracle
from paper_2508_19525_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bitrev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def schoolbook_negacyclic(a, b, q):
    N = len(a)
    out = [0] * N
    for i in range(N):
        ai = int(a[i])
        if not ai:
            continue
        for j in range(N):
            k = i + j
            v = ai * int(b[j])
            if k >= N:
                out[k - N] -= v
            else:
                out[k] += v
    return [x % q for x in out]


# --------------------------------------------------------------------------- primes
@pytest.mark.parametrize("prm", [wl.TINY, wl.BERT_CP, wl.BERT_CC, wl.SMALL, wl.MICRO])
def test_prime_rule(prm):
    o = oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum)
    twoN = 2 * prm.N
    bits = list(prm.q_bits) + list(prm.p_bits)
    assert len(set(o.primes)) == len(o.primes)
    for i, (q, b) in enumerate(zip(o.primes, bits)):
        assert sympy.isprime(q) and q % twoN == 1 and q < 2 ** b
        # largest such prime below 2^b not taken by an earlier index
        c = (2 ** b - 1) - ((2 ** b - 2) % twoN)
        while c > q:
            assert c in o.primes[:i] or not sympy.isprime(c)
            c -= twoN
        psi = o.psi[i]
        assert pow(psi, prm.N, q) == q - 1
        # psi comes from the first base x whose power has order 2N
        for x in range(2, 200):
            w = pow(x, (q - 1) // twoN, q)
            if pow(w, prm.N, q) == q - 1:
                assert w == psi
                break


def test_is_prime_matches_sympy():
    rng = np.random.default_rng(1)
    cands = [int(x) | 1 for x in rng.integers(2 ** 40, 2 ** 62, size=300, dtype=np.int64)]
    cands += [561, 1105, 1729, 2465, 2821, 6601, 3215031751, 3825123056546413051,
              2 ** 61 - 1, 2 ** 62 - 57, 1, 2, 3, 4]
    for c in cands:
        assert oracle.is_prime(c) == sympy.isprime(c), c


# --------------------------------------------------------------------------- NTT
@pytest.mark.parametrize("logN", [2, 4, 6, 8])
def test_ntt_matches_definition(logN):
    o = oracle.Oracle(logN, (30, 31), (32,), 1)
    N = 1 << logN
    for pi, q in enumerate(o.primes):
        psi = o.psi[pi]
        a = wl.random_residues([q], N, seed=logN * 10 + pi)[0, 0]
        A = o.ntt(a, pi)
        for k in range(N):
            e = 2 * bitrev(k, logN) + 1
            ref = sum(int(a[j]) * pow(psi, e * j, q) for j in range(N)) % q
            assert int(A[k]) == ref
        assert np.array_equal(o.intt(A, pi), a)


@pytest.mark.parametrize("logN", [4, 8, 10])
def test_negacyclic_mul_schoolbook(logN):
    o = oracle.Oracle(logN, (50, 40), (60,), 1)
    N = 1 << logN
    for pi, q in enumerate(o.primes):
        a = wl.random_residues([q], N, seed=100 + pi)[0, 0]
        b = wl.random_residues([q], N, seed=200 + pi)[0, 0]
        got = o.negacyclic_mul(a, b, pi)
        assert [int(x) for x in got] == schoolbook_negacyclic(a, b, q)


def test_rns_product_equals_bigint_product():
    """Residue-wise products CRT-reconstruct to the big-integer negacyclic
    product mod Q = prod q_i."""
    o = oracle.Oracle(6, (60, 40, 40, 40), (60,), 2)
    N = o.N
    qs = o.primes[:4]
    Q = 1
    for q in qs:
        Q *= q
    rng = np.random.default_rng(7)
    A = [int(rng.integers(0, 2 ** 62)) * 2 ** 124 + int(rng.integers(0, 2 ** 62)) * 2 ** 62
         + int(rng.integers(0, 2 ** 62)) for _ in range(N)]
    B = [int(rng.integers(0, 2 ** 62)) * 2 ** 62 + int(rng.integers(0, 2 ** 62)) for _ in range(N)]
    A = [x % Q for x in A]
    B = [x % Q for x in B]
    ref = schoolbook_negacyclic(A, B, Q)
    limbs = []
    for i, q in enumerate(qs):
        a = np.array([x % q for x in A], np.uint64)
        b = np.array([x % q for x in B], np.uint64)
        limbs.append([int(v) for v in o.negacyclic_mul(a, b, i)])
    for c in range(N):
        x = 0
        for i, q in enumerate(qs):
            Qi = Q // q
            x += limbs[i][c] * Qi * pow(Qi, -1, q)
        assert x % Q == ref[c]


# --------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox(v[0:4], v[4:6]) == v[6:10]


def test_philox_matches_curand_cpu_generator():
    """cuRAND's host-side PHILOX4_32_10 generator (runs on the CPU) emits block
    n of a seed as Philox at counter (0, 0, n, 0), key = (seed lo, seed hi)."""
    path = "/usr/local/cuda/lib64/libcurand.so"
    if not os.path.exists(path):
        pytest.skip("libcurand not present")
    cr = ctypes.CDLL(path)
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0
    seed = 0x0123456789ABCDEF
    assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    n = 32
    buf = (ctypes.c_uint * (4 * n))()
    assert cr.curandGenerate(gen, buf, 4 * n) == 0
    cr.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in range(n):
        assert oracle.philox([0, 0, b, 0], key) == list(buf[4 * b:4 * b + 4])


# --------------------------------------------------------------------------- samplers
def _dgauss_pmf():
    """Discrete Gaussian sigma=3.2 on |x| <= 19, with exp from the decimal module
    (independent of the C library's exp)."""
    getcontext().prec = 50
    s2 = Decimal(2) * Decimal("3.2") ** 2
    rho = {x: (-(Decimal(x * x)) / s2).exp() for x in range(-19, 20)}
    Z = sum(rho.values())
    return {x: rho[x] / Z for x in rho}


def test_cdt_table_against_decimal_exp():
    pmf = _dgauss_pmf()
    T = oracle.cdt_table()
    acc = Decimal(0)
    for k in range(19):
        acc += pmf[0] if k == 0 else 2 * pmf[k]
        ref = acc * Decimal(2) ** 64
        # the table is built in double precision: 53 significant bits
        assert abs(Decimal(int(T[k])) - ref) <= ref * Decimal(2) ** -50 + 1
    assert np.all(np.diff(T.astype(object)) > 0)


def test_gauss_sampler_distribution():
    N = 1 << 16
    e = np.concatenate([oracle.sample_gauss(N, 99, obj, oracle.ENC_E) for obj in range(8)])
    assert np.abs(e).max() <= 19
    pmf = _dgauss_pmf()
    var = float(sum(Decimal(x * x) * p for x, p in pmf.items()))
    assert abs(e.mean()) < 0.02
    assert abs(e.var() / var - 1) < 0.01
    # chi^2 over |x| <= 8 plus a tail bin
    obs = [np.sum(e == x) for x in range(-8, 9)] + [np.sum(np.abs(e) > 8)]
    exp_ = [float(pmf[x]) * len(e) for x in range(-8, 9)]
    exp_.append(len(e) - sum(exp_))
    chi2 = sum((o - x) ** 2 / x for o, x in zip(obs, exp_))
    assert chi2 < 60  # 17 dof: p ~ 1e-6


def test_ternary_and_uniform_samplers():
    N = 1 << 16
    s = oracle.sample_ternary(N, 5, 0, oracle.SECRET)
    counts = [np.sum(s == v) for v in (-1, 0, 1)]
    chi2 = sum((c - N / 3) ** 2 / (N / 3) for c in counts)
    assert set(np.unique(s)) <= {-1, 0, 1} and chi2 < 20
    q = (1 << 60) - 93  # any modulus: reduction of a 128-bit draw
    u = oracle.sample_uniform(N, q, 5, 3, oracle.MASK)
    assert u.max() < q
    hist = np.bincount((u.astype(np.float64) / q * 64).astype(int), minlength=64)
    chi2 = np.sum((hist - N / 64) ** 2 / (N / 64))
    assert chi2 < 120  # 63 dof
    # distinct (obj, purpose, j) give independent streams
    assert not np.array_equal(u, oracle.sample_uniform(N, q, 5, 4, oracle.MASK))
    assert not np.array_equal(u, oracle.sample_uniform(N, q, 5, 3, oracle.MASK, 1))


def test_uniform_sampler_is_128bit_draw_mod_q():
    q = 1125899906826241
    u = oracle.sample_uniform(8, q, 0xDEADBEEF, 7, oracle.KEY_A, 3)
    for i in range(8):
        r = oracle.philox([i, 3, 7, oracle.KEY_A], [0xDEADBEEF, 0])
        v = r[0] | (r[1] << 32) | (r[2] << 64) | (r[3] << 96)
        assert int(u[i]) == v % q
