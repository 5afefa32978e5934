"""Pins for the oracle's CKKS layer (Sec. 2.4, Sec. 6.1 Eq. 2) and hybrid key
switching.  References: the O(N^2) canonical-embedding definition in numpy,
exact closed forms (constant and monomial encodings), big-integer CRT and
rounding in Python, schoolbook products, and the exact error identity of
secret-key encryption."""
import numpy as np
import pytest

import oracle
from paper_2508_19525_b300 import workloads as wl


def make(prm):
    return oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum)


def crt(limbs, primes):
    """limbs: (n, N) residues -> list of centered big integers mod prod(primes)."""
    Q = 1
    for q in primes:
        Q *= q
    out = []
    for c in range(limbs.shape[1]):
        x = 0
        for i, q in enumerate(primes):
            Qi = Q // q
            x += int(limbs[i, c]) * Qi * pow(Qi, -1, q)
        x %= Q
        out.append(x - Q if x > Q // 2 else x)
    return out, Q


def schoolbook(a, b, N):
    out = [0] * N
    for i in range(N):
        if not a[i]:
            continue
        for j in range(N):
            k = i + j
            if k >= N:
                out[k - N] -= a[i] * b[j]
            else:
                out[k] += a[i] * b[j]
    return out


# --------------------------------------------------------------------------- encoding
def canonical_embedding_encode(z, N, scale):
    """m_t = round(scale * (2/N) * Re sum_j z_j zeta^(-t 5^j)), zeta = e^{i pi/N}."""
    s = N // 2
    five = np.array([pow(5, j, 2 * N) for j in range(s)], dtype=np.int64)
    t = np.arange(N)
    ang = -np.pi * np.outer(t, five) / N
    v = (2.0 / N) * (np.cos(ang) @ np.asarray(z))
    return np.rint(v * scale).astype(np.int64)


@pytest.mark.parametrize("logN", [4, 7, 10])
def test_encode_matches_definition(logN):
    o = oracle.Oracle(logN, (50, 40), (60,), 1)
    N = 1 << logN
    z = wl.slot_vector(N // 2, seed=logN)
    got = o.encode_int(z, 2.0 ** 40)
    ref = canonical_embedding_encode(z, N, 2.0 ** 40)
    assert np.max(np.abs(got - ref)) <= 1


def test_encode_closed_forms():
    o = make(wl.TINY)
    N, s = o.N, o.N // 2
    # a constant slot vector is the constant polynomial
    c = 0.625
    m = o.encode_int(np.full(s, c), 2.0 ** 40)
    assert m[0] == round(c * 2 ** 40) and np.all(m[1:] == 0)
    # decoding the monomial X^t gives zeta^(t 5^j) (real part) / scale
    for t in (1, 5, N - 1):
        coef = np.zeros(N, np.int64)
        coef[t] = 1 << 20
        z = o.decode(coef, 2.0 ** 20)
        five = np.array([pow(5, j, 2 * N) for j in range(s)])
        assert np.allclose(z, np.cos(np.pi * t * five / N), atol=1e-12)


@pytest.mark.parametrize("prm", [wl.TINY, wl.BERT_CP])
def test_decode_inverts_encode(prm):
    o = make(prm)
    z = wl.slot_vector(o.N // 2, seed=3)
    m = o.encode_int(z, 2.0 ** 40)
    assert np.max(np.abs(o.decode(m, 2.0 ** 40) - z)) < 2.0 ** -30
    # partial vectors pad with zeros
    m2 = o.encode_int(z[:100], 2.0 ** 40)
    z2 = o.decode(m2, 2.0 ** 40)
    assert np.max(np.abs(z2[:100] - z[:100])) < 2.0 ** -30 and np.max(np.abs(z2[100:])) < 2.0 ** -30


def test_encode_limbs_are_residues_of_signed_coefficients():
    o = make(wl.SMALL)
    z = wl.slot_vector(o.N // 2, seed=11)
    m = o.encode_int(z, 2.0 ** 40)
    limbs = o.encode(z, 4, 2.0 ** 40)
    for i in range(5):
        q = o.primes[i]
        assert all(int(limbs[i, t]) == int(m[t]) % q for t in range(o.N))


# --------------------------------------------------------------------------- encryption
def test_decrypt_of_encrypt_is_message_plus_sampled_error():
    """c0 + c1 s = (-a s + m + e) + a s = m + e exactly; e is the ENC_E draw."""
    o = make(wl.SMALL)
    s = o.keygen_secret(42)
    pt = o.encode(wl.slot_vector(o.N // 2, seed=1), 4, 2.0 ** 40)
    ct = o.encrypt(s, pt, 42, nonce=17)
    m = o.decrypt(s, ct)
    e = oracle.sample_gauss(o.N, 42, 17, oracle.ENC_E)
    for i in range(5):
        q = o.primes[i]
        assert np.array_equal(m[i], (pt[i].astype(object) + e.astype(object)) % q)
    # c1 is the uniform draw
    for i in range(5):
        assert np.array_equal(ct[1, i], oracle.sample_uniform(o.N, o.primes[i], 42, 17, oracle.ENC_A, i))
    assert np.array_equal(s, oracle.sample_ternary(o.N, 42, 0, oracle.SECRET))


def test_key_switching_key_relation():
    """b_j + a_j s = e_j + [t in D_j] (P mod q_t) s'  (mod every prime t), checked
    with schoolbook products at N=32."""
    o = make(wl.MICRO)
    N = o.N
    s = o.keygen_secret(5)
    sp = oracle.sample_ternary(N, 77, 0, oracle.SECRET)
    ksk = o.keygen_ksk(5, s, sp, obj=9)
    P = 1
    for p in o.primes[o.nQ:]:
        P *= p
    for j in range(o.dnum):
        e = oracle.sample_gauss(N, 5, 9, oracle.KEY_E, j)
        for t, q in enumerate(o.primes):
            b = [int(x) for x in ksk[j, 0, t]]
            a = [int(x) for x in ksk[j, 1, t]]
            a_s = schoolbook(a, [int(x) for x in s], N)
            in_digit = t < o.nQ and j * o.alpha <= t < (j + 1) * o.alpha
            for c in range(N):
                want = int(e[c]) + (P * int(sp[c]) if in_digit else 0)
                assert (b[c] + a_s[c] - want) % q == 0


def test_relin_key_uses_s_squared():
    o = make(wl.MICRO)
    N = o.N
    s = o.keygen_secret(3)
    s2 = schoolbook([int(x) for x in s], [int(x) for x in s], N)
    assert np.array_equal(o.keygen_relin(3, s), o.keygen_ksk(3, s, np.array(s2, np.int64), 0))


# --------------------------------------------------------------------------- automorphism
def test_automorphism_identities():
    o = make(wl.MICRO)
    N = o.N
    q = o.primes[0]
    a = wl.random_residues([q], N, 1)[0]
    b = wl.random_residues([q], N, 2)[0]
    g, h = o.galois_elt(3), o.galois_elt(5)
    ab = o.negacyclic_mul(a[0], b[0], 0)[None]
    lhs = o.automorphism(ab, g)
    rhs = o.negacyclic_mul(o.automorphism(a, g)[0], o.automorphism(b, g)[0], 0)[None]
    assert np.array_equal(lhs, rhs)
    assert np.array_equal(o.automorphism(o.automorphism(a, h), g), o.automorphism(a, (g * h) % (2 * N)))
    assert np.array_equal(o.automorphism(a, 1), a)
    assert o.galois_elt(-3) == pow(5, N // 2 - 3, 2 * N)


def test_rotation_shifts_slots_left():
    o = make(wl.TINY)
    s = o.keygen_secret(1)
    z = wl.slot_vector(o.N // 2, seed=2)
    ct = o.encrypt(s, o.encode(z, 2, 2.0 ** 40), 1, 0)
    for r in (1, 37, -5):
        gk = o.keygen_galois(1, s, o.galois_elt(r))
        rot = o.rotate(ct, r, gk)
        got = o.decode(o.centered(o.decrypt(s, rot)[0]), 2.0 ** 40)
        assert np.max(np.abs(got - np.roll(z, -r))) < 1e-6


# --------------------------------------------------------------------------- key switching
def _noise_free_key(o, sp, level_top=True):
    """Key with a_j = 0 and e_j = 0: b_j[t] = [t in D_j] (P mod q_t) s'."""
    N = o.N
    P = 1
    for p in o.primes[o.nQ:]:
        P *= p
    k = np.zeros(o.ksk_shape(), np.uint64)
    for j in range(o.dnum):
        for t, q in enumerate(o.primes):
            if t < o.nQ and j * o.alpha <= t < (j + 1) * o.alpha:
                k[j, 0, t] = [(P % q) * int(x) % q for x in sp]
    return k


@pytest.mark.parametrize("level", [4, 3, 2, 0])
def test_keyswitch_exact_with_noise_free_key(level):
    """With a zero mask and zero error the key inner product is an exact multiple
    of P, so decompose / ModUp / inner product / ModDown must return exactly
    (d * s' mod Q_l, 0)."""
    o = make(wl.HEParams(5, wl.SMALL.q_bits, wl.SMALL.p_bits, wl.SMALL.dnum))
    N = o.N
    sp = oracle.sample_ternary(N, 8, 0, oracle.SECRET)
    ksk = _noise_free_key(o, sp)
    d = wl.random_residues(o.primes[:level + 1], N, seed=level)[0]
    out = o.keyswitch(d, ksk)
    for i in range(level + 1):
        q = o.primes[i]
        ref = [x % q for x in schoolbook([int(v) for v in d[i]], [int(v) for v in sp], N)]
        assert [int(v) for v in out[0, i]] == ref
        assert not out[1, i].any()


@pytest.mark.parametrize("level", [4, 2, 0])
def test_keyswitch_noise_bound(level):
    """k0 + k1 s - d s' is small: (sum_j d~_j e_j)/P plus the ModDown rounding.
    Bound: beta * alpha * max(Q_j) * N * 19 / P + nP * (1 + N)."""
    prm = wl.HEParams(6, wl.SMALL.q_bits, wl.SMALL.p_bits, wl.SMALL.dnum)
    o = make(prm)
    N = o.N
    s = o.keygen_secret(21)
    sp = oracle.sample_ternary(N, 99, 0, oracle.SECRET)
    ksk = o.keygen_ksk(21, s, sp, obj=4)
    d = wl.random_residues(o.primes[:level + 1], N, seed=level + 50)[0]
    out = o.keyswitch(d, ksk)
    dec = o.decrypt(s, out)
    primes = o.primes[:level + 1]
    got, Q = crt(dec, primes)
    d_int, _ = crt(d, primes)
    want = schoolbook(d_int, [int(x) for x in sp], N)
    P = 1
    for p in o.primes[o.nQ:]:
        P *= p
    beta = (level + 1 + o.alpha - 1) // o.alpha
    Qj = max(o.primes[:level + 1]) ** o.alpha
    bound = beta * o.alpha * Qj * N * 19 // P + o.nP * (1 + N)
    for c in range(N):
        diff = (got[c] - want[c]) % Q
        diff = diff - Q if diff > Q // 2 else diff
        assert abs(diff) <= bound


# --------------------------------------------------------------------------- rescale
def test_rescale_is_rounded_division():
    prm = wl.HEParams(4, wl.SMALL.q_bits, wl.SMALL.p_bits, wl.SMALL.dnum)
    o = make(prm)
    for level in (4, 2, 1):
        primes = o.primes[:level + 1]
        ct = wl.random_residues(primes, o.N, seed=level, polys=2)
        out = o.rescale(ct)
        ql = primes[-1]
        for poly in range(2):
            x, Q = crt(ct[poly], primes)
            y, Qd = crt(out[poly], primes[:-1])
            for c in range(o.N):
                # round(x / q_l) with x taken in [0, Q)
                xv = x[c] % Q
                r = (2 * xv + ql) // (2 * ql)
                assert (y[c] - r) % Qd == 0


# --------------------------------------------------------------------------- products
def test_tensor_and_relinearize_decrypt_to_product():
    o = make(wl.TINY)
    s = o.keygen_secret(6)
    z1 = wl.slot_vector(o.N // 2, seed=8)
    z2 = wl.slot_vector(o.N // 2, seed=9)
    c1 = o.encrypt(s, o.encode(z1, 2, 2.0 ** 40), 6, 1)
    c2 = o.encrypt(s, o.encode(z2, 2, 2.0 ** 40), 6, 2)
    t = o.tensor(c1, c2)
    rk = o.keygen_relin(6, s)
    r = o.relinearize(t, rk)
    # both the 3-polynomial and the relinearized ciphertexts decrypt to z1*z2
    for ct in (t, r):
        res = o.rescale(ct)
        scale = 2.0 ** 80 / o.primes[2]
        got = o.decode(o.centered(o.decrypt(s, res)[0]), scale)
        assert np.max(np.abs(got - z1 * z2)) < 1e-6


@pytest.mark.parametrize("level", [4, 2, 0])
def test_moddown_is_rounded_division_by_P(level):
    """ModDown returns round(x / P) mod q_i for x given by its residues over
    Q_l u P (big-integer CRT and rounding in Python)."""
    prm = wl.HEParams(6, wl.SMALL.q_bits, wl.SMALL.p_bits, wl.SMALL.dnum)
    o = make(prm)
    n = level + 1
    basis = o.primes[:n] + o.primes[o.nQ:]
    acc = wl.random_residues(basis, o.N, seed=300 + level, polys=2)
    out = o.moddown(acc, level)
    QP = 1
    for q in basis:
        QP *= q
    P = 1
    for p in o.primes[o.nQ:]:
        P *= p
    for poly in range(2):
        for c in range(o.N):
            x = 0
            for i, q in enumerate(basis):
                Qi = QP // q
                x += int(acc[poly, i, c]) * Qi * pow(Qi, -1, q)
            x %= QP
            r = (2 * x + P) // (2 * P)  # round(x / P), x in [0, QP)
            for i in range(n):
                assert int(out[poly, i, c]) == r % o.primes[i], (poly, c, i)


def test_limb_consistency_check_catches_a_wrong_residue():
    """The full-size GPU tests check every limb of each decryption against
    limb 0 (assert_limbs_consistent); on the oracle, a clean decryption passes
    and one residue changed in limb 3 of the ciphertext fails."""
    from _helpers import assert_limbs_consistent
    o = make(wl.SMALL)
    sk = o.keygen_secret(1)
    ct = o.encrypt(sk, o.encode(wl.slot_vector(o.N // 2, seed=3), 4, 2.0 ** 40), 1, 1)
    assert_limbs_consistent(o.decrypt(sk, ct), o.primes)
    ct[0, 3, 7] = (int(ct[0, 3, 7]) + 1) % o.primes[3]
    with pytest.raises(AssertionError):
        assert_limbs_consistent(o.decrypt(sk, ct), o.primes)
