"""Pins for the oracle's hoisted rotations and one-ModDown rotation sums (the
key-switching forms the BSGS products use).  References written here, not taken
from the oracle: the automorphism X^i -> X^(i g) with its sign, schoolbook
negacyclic products, big-integer CRT, and the key-switching noise bound."""
import numpy as np
import pytest

import oracle
from paper_2508_19525_b300 import workloads as wl

from test_oracle_ckks import crt, make, schoolbook

PRM = wl.HEParams(5, wl.SMALL.q_bits, wl.SMALL.p_bits, wl.SMALL.dnum)


def sigma_int(a, g, N):
    """X^i -> X^(i g mod 2N) on integer coefficients (negated past N)."""
    out = [0] * N
    for i in range(N):
        k = (i * g) % (2 * N)
        if k < N:
            out[k] = a[i]
        else:
            out[k - N] = -a[i]
    return out


def noise_free_galois_key(o, s, g):
    """b_j[t] = [t in D_j] (P mod q_t) sigma_g(s), a_j = 0, no error."""
    sp = sigma_int([int(x) for x in s], g, o.N)
    P = 1
    for p in o.primes[o.nQ:]:
        P *= p
    k = np.zeros(o.ksk_shape(), np.uint64)
    for j in range(o.dnum):
        for t, q in enumerate(o.primes):
            if t < o.nQ and j * o.alpha <= t < (j + 1) * o.alpha:
                k[j, 0, t] = [(P % q) * x % q for x in sp]
    return k, sp


def expected_rotation(ct, g, sp, primes, N):
    """sigma_g(c0) + sigma_g(c1) sigma_g(s) per limb, exactly."""
    out = np.zeros((len(primes), N), np.uint64)
    for i, q in enumerate(primes):
        c0 = sigma_int([int(x) for x in ct[0, i]], g, N)
        c1 = sigma_int([int(x) for x in ct[1, i]], g, N)
        prod = schoolbook(c1, sp, N)
        out[i] = [(a + b) % q for a, b in zip(c0, prod)]
    return out


@pytest.mark.parametrize("level", [4, 2])
def test_hoisted_rotation_exact_with_noise_free_keys(level):
    """With a = 0 and e = 0 every inner product is an exact multiple of P on the
    digit's own primes and zero elsewhere, so each hoisted rotation must equal
    (sigma_g(c0) + sigma_g(c1) sigma_g(s), 0) exactly."""
    o = make(PRM)
    N, primes = o.N, o.primes[:level + 1]
    s = o.keygen_secret(3)
    ct = wl.random_residues(primes, N, seed=10 + level, polys=2)
    rots = [1, 3, -2, 7]
    keys, sps = [], []
    for r in rots:
        k, sp = noise_free_galois_key(o, s, o.galois_elt(r))
        keys.append(k)
        sps.append(sp)
    outs = o.rotate_hoisted(ct, rots, keys)
    for r, sp, out in zip(rots, sps, outs):
        assert not out[1].any()
        assert np.array_equal(out[0], expected_rotation(ct, o.galois_elt(r), sp, primes, N))


@pytest.mark.parametrize("level", [4, 1])
def test_hoisted_rotation_noise_bound(level):
    """k0 + k1 s - sigma_g(c0 + c1 s) is within the key-switching bound: the
    extended digits after sigma_g have the magnitudes of the digits of c1."""
    o = make(wl.HEParams(6, wl.SMALL.q_bits, wl.SMALL.p_bits, wl.SMALL.dnum))
    N, primes = o.N, o.primes[:level + 1]
    s = o.keygen_secret(21)
    ct = wl.random_residues(primes, N, seed=40 + level, polys=2)
    rots = [1, 5, -3]
    keys = [o.keygen_galois(21, s, o.galois_elt(r)) for r in rots]
    outs = o.rotate_hoisted(ct, rots, keys)
    c0, Q = crt(ct[0], primes)
    c1, _ = crt(ct[1], primes)
    s_int = [int(x) for x in s]
    m = [a + b for a, b in zip(c0, schoolbook(c1, s_int, N))]  # c0 + c1 s over the integers
    P = 1
    for p in o.primes[o.nQ:]:
        P *= p
    beta = (level + 1 + o.alpha - 1) // o.alpha
    Qj = max(primes) ** o.alpha
    bound = beta * o.alpha * Qj * N * 19 // P + o.nP * (1 + N)
    for r, out in zip(rots, outs):
        want = sigma_int(m, o.galois_elt(r), N)
        got, _ = crt(o.decrypt(s, out), primes)
        for c in range(N):
            diff = (got[c] - want[c]) % Q
            diff = diff - Q if diff > Q // 2 else diff
            assert abs(diff) <= bound, (r, c, diff, bound)


def test_hoisted_rotation_shifts_slots_left():
    o = make(wl.TINY)
    s = o.keygen_secret(1)
    z = wl.slot_vector(o.N // 2, seed=2)
    ct = o.encrypt(s, o.encode(z, 2, 2.0 ** 40), 1, 0)
    rots = [1, 37, -5, 64]
    outs = o.rotate_hoisted(ct, rots, [o.keygen_galois(1, s, o.galois_elt(r)) for r in rots])
    for r, out in zip(rots, outs):
        got = o.decode(o.centered(o.decrypt(s, out)[0]), 2.0 ** 40)
        assert np.max(np.abs(got - np.roll(z, -r))) < 1e-6


def test_rotate_sum_exact_with_noise_free_keys():
    """base + sum_x Rot^{r_x}(T_x) with noise-free keys and one ModDown equals
    base0 + sum_x (sigma(T_x.c0) + sigma(T_x.c1) sigma(s)) and base1, exactly."""
    o = make(PRM)
    level = 3
    N, primes = o.N, o.primes[:level + 1]
    s = o.keygen_secret(5)
    base = wl.random_residues(primes, N, seed=1, polys=2)
    rots = [2, 6, -1]
    Ts = [wl.random_residues(primes, N, seed=20 + x, polys=2) for x in range(len(rots))]
    keys, want0 = [], [[int(v) for v in base[0, i]] for i in range(len(primes))]
    for r, T in zip(rots, Ts):
        k, sp = noise_free_galois_key(o, s, o.galois_elt(r))
        keys.append(k)
        e = expected_rotation(T, o.galois_elt(r), sp, primes, N)
        for i in range(len(primes)):
            want0[i] = [a + int(b) for a, b in zip(want0[i], e[i])]
    out = o.rotate_sum(base, Ts, rots, keys)
    for i, q in enumerate(primes):
        assert [int(v) for v in out[0, i]] == [x % q for x in want0[i]]
    assert np.array_equal(out[1], base[1])


def test_rotate_sum_close_to_sum_of_rotations():
    """One ModDown for the whole sum differs from summing separately key-switched
    rotations only by rounding and key noise."""
    o = make(wl.TINY)
    s = o.keygen_secret(9)
    level = 2
    zs = [wl.slot_vector(o.N // 2, seed=60 + x) for x in range(4)]
    cts = [o.encrypt(s, o.encode(z, level, 2.0 ** 40), 9, x) for x, z in enumerate(zs)]
    rots = [3, 8, -4]
    keys = [o.keygen_galois(9, s, o.galois_elt(r)) for r in rots]
    out = o.rotate_sum(cts[0], cts[1:], rots, keys)
    got = o.decode(o.centered(o.decrypt(s, out)[0]), 2.0 ** 40)
    want = zs[0] + sum(np.roll(z, -r) for z, r in zip(zs[1:], rots))
    assert np.max(np.abs(got - want)) < 1e-6
    # and the empty sum is the base itself
    assert np.array_equal(o.rotate_sum(cts[0], [], [], []), cts[0])
