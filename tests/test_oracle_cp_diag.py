"""Pins for the oracle's diagonal-input matmul_cp (App. C.2), E = Concat_h(Att_h) W_O
with Att_h in matmul_cc's multi-head diagonal packing: decrypted outputs against
the FP64 product numpy computes, for a directly encrypted dense-diagonal input
and for the chain matmul_cc -> merge of complementary diagonals -> this product."""
import numpy as np
import pytest

import cc_schedule as cs
import oracle
from paper_2508_19525_b300 import workloads as wl

SEED = 0xD1A6


def dense_diagonals(Att, L, Hg, Kc, Dh):
    """Att: (Hg, L, Dh) -> (Dh/Kc, s) slot vectors: block h + Hg kappa of ciphertext j
    holds Att_h[i][(i + delta) mod Dh], delta = j Kc + kappa."""
    s = L * Hg * Kc
    out = np.zeros((Dh // Kc, s))
    i = np.arange(L)
    for j in range(Dh // Kc):
        for kappa in range(Kc):
            delta = j * Kc + kappa
            for h in range(Hg):
                b = h + Hg * kappa
                out[j, b * L:(b + 1) * L] = Att[h, i, (i + delta) % Dh]
    return out


def unpack_spatial(slots, L, k, d_out):
    cols = [z[b * L:(b + 1) * L] for z in slots for b in range(k)]
    return np.stack(cols[:d_out], axis=1)


def galois_keys(o, sk, rots):
    return {o.galois_elt(r): o.keygen_galois(SEED, sk, o.galois_elt(r)) for r in set(rots)}


def cp_rots(L, k, b1):
    return [b * L for b in range(1, b1)] + [g * b1 * L for g in range(1, k // b1)]


def test_diag_cp_direct_input():
    prm = wl.SMALL
    o = oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum)
    s, L, Dh, groups, d_out, b1 = o.N // 2, 32, 16, [4, 4], 64, 8
    k = s // L
    H = sum(groups)
    rng = np.random.default_rng(5)
    Att = rng.uniform(-1, 1, (H, L, Dh))
    W = rng.uniform(-1, 1, (H * Dh, d_out))
    level = o.nQ - 1
    sk = o.keygen_secret(SEED)
    cts, h0 = [], 0
    for Hg in groups:
        Kc = s // (L * Hg)
        for z in dense_diagonals(Att[h0:h0 + Hg], L, Hg, Kc, Dh):
            cts.append(o.encrypt(sk, o.encode(z, level, prm.scale), SEED, len(cts)))
        h0 += Hg
    Y = o.matmul_cp_diag(np.stack(cts), L, groups, Dh, W, d_out, b1, galois_keys(o, sk, cp_rots(L, k, b1)))
    slots = [o.decode(o.centered(o.decrypt(sk, y)[0]), prm.scale) for y in Y]
    E = np.concatenate([Att[h] for h in range(H)], axis=1) @ W
    assert np.abs(unpack_spatial(slots, L, k, d_out) - E).max() <= 1e-4


def test_diag_cp_after_matmul_cc():
    """Att_h = P_h V_h from the oracle's matmul_cc (V_h padded to L = 2 Dh
    columns), the outputs j and j + Dh/Kc added, then E = Concat(Att_h) W_O."""
    prm = wl.HEParams(12, (60,) + (40,) * 6, (60, 60, 60), 3)
    o = oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum)
    s, L, Dh, Hg, d_out, b1 = o.N // 2, 32, 16, 4, 64, 8
    Kc = s // (L * Hg)
    k = s // L
    level = o.nQ - 1
    sk = o.keygen_secret(SEED)
    rng = np.random.default_rng(9)
    P = rng.dirichlet(np.ones(L), size=(Hg, L))
    V = np.clip(rng.normal(0, 0.5, (Hg, L, Dh)), -1, 1)
    W = rng.uniform(-1, 1, (Hg * Dh, d_out))
    A, B = P, np.concatenate([V, np.zeros((Hg, L, L - Dh))], axis=2)
    n_c = L // Kc
    Az, Bz = cs.pack(A, L, Hg, Kc, n_c, rows=False), cs.pack(B, L, Hg, Kc, n_c, rows=True)
    Ac = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, c) for c, z in enumerate(Az)])
    Bc = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 50 + c) for c, z in enumerate(Bz)])
    b1s1, b1s2 = 4, 8
    cc_rots = []
    for c0 in range(1, b1s1):
        cc_rots.append(c0)
    for c0 in range(b1s1):
        cc_rots.append(c0 - L)
    for g1 in range(1, Kc // b1s1):
        cc_rots.append(g1 * b1s1)
    for b in range(1, b1s2):
        cc_rots.append(b)
    for b in range(b1s2):
        cc_rots.append(b - L)
    for g in range(1, L // b1s2):
        cc_rots.append(-g * b1s2)
    for t in range(1, L):
        g = t // b1s2
        cc_rots.append((g * b1s2 - (t % Kc) * Hg * L) % s)
    gk = galois_keys(o, sk, [r for r in cc_rots if r % s] + cp_rots(L, k, b1))
    C = o.matmul_cc(Ac, Bc, L, Hg, b1s1, b1s2, gk, o.keygen_relin(SEED, sk))
    half = Dh // Kc
    merged = np.stack([(C[j].astype(object) + C[j + half].astype(object)) for j in range(half)])
    lv = C.shape[2] - 1
    for lim in range(lv + 1):  # reduce the sums limb by limb
        merged[:, :, lim, :] %= o.primes[lim]
    merged = merged.astype(np.uint64)
    Y = o.matmul_cp_diag(merged, L, [Hg], Dh, W, d_out, b1, gk)
    scale_in = prm.scale * prm.scale / o.primes[level - 2]
    slots = [o.decode(o.centered(o.decrypt(sk, y)[0]), scale_in) for y in Y]
    Att = np.einsum("hik,hkj->hij", P, V)
    E = np.concatenate([Att[h] for h in range(Hg)], axis=1) @ W
    assert np.abs(unpack_spatial(slots, L, k, d_out) - E).max() <= 1e-4
