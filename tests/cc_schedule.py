"""Slot-level model of the matmul_cc schedule (Sec. 5.1, App. C.1) used by the
tests: plaintext slot vectors in FP64, left rotation = np.roll(v, -x),
HomMul = element-wise product.  It fixes the packing and the schedule that the
oracle and the CUDA path both implement, and lets the tests check the
schedule's algebra against the plain matrix product before any encryption.

Packing (multi-head, Sec. 5.1 "Multi-Head Optimization"): s slots form blocks of
L slots; block beta = h + Hg * kappa holds, for head h and column index
k = c * Kc + kappa of input ciphertext c, the column A_h[:, k] (spatial-first)
or the row B_h[k, :] (reduce-first), element i at slot beta * L + i;
Kc = s / (L * Hg).  Output ciphertext j holds diagonals
delta = j * Kc + kappa' of C_h = A_h B_h at block h + Hg * kappa', element i being
C_h[i, (i + delta) mod L] (diagonal packing).
"""
import numpy as np


def rot(v, x):
    """Rot_l^x: left rotation by x slots."""
    return np.roll(v, -int(x))


def geometry(s, L, Hg):
    Kc = s // (L * Hg)
    slot = np.arange(s)
    beta, i = slot // L, slot % L
    return Kc, beta % Hg, beta // Hg, i


def pack(mats, L, Hg, Kc, n_c, rows):
    """mats: (Hg, L, R) for A (columns) or (Hg, R, L) for B (rows = True)."""
    s = L * Hg * Kc
    out = np.zeros((n_c, s))
    for c in range(n_c):
        for kappa in range(Kc):
            k = c * Kc + kappa
            for h in range(Hg):
                beta = h + Hg * kappa
                R = mats.shape[1] if rows else mats.shape[2]
                if k < R:
                    out[c, beta * L:(beta + 1) * L] = mats[h, k, :] if rows else mats[h, :, k]
    return out


def unpack_diagonals(C, L, Hg, Kc):
    """C: (L/Kc, s) -> (Hg, L, L)."""
    out = np.zeros((Hg, L, L))
    for j in range(C.shape[0]):
        for kappa in range(Kc):
            delta = j * Kc + kappa
            for h in range(Hg):
                beta = h + Hg * kappa
                blk = C[j, beta * L:(beta + 1) * L]
                for i in range(L):
                    out[h, i, (i + delta) % L] = blk[i]
    return out


def masks(s, L, Hg, b1s1, b1s2):
    """All plaintext masks of the schedule, as slot vectors:
    m1[(g1, b0)] = (lo, hi) for step 1, m2[(g, b)] = (lo, hi) for step 2 (both
    already rotated right by the giant step), m3[t] = list of (j, mask)."""
    Kc, h, kap, i = geometry(s, L, Hg)
    G1, G2 = Kc // b1s1, L // b1s2
    m1 = {}
    for g1 in range(G1):
        for b0 in range(b1s1):
            kappa = g1 * b1s1 + b0
            lo = ((kap == kappa) & (i < L - kappa)).astype(float)
            hi = ((kap == kappa) & (i >= L - kappa)).astype(float)
            m1[(g1, b0)] = (rot(lo, -g1 * b1s1), rot(hi, -g1 * b1s1))
    m2 = {}
    for g in range(G2):
        for b in range(b1s2):
            t = g * b1s2 + b
            lo = (i < L - t).astype(float)
            hi = (i >= L - t).astype(float)
            m2[(g, b)] = (rot(lo, -g * b1s2), rot(hi, -g * b1s2))
    m3 = {}
    for t in range(L):
        kappa_src = (kap - t) % Kc
        delta = (t + kappa_src) % L
        j = delta // Kc
        m3[t] = [(jj, (j == jj).astype(float)) for jj in sorted(set(j.tolist()))]
    return m1, m2, m3


def step3_rotation(t, L, Hg, Kc, b1s2, s):
    g = t // b1s2
    return (g * b1s2 - (t % Kc) * Hg * L) % s


def simulate(Aslots, Bslots, L, Hg, b1s1, b1s2):
    """The schedule on plaintext slots.  Returns (C (L/Kc, s), rotation count)."""
    n_c, s = Aslots.shape
    Kc = s // (L * Hg)
    assert Kc * L * Hg == s and L % Kc == 0 and Kc % b1s1 == 0 and L % b1s2 == 0
    G1, G2 = Kc // b1s1, L // b1s2
    m1, m2, m3 = masks(s, L, Hg, b1s1, b1s2)
    nrot = 0
    # step 1: B'[c] block kappa holds B[k, (i + kappa) mod L]
    Bp = np.zeros_like(Bslots)
    for c in range(n_c):
        baby_lo = {b0: rot(Bslots[c], b0) for b0 in range(b1s1)}
        baby_hi = {b0: rot(Bslots[c], b0 - L) for b0 in range(b1s1)}
        nrot += (b1s1 - 1) + (b1s1 if G1 > 1 else b1s1 - 1)
        for g1 in range(G1):
            inner = sum(m1[(g1, b0)][0] * baby_lo[b0] + m1[(g1, b0)][1] * baby_hi[b0] for b0 in range(b1s1))
            Bp[c] += rot(inner, g1 * b1s1)
            nrot += g1 > 0
    # step 2: U[(g, b)] = sum_c Rot^{-g b1}(A_c) (.) V_{g,b}(B'_c)
    U = {}
    for c in range(n_c):
        blo = {b: rot(Bp[c], b) for b in range(b1s2)}
        bhi = {b: rot(Bp[c], b - L) for b in range(b1s2)}
        Ag = {g: rot(Aslots[c], -g * b1s2) for g in range(G2)}
        nrot += (b1s2 - 1) + b1s2 + (G2 - 1)
        for g in range(G2):
            for b in range(b1s2):
                V = m2[(g, b)][0] * blo[b] + m2[(g, b)][1] * bhi[b]
                U[(g, b)] = U.get((g, b), 0) + Ag[g] * V
    # step 3: one rotation per t, then route blocks to output ciphertexts
    C = np.zeros((L // Kc, s))
    for t in range(L):
        g, b = t // b1s2, t % b1s2
        r = step3_rotation(t, L, Hg, Kc, b1s2, s)
        Rt = rot(U[(g, b)], r)
        nrot += r != 0
        for j, m in m3[t]:
            C[j] += m * Rt
    return C, nrot
