"""Shared test helpers: packing of matrices into slot vectors (spatial-first,
Sec. 4.2.1) and construction of matching oracle / GPU objects."""
import numpy as np

import oracle
from paper_2508_19525_b300 import workloads as wl


def make_oracle(prm):
    return oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum)


def make_ctx(prm):
    from paper_2508_19525_b300 import blb
    return blb.Context(prm.logN, prm.q_bits, prm.p_bits, prm.dnum, prm.scale)


def pack_cols(X, m, k, n_cts):
    """ct c holds X[i, c k + b] at slot i + m b (zero past the last column)."""
    d = X.shape[1]
    out = np.zeros((n_cts, m * k))
    for c in range(n_cts):
        for b in range(k):
            col = c * k + b
            if col < d:
                out[c, b * m:(b + 1) * m] = X[:, col]
    return out


def unpack_cols(zs, m, k, d_out):
    Y = np.zeros((m, d_out))
    for e, z in enumerate(zs):
        for b in range(k):
            col = e * k + b
            if col < d_out:
                Y[:, col] = z[b * m:(b + 1) * m]
    return Y


def cp_rotations(m, b1, G):
    return [b * m for b in range(1, b1)] + [g * b1 * m for g in range(1, G)]


def oracle_galois(o, sk, seed, rots):
    return {o.galois_elt(r): o.keygen_galois(seed, sk, o.galois_elt(r)) for r in rots}


def assert_limbs_consistent(coeffs, primes, bound_bits=56):
    """The limbs of a decrypted polynomial (level+1, N; coefficient form) must
    be the residues of one small integer: limb 0 centered mod q_0, reduced mod
    q_i, equals limb i for every i (a ciphertext with a wrong residue in any
    limb decrypts to an unrelated value there).  The message + noise stays
    below 2^bound_bits in magnitude."""
    q0 = int(primes[0])
    c0 = coeffs[0].astype(np.int64)
    v = np.where(coeffs[0] > q0 // 2, c0 - q0, c0)
    assert np.abs(v).max() < (1 << bound_bits)
    for i in range(1, coeffs.shape[0]):
        qi = np.int64(primes[i])
        assert np.array_equal(np.mod(v, qi).astype(np.uint64), coeffs[i]), f"limb {i} disagrees with limb 0"
