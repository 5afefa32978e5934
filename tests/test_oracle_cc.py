"""Pins for the oracle's matmul_cc (Sec. 5.1, App. C.1): the encrypted
three-step protocol decrypts to the FP64 product A_h B_h of every head in
diagonal packing, within the 1e-4 bound, on attention-shaped operands."""
import numpy as np
import pytest

import cc_schedule as cs
import oracle
from paper_2508_19525_b300 import workloads as wl


def cc_rotations(L, Hg, Kc, b1s1, b1s2, s):
    G1, G2 = Kc // b1s1, L // b1s2
    r = set()
    r.update(range(1, b1s1))
    r.update(b0 - L for b0 in range(b1s1))
    r.update(g1 * b1s1 for g1 in range(1, G1))
    r.update(range(1, b1s2))
    r.update(b - L for b in range(b1s2))
    r.update(-g * b1s2 for g in range(1, G2))
    r.update(cs.step3_rotation(t, L, Hg, Kc, b1s2, s) for t in range(1, L))
    r.discard(0)
    return sorted(r)


def run_cc(o, A, B, L, Hg, b1s1, b1s2, seed=0):
    prm_scale = 2.0 ** 40
    s = o.N // 2
    Kc = s // (L * Hg)
    R = A.shape[2]
    n_c = -(-R // Kc)
    level = o.nQ - 1
    sk = o.keygen_secret(seed)
    Az = cs.pack(A, L, Hg, Kc, n_c, rows=False)
    Bz = cs.pack(B, L, Hg, Kc, n_c, rows=True)
    Acts = np.stack([o.encrypt(sk, o.encode(z, level, prm_scale), seed, c) for c, z in enumerate(Az)])
    Bcts = np.stack([o.encrypt(sk, o.encode(z, level, prm_scale), seed, 100 + c) for c, z in enumerate(Bz)])
    gal = {o.galois_elt(r): o.keygen_galois(seed, sk, o.galois_elt(r))
           for r in cc_rotations(L, Hg, Kc, b1s1, b1s2, s)}
    rk = o.keygen_relin(seed, sk)
    C = o.matmul_cc(Acts, Bcts, L, Hg, b1s1, b1s2, gal, rk)
    out_scale = prm_scale * prm_scale / o.primes[level - 2]
    zs = np.stack([o.decode(o.centered(o.decrypt(sk, c)[0]), out_scale) for c in C])
    return cs.unpack_diagonals(zs, L, Hg, Kc), C, sk, Acts, Bcts, gal, rk


@pytest.mark.parametrize("R,kind", [(16, "qk"), (32, "qk"), (16, "pv")])
def test_matmul_cc_decrypts_to_fp64_product(R, kind):
    o = oracle.Oracle(12, wl.SMALL.q_bits, wl.SMALL.p_bits, wl.SMALL.dnum)
    L, Hg, b1s1, b1s2 = 32, 4, 4, 8
    Q, K, V, P = wl.attention_operands(L, Hg, R, seed=R)
    if kind == "qk":
        A, B = Q, np.transpose(K, (0, 2, 1))          # Q_h K_h^T
    else:
        # Softmax(.) x V_h: A = P_h (L x L), B = V_h zero-padded to L x L (Sec. 5.2)
        A = P
        B = np.concatenate([V, np.zeros((Hg, L, L - V.shape[2]))], axis=2)
    got, *_ = run_cc(o, A, B, L, Hg, b1s1, b1s2)
    ref = np.einsum("hik,hkj->hij", A, B)
    err = np.abs(got - ref)
    assert err.max() <= 1e-4
    assert np.mean(err ** 2) < 1e-11


def test_cc_rotation_count_formula():
    o = oracle.Oracle(12, wl.SMALL.q_bits, wl.SMALL.p_bits, wl.SMALL.dnum)
    # matches the slot-level schedule's count (tests/test_cc_schedule.py)
    assert o.cc_num_rotations(2, 32, 16, 4, 8) == 2 * ((3 + 4 + 3) + (7 + 8 + 3)) + 31
    assert o.cc_num_rotations(1, 128, 64, 8, 8) == (7 + 8 + 7) + (7 + 8 + 15) + 127
