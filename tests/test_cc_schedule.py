"""The matmul_cc schedule (Sec. 5.1, App. C.1) on plaintext slots: the
three-step protocol with multi-head packing and baby-step giant-step splits must
reproduce A_h B_h for every head in diagonal packing (Observations 1-2 of
Sec. 5.1 make this an exact identity), for Q K^T-shaped (R < L) and
Softmax x V-shaped (R = L) operands."""
import numpy as np
import pytest

import cc_schedule as cs


@pytest.mark.parametrize("s,L,Hg,R,b1s1,b1s2", [
    (32, 4, 2, 8, 2, 2),        # the paper's toy size L = 4 (Fig. 7), two heads
    (2048, 32, 4, 16, 4, 8),    # Q K^T shaped: R < L, one input ciphertext per operand
    (2048, 32, 4, 32, 4, 8),    # Softmax x V shaped: R = L, two input ciphertexts
    (2048, 32, 2, 32, 8, 4),    # other head group and splits
    (2048, 16, 8, 48, 16, 1),   # no giant steps in step 2
])
def test_schedule_reproduces_matrix_product(s, L, Hg, R, b1s1, b1s2):
    Kc = s // (L * Hg)
    n_c = -(-R // Kc)
    rng = np.random.default_rng(s + L + Hg + R)
    A = rng.uniform(-1, 1, size=(Hg, L, R))
    B = rng.uniform(-1, 1, size=(Hg, R, L))
    Aslots = cs.pack(A, L, Hg, Kc, n_c, rows=False)
    Bslots = cs.pack(B, L, Hg, Kc, n_c, rows=True)
    C, nrot = cs.simulate(Aslots, Bslots, L, Hg, b1s1, b1s2)
    got = cs.unpack_diagonals(C, L, Hg, Kc)
    ref = np.einsum("hik,hkj->hij", A, B)
    assert np.max(np.abs(got - ref)) < 1e-12
    G1, G2 = Kc // b1s1, L // b1s2
    step1 = (b1s1 - 1) + (b1s1 if G1 > 1 else b1s1 - 1) + (G1 - 1)
    step2 = (b1s2 - 1) + b1s2 + (G2 - 1)
    assert nrot == n_c * (step1 + step2) + (L - 1)
