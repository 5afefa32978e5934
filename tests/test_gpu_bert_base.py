"""The BERT-base fused linear step exactly as the benchmark times it (N = 2^15,
8 primes, 3 special primes, dnum 3, X 128x768 @ W_QKV 768x2304 then the first
768 columns @ W_O 768x768, b1 = 16, masking and P0's decryption of the 18
outputs): every decrypted output against FP64 within 1e-4, and, limb for limb
against the oracle, what the oracle computes one by one at this size: the
step's encrypted inputs, the masked outputs and P1's shares of the step (all
18), P0's decryption of them, and a narrower matmul_cp (128 x 128 @ 128 x 128)
on the same ring, level, primes, dnum, m and b1.  The packed batch form (two
sequences per ciphertext) against FP64, and a narrow product in its geometry
against the oracle."""
import numpy as np
import pytest

from paper_2508_19525_b300 import workloads as wl

from _helpers import (assert_limbs_consistent, cp_rotations, make_ctx, make_oracle, oracle_galois, pack_cols,
                      unpack_cols)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    import torch
    import bench
    w = bench.Workload(torch.device("cuda", 0))
    n0 = w.nonce
    Y, O, cts = w.step(keep=True)
    torch.cuda.synchronize()
    return bench, w, n0, Y, O, cts


def test_step_outputs_match_fp64(run):
    bench, w, _, Y, O, _ = run
    ctx, keys = w.ctx, w.keys
    assert len(Y) == 18 and len(O) == 6
    got_qkv = bench.unpack_columns(np.stack([ctx.decrypt(keys, y, coeffs=False)[1] for y in Y]), bench.M, w.k,
                                   bench.D_QKV)
    got_o = bench.unpack_columns(np.stack([ctx.decrypt(keys, y, coeffs=False)[1] for y in O]), bench.M, w.k,
                                 bench.D_O)
    assert np.abs(got_qkv - w.ref_qkv).max() <= 1e-4
    assert np.abs(got_o - w.ref_o).max() <= 1e-4
    # the slots above decode limb 0 only: every other limb of every output must
    # hold the residues of the same decrypted integers
    primes = ctx.primes
    for y in Y + O:
        assert_limbs_consistent(ctx.decrypt(keys, y, slots=False)[0], primes)


def test_step_inputs_masks_and_shares_match_the_oracle(run):
    bench, w, n0, Y, O, cts = run
    o = make_oracle(wl.BERT_CP)
    sk = o.keygen_secret(0)  # the workload's key seed
    Z = w.Zhost.numpy()
    for c in range(w.n_in):
        ref = o.encrypt(sk, o.encode(Z[c], bench.LEVEL, wl.BERT_CP.scale), 0, n0 + 1 + c)
        assert np.array_equal(w.ctx.ct_export(cts[c]), ref), c
    outs = Y[w.n_in:] + O
    p0, p1 = w.p0_dev.cpu().numpy(), w.p1_dev.cpu().numpy()
    for e, y in enumerate(outs):
        masked, share = o.he2mpc(w.ctx.ct_export(y), 0, n0 + 1 + w.n_in + e)
        assert np.array_equal(p1[e], share), e
        assert np.array_equal(p0[e], o.decrypt(sk, masked)[0]), e


def test_narrow_matmul_cp_at_the_step_parameters_matches_the_oracle():
    prm = wl.BERT_CP
    o, ctx = make_oracle(prm), make_ctx(prm)
    m, d, d_out, b1 = 128, 128, 128, 16
    k = o.N // 2 // m
    G = k // b1
    level = o.nQ - 1
    X, W = wl.cp_operands(m, d, d_out, seed=77)
    sk = o.keygen_secret(3)
    rots = cp_rotations(m, b1, G)
    keys = ctx.keygen(3, rots)
    zs = pack_cols(X, m, k, 1)
    ct = ctx.encrypt(keys, ctx.encode(zs[0], level), nonce=5)
    ref_in = o.encrypt(sk, o.encode(zs[0], level, prm.scale), 3, 5)
    assert np.array_equal(ctx.ct_export(ct), ref_in)
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)
    Y = ctx.matmul_cp_plan(keys, plan, [ct])
    ref = o.matmul_cp(ref_in[None], m, d, W, d_out, b1, oracle_galois(o, sk, 3, rots))
    assert len(Y) == len(ref) == 1
    assert np.array_equal(ctx.ct_export(Y[0]), ref[0])
    got = unpack_cols([ctx.decrypt(keys, Y[0], coeffs=False)[1]], m, k, d_out)
    assert np.abs(got - X @ W).max() <= 1e-4


def test_nine_sequence_batch_at_the_step_parameters_equals_single_calls():
    """matmul_cp over 9 sequences in one batched call (an 8-sequence launch and
    a 1-sequence launch) gives every sequence the limbs of its own call, at the
    step's ring, primes, dnum, m, b1 and 96 plaintext terms per output (where a
    tile of the 8-sequence launch holds one coefficient)."""
    prm = wl.BERT_CP
    ctx = make_ctx(prm)
    m, d, d_out, b1 = 128, 768, 128, 16
    k = ctx.N // 2 // m
    level = ctx.nQ - 1
    keys = ctx.keygen(3, cp_rotations(m, b1, k // b1))
    _, W = wl.cp_operands(m, d, d_out, seed=78)
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)
    seqs = []
    for s in range(9):
        X = wl.cp_operands(m, d, d_out, seed=90 + s)[0]
        seqs.append([ctx.encrypt(keys, ctx.encode(z, level), 100 * s + c)
                     for c, z in enumerate(pack_cols(X, m, k, d // k))])
    batched = ctx.matmul_cp_batch(keys, plan, seqs)
    for s, cts in enumerate(seqs):
        single = ctx.matmul_cp_plan(keys, plan, cts)
        assert len(batched[s]) == len(single)
        for a, b in zip(batched[s], single):
            assert np.array_equal(ctx.ct_export(a), ctx.ct_export(b)), s


@pytest.mark.parametrize("per", [2, 4])
def test_several_sequences_per_ciphertext_chain_matches_fp64(run, per):
    """The benchmark's packed batch forms (two or four 128-token sequences per
    ciphertext, m = 256 or 512, k = 64 or 32): QKV then W_O on the QKV output,
    every sequence of a packed input within 1e-4 of FP64."""
    bench, w, _, _, _, _ = run
    try:
        assert w.packed(per) == bench.D // (w.N // 2 // (per * bench.M))
        assert w.packed_accuracy() <= 1e-4
    finally:
        w.free_packed()


def test_narrow_two_sequence_matmul_cp_matches_the_oracle():
    """A narrower product in the packed form's geometry (m = 256 rows, k = 64
    columns per ciphertext, b1 = 8) at the step's ring, level, primes and dnum:
    two sequences' rows in one ciphertext, limb for limb against the oracle."""
    prm = wl.BERT_CP
    o, ctx = make_oracle(prm), make_ctx(prm)
    m, d, d_out, b1 = 256, 64, 64, 8
    k = o.N // 2 // m
    level = o.nQ - 1
    X, W = wl.cp_operands(m, d, d_out, seed=79)
    sk = o.keygen_secret(4)
    rots = cp_rotations(m, b1, k // b1)
    keys = ctx.keygen(4, rots)
    zs = pack_cols(X, m, k, 1)
    ct = ctx.encrypt(keys, ctx.encode(zs[0], level), nonce=6)
    ref_in = o.encrypt(sk, o.encode(zs[0], level, prm.scale), 4, 6)
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)
    Y = ctx.matmul_cp_plan(keys, plan, [ct])
    ref = o.matmul_cp(ref_in[None], m, d, W, d_out, b1, oracle_galois(o, sk, 4, rots))
    assert len(Y) == len(ref) == 1
    assert np.array_equal(ctx.ct_export(Y[0]), ref[0])
    got = unpack_cols([ctx.decrypt(keys, Y[0], coeffs=False)[1]], m, k, d_out)
    assert np.abs(got - X @ W).max() <= 1e-4
