"""GPU parity: every C-ABI call against the CPU oracle, bit-exact on every RNS
limb in coefficient form, at sizes that span several tiles, ragged tails and
multi-digit key switching.  Inputs are seeded and shared by both sides."""
import numpy as np
import pytest

import oracle
from paper_2508_19525_b300 import workloads as wl

from _helpers import cp_rotations, make_ctx, make_oracle, oracle_galois, pack_cols, unpack_cols

pytestmark = pytest.mark.gpu

PRMS = {"tiny": wl.TINY, "small": wl.SMALL}
SEED = 0x5EED


@pytest.fixture(scope="module", params=sorted(PRMS))
def pair(request):
    prm = PRMS[request.param]
    return prm, make_oracle(prm), make_ctx(prm)


# ------------------------------------------------------------------ transforms
@pytest.mark.parametrize("logN", [10, 12, 13, 15, 16])
def test_ntt_parity(logN):
    prm = wl.HEParams(logN, (60, 40, 50), (60, 61), 2)
    o, ctx = make_oracle(prm), make_ctx(prm)
    np_ = len(o.primes)
    data = np.concatenate([wl.random_residues(o.primes, o.N, seed=logN)[0]] * 2)
    pidx = list(range(np_)) * 2
    fwd = ctx.ntt(data, pidx)
    for r in range(0, len(pidx), 3 if logN >= 15 else 1):
        assert np.array_equal(fwd[r], o.ntt(data[r], pidx[r])), r
    back = ctx.ntt(fwd, pidx, inverse=True)
    assert np.array_equal(back, data)


@pytest.mark.parametrize("logN", [10, 12, 13, 15, 16, 17])
def test_ntt_every_pass_split_matches_the_oracle(logN):
    """The three column/row pass splits and both radices of the register
    rounds compute the same butterflies: every pair gives the oracle's forward
    transform, and the inverse restores the input; the autotuner keeps one."""
    prm = wl.HEParams(logN, (60, 40), (60,), 2)
    o, ctx = make_oracle(prm), make_ctx(prm)
    data = wl.random_residues(o.primes, o.N, seed=logN + 7)[0]
    pidx = list(range(len(o.primes)))
    ref = [o.ntt(data[r], r) for r in range(len(pidx))]
    for radix in (8, 16):
        ctx.ntt_set_radix(radix)
        for split in (-1, 0, 1):
            ctx.ntt_set_split(split)
            fwd = ctx.ntt(data, pidx)
            for r in range(len(pidx)):
                assert np.array_equal(fwd[r], ref[r]), (radix, split, r)
            assert np.array_equal(ctx.ntt(fwd, pidx, inverse=True), data), (radix, split)
    split, radix, us = ctx.ntt_autotune(16)
    want = {(rx, sp) for rx in (8, 16) for sp in ((-1, 0, 1) if logN > 12 else (0,))}
    assert set(us) == want and us[(radix, split)] == min(us.values())
    with pytest.raises(Exception):
        ctx.ntt_set_radix(4)


# ------------------------------------------------------------------ keys
def test_keygen_parity(pair):
    prm, o, ctx = pair
    rots = [1, 5, -3]
    keys = ctx.keygen(SEED, rots, relin=True)
    sk = o.keygen_secret(SEED)
    assert np.array_equal(ctx.keys_export(keys, 0), sk)
    assert np.array_equal(ctx.keys_export(keys, 1), o.keygen_relin(SEED, sk))
    for r in rots:
        assert np.array_equal(ctx.keys_export(keys, 2, r), o.keygen_galois(SEED, sk, o.galois_elt(r))), r


# ------------------------------------------------------------------ encoding
@pytest.mark.parametrize("prm,level,n", [(wl.TINY, 2, 2048), (wl.SMALL, 4, 1000), (wl.BERT_CP, 7, 16384),
                                         (wl.BERT_CC, 11, 32768), (wl.BERT_CP, 0, 5)])
def test_encode_parity(prm, level, n):
    o, ctx = make_oracle(prm), make_ctx(prm)
    z = wl.slot_vector(n, seed=n)
    for scale in (prm.scale, float(o.primes[level])):
        pt = ctx.encode(z, level, scale)
        assert np.array_equal(ctx.pt_export(pt, level), o.encode(z, level, scale))


def test_encode_rejects_overflow():
    from paper_2508_19525_b300 import blb
    ctx = make_ctx(wl.TINY)
    with pytest.raises(blb.BlbError):
        ctx.encode(np.full(16, 1e12), 2, 2.0 ** 40)


def test_deferred_encode_check_reports_overflow_at_sync():
    """With deferred checks an overflowing encoding returns at once and the
    next sync reports it (once); an encoding that fits leaves sync clean and
    gives the same limbs as the checked encoding."""
    from paper_2508_19525_b300 import blb
    prm = wl.TINY
    o, ctx = make_oracle(prm), make_ctx(prm)
    z = wl.slot_vector(o.N // 2, seed=5)
    ref = ctx.pt_export(ctx.encode(z, 2, prm.scale), 2)
    ctx.set_deferred_encode_check(True)
    pt = ctx.encode(z, 2, prm.scale)
    ctx.sync()
    assert np.array_equal(ctx.pt_export(pt, 2), ref)
    ctx.encode(np.full(16, 1e12), 2, 2.0 ** 40)
    ctx.encode(z, 2, prm.scale)  # a later good encoding does not clear the condition
    with pytest.raises(blb.BlbError) as e:
        ctx.sync()
    assert e.value.code == blb.ERR_ARG
    ctx.sync()  # cleared
    ctx.set_deferred_encode_check(False)
    with pytest.raises(blb.BlbError):
        ctx.encode(np.full(16, 1e12), 2, 2.0 ** 40)
    ctx.sync()


# ------------------------------------------------------------------ encryption
def test_encrypt_decrypt_parity(pair):
    prm, o, ctx = pair
    level = o.nQ - 1
    z = wl.slot_vector(o.N // 2, seed=7)
    keys = ctx.keygen(SEED)
    sk = o.keygen_secret(SEED)
    ct = ctx.encrypt(keys, ctx.encode(z, level), nonce=42)
    ref = o.encrypt(sk, o.encode(z, level, prm.scale), SEED, 42)
    assert np.array_equal(ctx.ct_export(ct), ref)
    coef, slots = ctx.decrypt(keys, ct)
    assert np.array_equal(coef, o.decrypt(sk, ref))
    ref_slots = o.decode(o.centered(coef[0]), prm.scale)
    assert np.max(np.abs(slots - ref_slots)) == 0.0
    assert np.max(np.abs(slots - z)) < 1e-6


# ------------------------------------------------------------------ operations
def _oracle_ct(o, sk, prm, level, seed, nonce):
    z = wl.slot_vector(o.N // 2, seed=seed)
    return o.encrypt(sk, o.encode(z, level, prm.scale), SEED, nonce), z


def test_rotate_parity(pair):
    prm, o, ctx = pair
    rots = [1, 7, -2, o.N // 4]
    keys = ctx.keygen(SEED, rots)
    sk = o.keygen_secret(SEED)
    for level in (o.nQ - 1, 1, 0):
        ref, z = _oracle_ct(o, sk, prm, level, seed=level, nonce=level)
        ct = ctx.ct_import(ref, prm.scale)
        for r in rots:
            got = ctx.ct_export(ctx.rotate(keys, ct, r))
            assert np.array_equal(got, o.rotate(ref, r, o.keygen_galois(SEED, sk, o.galois_elt(r)))), (level, r)


def test_keyswitch_parity(pair):
    prm, o, ctx = pair
    keys = ctx.keygen(SEED, [3])
    sk = o.keygen_secret(SEED)
    gk = o.keygen_galois(SEED, sk, o.galois_elt(3))
    for level in range(o.nQ):
        d = wl.random_residues(o.primes[:level + 1], o.N, seed=100 + level)[0]
        assert np.array_equal(ctx.keyswitch_coeffs(keys, 3, d), o.keyswitch(d, gk)), level


def test_rescale_parity(pair):
    prm, o, ctx = pair
    for level in range(1, o.nQ):
        for npolys in (2, 3):
            ref = wl.random_residues(o.primes[:level + 1], o.N, seed=level * 10 + npolys, polys=npolys)
            ct = ctx.ct_import(ref, prm.scale)
            ctx.rescale(ct)
            assert ct.level == level - 1
            assert np.array_equal(ctx.ct_export(ct), o.rescale(ref)), (level, npolys)


def test_tensor_relin_parity(pair):
    prm, o, ctx = pair
    keys = ctx.keygen(SEED, relin=True)
    sk = o.keygen_secret(SEED)
    level = o.nQ - 1
    a, za = _oracle_ct(o, sk, prm, level, 1, 1)
    b, zb = _oracle_ct(o, sk, prm, level, 2, 2)
    ca, cb = ctx.ct_import(a, prm.scale), ctx.ct_import(b, prm.scale)
    t = ctx.mul(None, ca, cb, relin=False)
    ref_t = o.tensor(a, b)
    assert np.array_equal(ctx.ct_export(t), ref_t)
    r = ctx.relinearize(keys, t)
    ref_r = o.relinearize(ref_t, o.keygen_relin(SEED, sk))
    assert np.array_equal(ctx.ct_export(r), ref_r)
    assert np.array_equal(ctx.ct_export(ctx.mul(keys, ca, cb)), ref_r)
    ctx.rescale(r)
    _, slots = ctx.decrypt(keys, r)
    assert np.max(np.abs(slots - za * zb)) < 1e-6


def test_add_and_mul_plain_parity(pair):
    prm, o, ctx = pair
    sk = o.keygen_secret(SEED)
    level = o.nQ - 1
    a, _ = _oracle_ct(o, sk, prm, level, 3, 3)
    b, _ = _oracle_ct(o, sk, prm, level, 4, 4)
    ca, cb = ctx.ct_import(a, prm.scale), ctx.ct_import(b, prm.scale)
    n = level + 1
    ref_add = np.zeros_like(a)
    for p in range(2):
        for i in range(n):
            ref_add[p, i] = np.array((a[p, i].astype(object) + b[p, i].astype(object)) % o.primes[i], np.uint64)
    assert np.array_equal(ctx.ct_export(ctx.add(ca, cb)), ref_add)
    z = wl.slot_vector(o.N // 2, seed=5)
    pt = ctx.encode(z, level, float(o.primes[level]))
    assert np.array_equal(ctx.ct_export(ctx.mul_plain(ca, pt)), o.mul_plain(a, o.encode(z, level, float(o.primes[level]))))


# ------------------------------------------------------------------ protocols
CP_CASES = [
    # params, m, d, d_out, b1: one ct in and out; three in, two out, ragged d and d_out
    (wl.TINY, 32, 64, 64, 8),
    (wl.SMALL, 64, 80, 40, 4),
    (wl.SMALL, 128, 40, 20, 16),
]


@pytest.mark.parametrize("case", CP_CASES)
def test_matmul_cp_parity(case):
    prm, m, d, d_out, b1 = case
    o, ctx = make_oracle(prm), make_ctx(prm)
    k = o.N // 2 // m
    G = k // b1
    level = o.nQ - 1
    X, W = wl.cp_operands(m, d, d_out, seed=m + d)
    nX = (d + k - 1) // k
    sk = o.keygen_secret(SEED)
    keys = ctx.keygen(SEED, cp_rotations(m, b1, G))
    zs = pack_cols(X, m, k, nX)
    cts = [ctx.encrypt(keys, ctx.encode(z, level), nonce=c) for c, z in enumerate(zs)]
    ref_in = np.stack([o.encrypt(sk, o.encode(z, level, prm.scale), SEED, c) for c, z in enumerate(zs)])
    for c in range(nX):
        assert np.array_equal(ctx.ct_export(cts[c]), ref_in[c])
    plan = ctx.cp_plan(m, d, W, d_out, level, b1)
    info = plan.info()
    assert (info["nX"], info["b1"], info["G"]) == (nX, b1, G)
    Y = ctx.matmul_cp_plan(keys, plan, cts)
    ref = o.matmul_cp(ref_in, m, d, W, d_out, b1, oracle_galois(o, sk, SEED, cp_rotations(m, b1, G)))
    assert len(Y) == len(ref)
    slots = []
    for e, y in enumerate(Y):
        assert y.level == level - 1 and y.scale == prm.scale
        assert np.array_equal(ctx.ct_export(y), ref[e]), e
        slots.append(ctx.decrypt(keys, y, coeffs=False)[1])
    err = np.abs(unpack_cols(slots, m, k, d_out) - X @ W)
    assert err.max() <= 1e-4
    # the one-shot form gives the same limbs
    Y2 = ctx.matmul_cp(keys, cts, m, d, W, d_out, b1)
    assert all(np.array_equal(ctx.ct_export(a), ctx.ct_export(b)) for a, b in zip(Y, Y2))


def test_he2mpc_parity(pair):
    prm, o, ctx = pair
    keys = ctx.keygen(SEED)
    sk = o.keygen_secret(SEED)
    for level in (o.nQ - 1, 0):
        ref, z = _oracle_ct(o, sk, prm, level, 9, 9)
        ct = ctx.ct_import(ref, prm.scale)
        masked, share = ctx.he2mpc(keys, ct, nonce=77)
        ref_masked, ref_share = o.he2mpc(ref, SEED, 77)
        assert np.array_equal(ctx.ct_export(masked), ref_masked)
        assert np.array_equal(share, ref_share)
        u0 = ctx.decrypt(keys, masked, slots=False)[0][0]
        q0 = o.primes[0]
        assert np.array_equal((u0.astype(object) + share.astype(object)) % q0, o.decrypt(sk, ref)[0].astype(object))


# ------------------------------------------------------------------ errors
def test_error_paths():
    from paper_2508_19525_b300 import blb
    prm = wl.TINY
    o, ctx = make_oracle(prm), make_ctx(prm)
    keys = ctx.keygen(SEED, [1])
    ct = ctx.encrypt(keys, ctx.encode(np.ones(4), 2), 0)
    with pytest.raises(blb.BlbError) as e:
        ctx.rotate(keys, ct, 2)
    assert e.value.code == blb.ERR_NO_KEY
    with pytest.raises(blb.BlbError) as e:
        ctx.relinearize(keys, ctx.mul(None, ct, ct, relin=False))
    assert e.value.code == blb.ERR_NO_KEY
    c0 = ctx.encrypt(keys, ctx.encode(np.ones(4), 0), 1)
    with pytest.raises(blb.BlbError) as e:
        ctx.rescale(c0)
    assert e.value.code == blb.ERR_LEVEL
    other = ctx.encrypt(keys, ctx.encode(np.ones(4), 2, 2.0 ** 30), 2)
    with pytest.raises(blb.BlbError) as e:
        ctx.add(ct, other)
    assert e.value.code == blb.ERR_SCALE
    with pytest.raises(blb.BlbError) as e:
        ctx.cp_plan(48, 64, np.zeros((64, 64)), 64, 2)
    assert e.value.code == blb.ERR_ARG
    with pytest.raises(blb.BlbError) as e:
        ctx.matmul_cp(keys, [ct], 32, 64, np.zeros((64, 64)), 64, 8)
    assert e.value.code == blb.ERR_NO_KEY


def test_matmul_cp_batch_equals_per_sequence():
    """The batched form (one plaintext stream for several sequences) gives the
    same limbs as one call per sequence; 5 sequences exercise the 4 + 1 split."""
    prm, m, d, d_out, b1 = wl.SMALL, 64, 80, 40, 4
    ctx = make_ctx(prm)
    k = ctx.N // 2 // m
    level = ctx.nQ - 1
    keys = ctx.keygen(SEED, cp_rotations(m, b1, k // b1))
    plan = ctx.cp_plan(m, d, wl.cp_operands(m, d, d_out, seed=1)[1], d_out, level, b1)
    seqs = []
    for s in range(5):
        X = wl.cp_operands(m, d, d_out, seed=10 + s)[0]
        seqs.append([ctx.encrypt(keys, ctx.encode(z, level), 10 * s + c)
                     for c, z in enumerate(pack_cols(X, m, k, (d + k - 1) // k))])
    singles = [ctx.matmul_cp_plan(keys, plan, X) for X in seqs]
    # both kernels of batched plaintext products: mma.sync (1) and tcgen05 (2),
    # at 4 + 1 and at 2 sequences per launch
    for kind in (0, 1, 2):
        ctx.set_batch_mac(kind)
        for group in (seqs, seqs[:2]):
            batched = ctx.matmul_cp_batch(keys, plan, group)
            for s in range(len(group)):
                for a, b in zip(batched[s], singles[s]):
                    assert np.array_equal(ctx.ct_export(a), ctx.ct_export(b)), (kind, len(group), s)
    ctx.set_batch_mac(0)
