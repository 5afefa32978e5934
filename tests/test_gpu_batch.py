"""The batched encode / encrypt / CKKS->MPC masking / decrypt calls give, member
for member, the limbs of the single calls (same nonces, same Philox streams)."""
import numpy as np
import pytest

from paper_2508_19525_b300 import workloads as wl

from _helpers import make_ctx

pytestmark = pytest.mark.gpu
SEED = 0xBA7C


@pytest.mark.parametrize("count", [1, 5])
def test_batched_calls_equal_single_calls(count):
    prm = wl.SMALL
    ctx = make_ctx(prm)
    keys = ctx.keygen(SEED, [1], relin=True)
    level = ctx.nQ - 1
    vals = np.stack([wl.slot_vector(ctx.N // 2, seed=30 + k) for k in range(count)])
    nonces = [1000 + 7 * k for k in range(count)]

    pts = ctx.encode_batch(vals, level)
    singles = [ctx.encode(v, level) for v in vals]
    for a, b in zip(pts, singles):
        assert np.array_equal(ctx.pt_export(a, level), ctx.pt_export(b, level))

    cts = ctx.encrypt_batch(keys, pts, nonces)
    ref = [ctx.encrypt(keys, p, nc) for p, nc in zip(singles, nonces)]
    for a, b in zip(cts, ref):
        assert np.array_equal(ctx.ct_export(a), ctx.ct_export(b))

    # decryption: 2-polynomial ciphertexts and 3-polynomial products
    coeffs, slots = ctx.decrypt_batch(keys, cts, slots=True)
    for k, c in enumerate(ref):
        c1, s1 = ctx.decrypt(keys, c)
        assert np.array_equal(coeffs[k], c1)
        assert np.array_equal(slots[k], s1)
    prods = [ctx.mul(keys, c, c, relin=False) for c in cts]
    coeffs3, _ = ctx.decrypt_batch(keys, prods)
    for k, c in enumerate(prods):
        assert np.array_equal(coeffs3[k], ctx.decrypt(keys, c, slots=False)[0])

    # masking of ciphertexts at different levels
    mixed = [ctx.rescale(ctx.encrypt(keys, ctx.encode(v, level), 77 + k)) if k % 2 else c
             for k, (v, c) in enumerate(zip(vals, cts))]
    masked, shares = ctx.he2mpc_batch(keys, mixed, nonces)
    for k, c in enumerate(mixed):
        m1, s1 = ctx.he2mpc(keys, c, nonces[k])
        assert masked[k].level == 0
        assert np.array_equal(ctx.ct_export(masked[k]), ctx.ct_export(m1))
        assert np.array_equal(shares[k], s1)


def test_batch_rejects_mixed_levels():
    from paper_2508_19525_b300 import blb
    ctx = make_ctx(wl.SMALL)
    keys = ctx.keygen(SEED)
    level = ctx.nQ - 1
    v = wl.slot_vector(ctx.N // 2, seed=1)
    a = ctx.encrypt(keys, ctx.encode(v, level), 1)
    b = ctx.encrypt(keys, ctx.encode(v, level - 1), 2)
    with pytest.raises(blb.BlbError):
        ctx.decrypt_batch(keys, [a, b])
    with pytest.raises(blb.BlbError):
        ctx.encrypt_batch(keys, [ctx.encode(v, level), ctx.encode(v, level - 1)], [1, 2])


# the two refused captures end empty (the library refuses before it launches)
@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_masking_and_decryption_replay_from_a_graph():
    """The batched masking and decryption captured into a CUDA graph (their
    host tables go to buffers the context keeps, so a replay never reads
    freed host memory): a replay gives the eager P1 shares and P0
    coefficients.  A host output buffer and encoding are refused during
    capture."""
    import torch
    from paper_2508_19525_b300 import blb
    prm = wl.SMALL
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, prm.dnum, prm.scale, stream=torch.cuda.Stream())
    keys = ctx.keygen(SEED, [1])
    level = ctx.nQ - 1
    vals = np.stack([wl.slot_vector(ctx.N // 2, seed=70 + k) for k in range(3)])
    cts = ctx.encrypt_batch(keys, ctx.encode_batch(vals, level), [10, 11, 12])

    def fn(share, p0):
        masked, _ = ctx.he2mpc_batch(keys, cts, [20, 21, 22], share_out=share)
        ctx.decrypt_batch(keys, masked, coeff_out=p0)
        return masked

    u64 = dict(dtype=torch.uint64, device="cuda")
    share_e, p0_e = torch.zeros((3, ctx.N), **u64), torch.zeros((3, ctx.N), **u64)
    fn(share_e, p0_e)
    ctx.sync()
    share_g, p0_g = torch.zeros((3, ctx.N), **u64), torch.zeros((3, ctx.N), **u64)
    graph, masked = ctx.capture(lambda: fn(share_g, p0_g), warmup=False)
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(share_g.cpu().numpy(), share_e.cpu().numpy())
    assert np.array_equal(p0_g.cpu().numpy(), p0_e.cpu().numpy())
    with pytest.raises(blb.BlbError):  # P1's shares into a host array
        ctx.capture(lambda: ctx.he2mpc_batch(keys, cts, [30, 31, 32]), warmup=False)
    with pytest.raises(blb.BlbError):  # encoding reads its overflow flag on the host
        ctx.capture(lambda: ctx.encode_batch(vals, level), warmup=False)
