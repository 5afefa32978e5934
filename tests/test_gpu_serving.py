"""Cross-client batching on the GPU: blb_matmul_cp_multi gives each client the
limbs of its own single product, and a request served among others (arriving
at random, batched with other clients' requests at other stages) returns the
same limbs as when it is served alone; its decrypted result matches FP64.
Both engines: whole requests padded to a bucket, and token-chunked requests."""
import numpy as np
import pytest

from paper_2508_19525_b300 import workloads as wl
from paper_2508_19525_b300.serving import ChunkEngine, GpuEngine, Request, Server, bucket

from _helpers import cp_rotations, make_ctx, pack_cols

pytestmark = pytest.mark.gpu
D, D_QKV = 64, 192
BUCKETS = (16, 32)


def test_multi_key_product_equals_per_client_products():
    prm = wl.SMALL
    ctx = make_ctx(prm)
    m, b1 = 32, 8
    k = ctx.N // 2 // m
    level = ctx.nQ - 1
    rots = cp_rotations(m, b1, k // b1)
    W = wl.uniform((D, D_QKV), seed=5)
    plan = ctx.cp_plan(m, D, W, D_QKV, level, b1)
    keys = [ctx.keygen(40 + i, rots) for i in range(3)]
    Xs = []
    for i in range(3):
        X = wl.uniform((m, D), seed=60 + i)
        Xs.append([ctx.encrypt(keys[i], ctx.encode(z, level), 10 * i + c)
                   for c, z in enumerate(pack_cols(X, m, k, (D + k - 1) // k))])
    multi = ctx.matmul_cp_multi(keys, plan, Xs)
    for i in range(3):
        single = ctx.matmul_cp_plan(keys[i], plan, Xs[i])
        for a, b in zip(multi[i], single):
            assert np.array_equal(ctx.ct_export(a), ctx.ct_export(b))


def _server(ctx, plans, keep=False):
    eng = GpuEngine(ctx, plans, ctx.nQ - 1, D, D_QKV, keep_outputs=keep)
    return Server(eng, budget_bytes=8 << 30, max_batch=4)


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for i in range(n):
        t += rng.exponential(0.005)
        seq = int(rng.integers(8, max(BUCKETS) + 1))
        out.append(Request(rid=i, client_seed=500 + i, model="a" if i % 2 else "b", seq=seq,
                           m=bucket(seq, BUCKETS), arrival=t, X=wl.uniform((seq, D), seed=900 + i)))
    return out


def test_result_alone_equals_result_in_the_mix():
    prm = wl.SMALL
    ctx = make_ctx(prm)
    level = ctx.nQ - 1
    weights = {name: (wl.uniform((D, D_QKV), seed=s), wl.uniform((D, D), seed=s + 1))
               for name, s in (("a", 11), ("b", 21))}
    plans = {}
    for name, (Wq, Wo) in weights.items():
        for m in BUCKETS:
            k = ctx.N // 2 // m
            b1 = 1
            while b1 * b1 < k:
                b1 *= 2
            qkv = ctx.cp_plan(m, D, Wq, D_QKV, level, b1)
            o = ctx.cp_plan(m, D, Wo, D, level - 1, b1)
            plans[(name, m)] = (qkv, o, cp_rotations(m, b1, k // b1))
    mix = _requests(6, seed=3)
    srv = _server(ctx, plans, keep=True)
    done = srv.run(mix)
    assert len(done) == 6 and max(n for _, n in srv.iterations) > 1
    for r in mix:
        alone = _requests(6, seed=3)[r.rid]
        _server(ctx, plans).run([alone])
        assert np.array_equal(r.state["p0"], alone.state["p0"]), r.rid
        assert np.array_equal(r.state["shares"], alone.state["shares"]), r.rid
        # the unmasked outputs decrypt to the FP64 products: QKV output
        # ciphertexts nX.. (columns nX k ...) and the output projection
        Wq, Wo = weights[r.model]
        m, k = r.m, ctx.N // 2 // r.m
        nX, nY = (D + k - 1) // k, (D_QKV + k - 1) // k
        Xp = np.zeros((m, D))
        Xp[: r.seq] = r.X
        Yq = Xp @ Wq
        slots = np.stack([ctx.decrypt(r.state["keys"], c, coeffs=False)[1] for c in r.state["outs"]])
        got = np.concatenate([z.reshape(k, m).T for z in slots], axis=1)
        got_q = got[:, : D_QKV - nX * k]
        got_o = got[:, (nY - nX) * k: (nY - nX) * k + D]
        assert np.abs(got_q - Yq[:, nX * k:]).max() <= 1e-4
        assert np.abs(got_o - Yq[:, :D] @ Wo).max() <= 1e-4


@pytest.mark.parametrize("m,b1", [(16, 8), (64, 8)])
def test_chunked_result_alone_equals_result_in_the_mix(m, b1):
    """Requests of 8-60 tokens cut into m-row chunks (16 rows: 1-4 chunks of one
    input ciphertext; 64 rows: one chunk of two input ciphertexts, as the
    serving benchmark's larger chunks have several; one plan pair per model),
    served in a mix with up to 3 chunks per cross-client product and alone:
    same masked limbs and shares; every chunk's outputs decrypt to the FP64
    products."""
    prm = wl.SMALL
    ctx = make_ctx(prm)
    level = ctx.nQ - 1
    k = ctx.N // 2 // m
    weights = {name: (wl.uniform((D, D_QKV), seed=s), wl.uniform((D, D), seed=s + 1))
               for name, s in (("a", 31), ("b", 41))}
    plans = {name: (ctx.cp_plan(m, D, Wq, D_QKV, level, b1), ctx.cp_plan(m, D, Wo, D, level - 1, b1),
                    cp_rotations(m, b1, k // b1))
             for name, (Wq, Wo) in weights.items()}

    def reqs():
        rng = np.random.default_rng(8)
        t, out = 0.0, []
        for i in range(6):
            t += rng.exponential(0.005)
            seq = int(rng.integers(8, 61))
            out.append(Request(rid=i, client_seed=700 + i, model="a" if i % 2 else "b", seq=seq, m=m,
                               arrival=t, X=wl.uniform((seq, D), seed=950 + i)))
        return out

    def server(keep=False):
        return Server(ChunkEngine(ctx, plans, level, D, D_QKV, m, group=3, keep_outputs=keep),
                      budget_bytes=8 << 30, max_batch=4)

    mix = reqs()
    srv = server(keep=True)
    done = srv.run(mix)
    assert len(done) == 6 and max(n for _, n in srv.iterations) > 1
    nX, nY = (D + k - 1) // k, (D_QKV + k - 1) // k
    assert nX == max(1, D // k)          # two input ciphertexts per chunk at 64 rows
    for r in mix:
        alone = reqs()[r.rid]
        server().run([alone])
        assert np.array_equal(r.state["p0"], alone.state["p0"]), r.rid
        assert np.array_equal(r.state["shares"], alone.state["shares"]), r.rid
        Wq, Wo = weights[r.model]
        per = nY - nX + -(-D // k)          # QKV outputs past the first nX, then W_O's
        n_ch = -(-r.seq // m)
        assert len(r.state["outs"]) == n_ch * per
        Xp = np.zeros((n_ch * m, D))
        Xp[: r.seq] = r.X
        for c in range(n_ch):
            Yq = Xp[c * m:(c + 1) * m] @ Wq
            cts = r.state["outs"][c * per:(c + 1) * per]
            slots = np.stack([ctx.decrypt(r.state["keys"], x, coeffs=False)[1] for x in cts])
            got = np.concatenate([z.reshape(k, m).T for z in slots], axis=1)
            got_q = got[:, : D_QKV - nX * k]
            got_o = got[:, (nY - nX) * k: (nY - nX) * k + D]
            assert np.abs(got_q - Yq[:, nX * k:]).max() <= 1e-4, (r.rid, c)
            assert np.abs(got_o - Yq[:, :D] @ Wo).max() <= 1e-4, (r.rid, c)
