"""Segments 3-6 of the hybrid encoder layer, limb for limb against the oracle.
Each HE segment of BertLayer (layer.py) runs on the GPU on seeded encryptions;
the oracle runs the same operations on its own encryptions of the same values
(same keys and nonces, so the inputs are equal limb for limb):

* segment 3 (the big context): P times the reciprocal row sums (smul_cc), P V
  (matmul_cc, Sec. 5.1), the merge of complementary diagonals, Concat(Att) W_O
  (the diagonal-input matmul_cp, App. C.2), the residual and the LayerNorm head;
* segment 4: the LN1 tail (smul_cc, ewmul_cp, ewadd_cp), W_1 and the two GeLU
  polynomial pieces; segment 6, the LN2 tail, is the same tail;
* segment 5: W_2, the residual and the LayerNorm head.

The oracle side restates each element-wise operation from its definition: a
ct x ct product is the tensor product then relinearization; a rescale divides
by the last prime; mul_const multiplies by the constant encoded at scale
target x q_l / scale and rescales; add_plain adds the encoding to the first
polynomial; drop_level keeps the first limbs; add / sub work limb by limb.
Scales follow the library's documented rules; the test tracks them itself and
checks them against the GPU ciphertexts' metadata before encoding with them."""
import numpy as np
import pytest

from paper_2508_19525_b300 import layer as ly
from paper_2508_19525_b300 import workloads as wl

from _helpers import make_ctx, make_oracle

pytestmark = pytest.mark.gpu
SEED = 0x5E6
P_SMALL = wl.HEParams(12, (60,) + (40,) * 7, (60,) * 3, 3)
P_BIG = wl.HEParams(13, (60,) + (40,) * 11, (60,) * 3, 4)


class Orc:
    """The oracle with one secret key, its relinearization key, its Galois
    keys for `rots`, and the element-wise operations restated."""

    def __init__(self, prm, seed, rots):
        self.o = o = make_oracle(prm)
        self.prm, self.seed = prm, seed
        self.sk = o.keygen_secret(seed)
        self.rk = o.keygen_relin(seed, self.sk)
        self.gal = {o.galois_elt(r): o.keygen_galois(seed, self.sk, o.galois_elt(r)) for r in rots}

    def q(self, n):
        return np.array(self.o.primes[:n], np.uint64)[:, None]

    def enc(self, z, level, nonce):
        o = self.o
        return o.encrypt(self.sk, o.encode(z, level, self.prm.scale), self.seed, nonce)

    def add(self, a, b):
        return (a + b) % self.q(a.shape[1])

    def sub(self, a, b):
        q = self.q(a.shape[1])
        return (a + q - b) % q

    def mul(self, a, b):
        return self.o.relinearize(self.o.tensor(a, b), self.rk)

    def rescale(self, a, scale):
        lv = a.shape[1] - 1
        return self.o.rescale(a), scale / float(self.o.primes[lv])

    def mul_const(self, a, scale, vals, target=None):
        lv = a.shape[1] - 1
        target = scale if target is None else target
        z = np.broadcast_to(np.asarray(vals, np.float64), (self.o.N // 2,))
        pt = self.o.encode(np.ascontiguousarray(z), lv, target * float(self.o.primes[lv]) / scale)
        return self.o.rescale(self.o.mul_plain(a, pt)), target

    def add_plain(self, a, vals, scale):
        lv = a.shape[1] - 1
        out = a.copy()
        out[0] = (a[0] + self.o.encode(vals, lv, scale)) % self.q(lv + 1)
        return out

    def ln_keys(self, L, k):
        o = self.o
        return [o.keygen_galois(self.seed, self.sk, o.galois_elt(L << i)) for i in range(int(np.log2(k)))]


def _layer():
    ctx, big = make_ctx(P_SMALL), make_ctx(P_BIG)
    lay = ly.BertLayer(ctx, big, L=32, d=128, H=8, Dh=16, f=256, groups=(8,), seed=3, b1=8)
    return ctx, big, lay


def _same(ctx, cts, refs, what):
    assert len(cts) == len(refs), what
    for j, (c, r) in enumerate(zip(cts, refs)):
        assert np.array_equal(ctx.ct_export(c), r), (what, j)


def test_segment3_attention_output_projection_ln1_head():
    ctx, big, lay = _layer()
    L, d, Dh, Hg, topb = lay.L, lay.d, lay.Dh, 8, lay.topb
    _, rb = lay.rotations()
    keysb = big.keygen(SEED + 1, rb, relin=True)
    orc = Orc(P_BIG, SEED + 1, rb)
    pl = lay.cc_pv[Hg]
    inf = pl.info()
    Kc, n_c = inf["Kc"], inf["n_c"]
    rng = np.random.default_rng(31)
    E = rng.exponential(1.0, (Hg, L, L))
    rinv = 1.0 / E.sum(axis=2)
    V = rng.uniform(-1, 1, (Hg, L, Dh))
    Pz = ly.pack_heads(E, L, Hg, Kc, n_c, rows=False)
    Rz = ly.pack_heads(np.repeat(rinv[:, :, None], L, axis=2), L, Hg, Kc, n_c, rows=False)
    Vz = ly.pack_heads(np.concatenate([V, np.zeros((Hg, L, L - Dh))], axis=2), L, Hg, Kc, n_c, rows=True)
    lvls = (topb, topb, topb - 1)
    gpu_in, orc_in = [], []
    for t, (Z, lv) in enumerate(zip((Pz, Rz, Vz), lvls)):
        gpu_in.append([big.encrypt(keysb, big.encode(z, lv), 100 * t + c) for c, z in enumerate(Z)])
        orc_in.append([orc.enc(z, lv, 100 * t + c) for c, z in enumerate(Z)])
    # GPU
    merged = lay.he_attention(keysb, Hg, *gpu_in)
    Eo = lay.he_output_projection(keysb, merged)
    # oracle: smul_cc, matmul_cc, merge, W_O
    D = P_BIG.scale
    Pn = []
    for p_, r_ in zip(orc_in[0], orc_in[1]):
        y, s_pn = orc.rescale(orc.mul(p_, r_), D * D)
        Pn.append(y)
    C = orc.o.matmul_cc(np.stack(Pn), np.stack(orc_in[2]), L, Hg, inf["b1s1"], inf["b1s2"], orc.gal, orc.rk)
    half = Dh // Kc
    m_o = [orc.add(C[j], C[j + half]) for j in range(half)]
    _same(big, merged, m_o, "merged")
    Eo_o = orc.o.matmul_cp_diag(np.stack(m_o), L, list(lay.groups), Dh, lay.Wo, d, lay.p_o.info()["b1"], orc.gal)
    _same(big, Eo, Eo_o, "W_O")
    # the product's scale: (Delta^2 / q_topb) Delta / q_{l0 - 2} for matmul_cc at l0 = topb - 1
    # (its masks carry the primes it drops); the ct-pt product keeps it
    s_e = s_pn * D / float(orc.o.primes[topb - 3])
    assert Eo[0].scale == s_e and Eo[0].level == topb - 6
    # residual and LayerNorm head
    Xr = rng.uniform(-1, 1, (L, d))
    Xz = ly.pack_columns(Xr, L, lay.kb)
    Xres = [big.encrypt(keysb, big.encode(z, Eo[0].level, s_e), 500 + c) for c, z in enumerate(Xz)]
    Xmu, var = lay.he_residual_ln_head(big, keysb, Eo, Xres)
    Xres_o = [orc.o.encrypt(orc.sk, orc.o.encode(z, topb - 6, s_e), orc.seed, 500 + c) for c, z in enumerate(Xz)]
    R1 = np.stack([orc.add(a, b) for a, b in zip(Eo_o, Xres_o)])
    rx, rv = orc.o.layernorm_head(R1, L, d, orc.ln_keys(L, lay.kb), orc.rk)
    _same(big, Xmu, rx, "X_mu")
    _same(big, var, [rv], "var")
    # the values: LayerNorm head of (E / rowsum) V W_O + X
    Att = np.einsum("hij,hjk->hik", E * rinv[:, :, None], V)
    ref = np.concatenate(list(Att), axis=1) @ lay.Wo + Xr
    got, want = big.decrypt(keysb, var[0], coeffs=False)[1][:L], ref.var(axis=1)
    assert np.abs(got - want).max() < 1e-4 * max(1.0, np.abs(want).max())


def test_segment4_ln1_tail_w1_gelu_pieces():
    ctx, big, lay = _layer()
    L, d, k, top = lay.L, lay.d, lay.k, lay.top
    rs, _ = lay.rotations()
    keys = ctx.keygen(SEED, rs, relin=True)
    orc = Orc(P_SMALL, SEED, rs)
    rng = np.random.default_rng(41)
    xmu = rng.uniform(-1, 1, (L, d))
    rs1 = rng.uniform(0.5, 2.0, L)
    Xz = ly.pack_columns(xmu, L, k)
    Rz = np.tile(rs1, k)[None]
    g1z, b1z = ly.pack_columns(np.tile(lay.g1, (L, 1)), L, k), ly.pack_columns(np.tile(lay.b1, (L, 1)), L, k)
    Xm = [ctx.encrypt(keys, ctx.encode(z, top), 10 + c) for c, z in enumerate(Xz)]
    Rs = ctx.encrypt(keys, ctx.encode(Rz[0], top), 9)
    Xm_o = [orc.enc(z, top, 10 + c) for c, z in enumerate(Xz)]
    Rs_o = orc.enc(Rz[0], top, 9)
    # GPU
    hs = lay.he_ln_tail(keys, Xm, Rs, g1z, b1z)
    U, F0, F1 = lay.he_ffn_up(keys, hs)
    # oracle: the tail
    D = P_SMALL.scale
    hs_o = []
    for c, x in enumerate(Xm_o):
        y, s = orc.rescale(orc.mul(x, Rs_o), D * D)
        y, s = orc.mul_const(y, s, g1z[c])
        hs_o.append(orc.add_plain(y, b1z[c], s))
    assert hs[0].scale == s and hs[0].level == top - 2
    _same(ctx, hs, hs_o, "LN1 tail")
    # W_1 (the ct-pt product keeps the scale)
    U_o = orc.o.matmul_cp(np.stack(hs_o), L, d, lay.W1, lay.f, lay.p_w1.info()["b1"], orc.gal)
    _same(ctx, U, U_o, "W_1")
    # the GeLU pieces
    a, b, cc, dd, e = ly.GELU
    su = s
    F0_o, F1_o = [], []
    for x in U_o:
        x2, s2 = orc.rescale(orc.mul(x, x), su * su)
        x1d = x[:, :x2.shape[1]]
        x3, s3 = orc.rescale(orc.mul(x2, x1d), s2 * su)
        x4, s4 = orc.rescale(orc.mul(x2, x2), s2 * s2)
        t4, _ = orc.mul_const(x4, s4, a, su)
        t3, _ = orc.mul_const(x3, s3, b, su)
        x2d, x1dd = x2[:, :x3.shape[1]], x[:, :x3.shape[1]]
        t2, _ = orc.mul_const(x2d, s2, cc, su)
        tm, _ = orc.mul_const(x1dd, su, 0.5 - dd, su)
        tp, _ = orc.mul_const(x1dd, su, 0.5 + dd, su)
        base = orc.add_plain(orc.add(t4, t2), np.full(orc.o.N // 2, e), su)
        F0_o.append(orc.add(orc.sub(base, t3), tm))
        F1_o.append(orc.add(orc.add(base, t3), tp))
    _same(ctx, F0, F0_o, "GeLU F0")
    _same(ctx, F1, F1_o, "GeLU F1")
    # the values of one output ciphertext against the polynomials in FP64
    u = ctx.decrypt(keys, U[0], coeffs=False)[1]
    got0 = ctx.decrypt(keys, F0[0], coeffs=False)[1]
    want0 = e + cc * u ** 2 + a * u ** 4 - b * u ** 3 + (0.5 - dd) * u
    assert np.abs(got0 - want0).max() < 1e-4 * max(1.0, np.abs(want0).max())


def test_segment5_w2_residual_ln2_head():
    ctx, big, lay = _layer()
    L, d, f, k, top = lay.L, lay.d, lay.f, lay.k, lay.top
    rs, _ = lay.rotations()
    keys = ctx.keygen(SEED, rs, relin=True)
    orc = Orc(P_SMALL, SEED, rs)
    rng = np.random.default_rng(51)
    g = rng.uniform(-1, 1, (L, f))
    hmid = rng.uniform(-1, 1, (L, d))
    Gz, Hz = ly.pack_columns(g, L, k), ly.pack_columns(hmid, L, k)
    Gc = [ctx.encrypt(keys, ctx.encode(z, top), 20 + c) for c, z in enumerate(Gz)]
    W2o = ctx.matmul_cp_plan(keys, lay.p_w2, Gc)
    s_w = P_SMALL.scale  # the ct-pt product keeps the scale
    assert W2o[0].scale == s_w and W2o[0].level == top - 1
    Hc = [ctx.encrypt(keys, ctx.encode(z, top - 1, s_w), 60 + c) for c, z in enumerate(Hz)]
    Xmu, var = lay.he_residual_ln_head(ctx, keys, W2o, Hc)
    W2o_o = orc.o.matmul_cp(np.stack([orc.enc(z, top, 20 + c) for c, z in enumerate(Gz)]), L, f, lay.W2, d,
                            lay.p_w2.info()["b1"], orc.gal)
    _same(ctx, W2o, W2o_o, "W_2")
    Hc_o = [orc.o.encrypt(orc.sk, orc.o.encode(z, top - 1, s_w), orc.seed, 60 + c) for c, z in enumerate(Hz)]
    R2 = np.stack([orc.add(a_, b_) for a_, b_ in zip(W2o_o, Hc_o)])
    rx, rv = orc.o.layernorm_head(R2, L, d, orc.ln_keys(L, k), orc.rk)
    _same(ctx, Xmu, rx, "X_mu")
    _same(ctx, var, [rv], "var")
    ref = g @ lay.W2 + hmid
    got, want = ctx.decrypt(keys, var[0], coeffs=False)[1][:L], ref.var(axis=1)
    assert np.abs(got - want).max() < 1e-4 * max(1.0, np.abs(want).max())
