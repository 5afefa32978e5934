"""One BERT-base encoder layer evaluated the hybrid way: the linear operators in
RNS-CKKS blocks on the GPU, the nonlinear operators on additive shares.

The paper fuses the linear operators of a Transformer layer into five blocks
(Sec. 4, Sec. 7.1, Table eva_params), between which the state is converted
from CKKS to MPC shares (Alg. 1) and back (Alg. 2) so that the nonlinear
operators (Alg. Softmax, LayerNorm and GeLU, red steps) run in MPC.  The
figure that draws the blocks is not in the text; the reading here follows the
green/red steps of those algorithms and the layer order, with the LayerNorm-2
tail counted into the next layer's first block:

  1  LN2 tail of the previous layer + QKV (matmul_cp) + Q K^T (matmul_cc)
  2  softmax exponential: X - max, x / 64 + 1, six squarings
  3  normalisation by the row sums (smul_cc) + P V (matmul_cc) + W_O
     (diagonal-input matmul_cp, App. C.2) + residual + LayerNorm-1 head
  4  LayerNorm-1 tail + W_1 (matmul_cp) + the GeLU polynomials F_0, F_1
  5  W_2 (matmul_cp) + residual + LayerNorm-2 head

whose depths (4, 7, 7, 7, ~6) match the table.  Block 1 is one HE segment:
the columns of W_Q and W_K are reordered in plaintext (Sec. 5.1, multi-head
packing) so that the spatial-first output ciphertexts of the QKV matmul_cp
are already the head-packed operands of Q K^T (column b = h + Hg kappa of
output ciphertext c of a head group holds column c Kc + kappa of head h), and
matmul_cc runs on them directly; only V and Q K^T leave the block.  The LN2
tail runs as a last segment of this layer (segment 6 below).  Segments 1, 2,
4, 5, 6 run on `ctx` (BERT-base: N = 2^15, 8 primes), segment 3 (depth 9
here, matmul_cc taking four levels) on `ctx_big` (N = 2^16, 12 primes).

MPC is simulated: both parties live in this process, every value between
blocks is held as additive shares over Z_{2^43} at scale 2^-13 (Sec. 7.1),
and each nonlinear step computes its ideal functionality on the revealed
values and shares the result again.  Every HE step and both parties' local
conversion steps run in the library's kernels.
"""
import time

import numpy as np

L_MPC, SF = 43, 13
T_EXP = -13.0                                    # exp clipping threshold (App. B)
GELU = (0.020848611754127593, -0.18352506127082727, 0.5410550166368381,
        -0.03798164612714154, 0.001620808531841547)  # BOLT's a, b, c, d, e (App. B)


# ---------------------------------------------------------------------------
# packing
# ---------------------------------------------------------------------------
def pack_columns(X, m, k):
    """Spatial-first (Sec. 4.2.1): ciphertext c holds X[i, c k + b] at slot i + m b."""
    n_cts = -(-X.shape[1] // k)
    Z = np.zeros((n_cts, m * k))
    for c in range(n_cts):
        blk = X[:, c * k:(c + 1) * k]
        Z[c, :blk.shape[1] * m] = blk.T.reshape(-1)
    return Z


def unpack_columns(Z, m, k, d_out):
    cols = [Z[e, b * m:(b + 1) * m] for e in range(Z.shape[0]) for b in range(k)]
    return np.stack(cols[:d_out], axis=1)


def pack_heads(mats, L, Hg, Kc, n_c, rows):
    """Multi-head packing (Sec. 5.1): block h + Hg kappa of ciphertext c holds
    column (rows=False, mats (Hg, L, R)) or row (rows=True, mats (Hg, R, L))
    c Kc + kappa of head h, element i at slot (h + Hg kappa) L + i."""
    Z = np.zeros((n_c, L * Hg * Kc))
    R = mats.shape[1] if rows else mats.shape[2]
    for c in range(n_c):
        for kappa in range(Kc):
            k = c * Kc + kappa
            if k < R:
                for h in range(Hg):
                    b = h + Hg * kappa
                    Z[c, b * L:(b + 1) * L] = mats[h, k, :] if rows else mats[h, :, k]
    return Z


def head_permutation(groups, Dh, k):
    """Column order of W_Q / W_K (Sec. 5.1, multi-head packing): output column
    e k + b of the reordered weight is column perm[e k + b] of the original, so
    that output ciphertext e of head group g (first head h0, Kc = k / Hg) holds
    at block b = h + Hg kappa the column c Kc + kappa of head h0 + h, c = e - (the
    group's first ciphertext)."""
    perm, h0 = [], 0
    for Hg in groups:
        Kc = k // Hg
        assert Kc * Hg == k and Dh % Kc == 0, "head dimension must be a multiple of k / Hg"
        for c in range(Dh // Kc):
            for b in range(k):
                h, kappa = b % Hg, b // Hg
                perm.append((h0 + h) * Dh + c * Kc + kappa)
        h0 += Hg
    return np.array(perm)


def diag_index(L, Hg, Kc, n_out):
    """Diagonal packing of matmul_cc outputs: for output ciphertext j and slot t,
    the (head, row, column) it holds (block h + Hg kappa, diagonal j Kc + kappa,
    element i = C_h[i, (i + delta) mod L])."""
    s = L * Hg * Kc
    t = np.arange(s)
    blk, i = t // L, t % L
    h, kappa = blk % Hg, blk // Hg
    out = []
    for j in range(n_out):
        delta = j * Kc + kappa
        out.append((h, i, (i + delta) % L))
    return out


def pack_diagonals(C, L, Hg, Kc, n_out):
    """(Hg, L, L) -> (n_out, s) in the diagonal packing."""
    return np.stack([C[h, i, col] for h, i, col in diag_index(L, Hg, Kc, n_out)])


def unpack_diagonals(Z, L, Hg, Kc):
    out = np.zeros((Hg, L, L))
    for j, (h, i, col) in enumerate(diag_index(L, Hg, Kc, Z.shape[0])):
        out[h, i, col] = Z[j]
    return out


# ---------------------------------------------------------------------------
# simulated MPC and the conversions at block boundaries
# ---------------------------------------------------------------------------
class Mpc:
    """Additive shares over Z_{2^l} at scale 2^-sf; nonlinear functions are the
    ideal functionalities on the revealed values (the MPC protocols themselves
    are out of scope)."""

    def __init__(self, seed, l=L_MPC, sf=SF):
        self.rng = np.random.default_rng(seed)
        self.l, self.sf = l, sf
        self.mask = (1 << l) - 1

    def share(self, v):
        xi = np.round(np.asarray(v, np.float64) * 2.0 ** self.sf).astype(np.int64)
        x0 = self.rng.integers(0, 1 << self.l, xi.shape, dtype=np.uint64)
        x1 = ((xi.astype(np.uint64) - x0) & np.uint64(self.mask)).astype(np.uint64)
        return x0, x1

    def reveal(self, x0, x1):
        v = (np.asarray(x0, np.uint64) + np.asarray(x1, np.uint64)) & np.uint64(self.mask)
        s = v.astype(np.int64)
        s = np.where(s >= (1 << (self.l - 1)), s - (1 << self.l), s)
        return s.astype(np.float64) / 2.0 ** self.sf


class Bridge:
    """CKKS <-> MPC on one context: masking, decryption by P0, field to ring and
    decoding of shares (Alg. 1); extension and encoding of shares, ring to
    field, encryption by P0 and addition by P1 (Alg. 2).  The comparisons of
    the ring/field extensions use their simulated ideal functionality."""

    def __init__(self, ctx, keys, mpc, seed):
        self.ctx, self.keys, self.mpc, self.seed = ctx, keys, mpc, seed
        self.nonce = 1 << 20

    def _nonces(self, k):
        self.nonce += k
        return list(range(self.nonce - k, self.nonce))

    def to_mpc(self, cts):
        """Ciphertexts -> the revealed slot values of their shares (count, N/2)."""
        ctx = self.ctx
        masked, p1 = ctx.he2mpc_batch(self.keys, cts, self._nonces(len(cts)))
        p0 = np.ascontiguousarray(ctx.decrypt_batch(self.keys, masked)[0][:, 0, :])
        w0, w1 = ctx.f2r_wrap_sim(p0, p1, self.seed, self._nonces(len(cts)))
        scales = [c.scale for c in cts]
        out = np.zeros((len(cts), ctx.N // 2))
        for sc in sorted(set(scales)):                    # one call per scale
            idx = [k for k, x in enumerate(scales) if x == sc]
            y0 = ctx.c2m_local(0, p0[idx], w0[idx], sc, self.mpc.l, self.mpc.sf)
            y1 = ctx.c2m_local(1, p1[idx], w1[idx], sc, self.mpc.l, self.mpc.sf)
            out[idx] = self.mpc.reveal(y0, y1)
        return out

    def to_ckks(self, Z, level, scale=None):
        """Slot vectors (count, <= N/2) -> ciphertexts at `level` and `scale`:
        shared, extended, encoded and reduced by both parties, encrypted by P0,
        completed by P1."""
        ctx = self.ctx
        scale = ctx.scale if scale is None else scale
        Z = np.atleast_2d(Z)
        count, n = Z.shape
        x0, x1 = self.mpc.share(Z)
        v0, v1 = ctx.ext_wrap_sim(x0, x1, n, self.mpc.l, self.seed, self._nonces(count))
        m0 = ctx.m2c_local(0, x0, v0, n, level, scale, self.mpc.l, self.mpc.sf)
        m1 = ctx.m2c_local(1, x1, v1, n, level, scale, self.mpc.l, self.mpc.sf)
        cts = []
        for k, nonce in enumerate(self._nonces(count)):
            c0 = ctx.encrypt(self.keys, ctx.pt_import(m0[k], level, scale), nonce)
            cts.append(ctx.add_plain(c0, ctx.pt_import(m1[k], level, scale)))
        return cts


# ---------------------------------------------------------------------------
# the layer
# ---------------------------------------------------------------------------
def gelu_approx(x):
    a, b, c, d, e = GELU
    ax = np.abs(x)
    mid = a * ax ** 4 + b * ax ** 3 + c * ax ** 2 + d * ax + e + 0.5 * x
    return np.where(x > 2.7, x, np.where(x < -2.7, 0.0, mid))


def exp_approx(x):
    return np.where(x < T_EXP, 0.0, (1.0 + x / 64.0) ** 64)


def layernorm(X, gamma, beta):
    mu = X.mean(axis=1, keepdims=True)
    var = ((X - mu) ** 2).mean(axis=1, keepdims=True)
    return (X - mu) / np.sqrt(var) * gamma + beta


class BertLayer:
    """Weights and plans of one BERT-base-shaped encoder layer (L tokens,
    hidden d, H heads of Dh, FFN f; W_Q pre-scaled by 1/sqrt(Dh)), on two
    contexts: ctx (N = 2^15, 8 primes) and ctx_big (N = 2^16, 12 primes)."""

    def __init__(self, ctx, ctx_big, L=128, d=768, H=12, Dh=64, f=3072, groups=(8, 4), seed=7, b1=16, b1_down=None):
        self.ctx, self.big = ctx, ctx_big
        self.L, self.d, self.H, self.Dh, self.f, self.groups = L, d, H, Dh, f, list(groups)
        rng = np.random.default_rng(seed)
        u = lambda shape, fan_in: rng.uniform(-1.0, 1.0, shape) / np.sqrt(fan_in)
        self.Wqkv = u((d, 3 * d), d)
        self.Wqkv[:, :d] /= np.sqrt(Dh)
        self.Wo, self.W1, self.W2 = u((d, d), d), u((d, f), d), u((f, d), f)
        self.g1, self.b1 = 1.0 + 0.1 * rng.uniform(-1, 1, d), 0.1 * rng.uniform(-1, 1, d)
        self.g2, self.b2 = 1.0 + 0.1 * rng.uniform(-1, 1, d), 0.1 * rng.uniform(-1, 1, d)
        self.k = ctx.N // 2 // L            # columns per ciphertext on ctx
        self.kb = ctx_big.N // 2 // L       # on ctx_big
        top, topb = ctx.nQ - 1, ctx_big.nQ - 1
        assert self.k > 0 and self.kb > 0
        self.top, self.topb = top, topb
        t0 = time.perf_counter()
        # W_Q, W_K columns in the head-packed order (block 1 runs Q K^T on the
        # QKV product's output ciphertexts), W_V in the natural order
        self.perm = head_permutation(self.groups, Dh, self.k)
        self.Wqkv_he = np.concatenate([self.Wqkv[:, :d][:, self.perm], self.Wqkv[:, d:2 * d][:, self.perm],
                                       self.Wqkv[:, 2 * d:]], axis=1)
        self.p_qkv = ctx.cp_plan(L, d, self.Wqkv_he, 3 * d, top, b1)
        self.p_w1 = ctx.cp_plan(L, d, self.W1, f, top - 2, b1)      # after the LN1 tail (two rescales)
        # the W_2 product has f / k input ciphertexts: fewer baby steps keep its
        # terms per output (inputs x b1) within the MAC's shared-memory tile
        if b1_down is None:
            b1_down = b1
            while b1_down > 1 and (f // self.k) * b1_down > 96:
                b1_down //= 2
        self.p_w2 = ctx.cp_plan(L, f, self.W2, d, top, b1_down)
        self.cc_qk = {Hg: ctx.cc_plan(L, Hg, Dh, top - 1) for Hg in self.groups}
        self.cc_pv = {Hg: ctx_big.cc_plan(L, Hg, L, topb - 1) for Hg in self.groups}
        self.p_o = ctx_big.cp_plan_diag(L, self.groups, Dh, self.Wo, d, topb - 5, b1)
        ctx.sync()
        ctx_big.sync()
        self.encode_s = time.perf_counter() - t0

    def rotations(self):
        """Rotation amounts needed on each context."""
        def cp_rots(p, m):
            i = p.info()
            return [b * m for b in range(1, i["b1"])] + [g * i["b1"] * m for g in range(1, i["G"])]
        small = set(cp_rots(self.p_qkv, self.L)) | set(cp_rots(self.p_w1, self.L)) | set(cp_rots(self.p_w2, self.L))
        for p in self.cc_qk.values():
            small |= set(p.rotations())
        small |= {self.L << i for i in range(int(np.log2(self.k)))}
        big = set(cp_rots(self.p_o, self.L)) | {self.L << i for i in range(int(np.log2(self.kb)))}
        for p in self.cc_pv.values():
            big |= set(p.rotations())
        return sorted(r % (self.ctx.N // 2) for r in small if r % (self.ctx.N // 2)), \
            sorted(r % (self.big.N // 2) for r in big if r % (self.big.N // 2))

    # -- the reference with the same approximations, in FP64 -----------------
    def reference(self, X):
        L, d, H, Dh = self.L, self.d, self.H, self.Dh
        QKV = X @ self.Wqkv
        Q = QKV[:, :d].reshape(L, H, Dh).transpose(1, 0, 2)
        K = QKV[:, d:2 * d].reshape(L, H, Dh).transpose(1, 0, 2)
        V = QKV[:, 2 * d:].reshape(L, H, Dh).transpose(1, 0, 2)
        S = np.einsum("hik,hjk->hij", Q, K)
        E = exp_approx(S - S.max(axis=2, keepdims=True))
        P = E / E.sum(axis=2, keepdims=True)
        Att = np.einsum("hij,hjk->hik", P, V)
        h = layernorm(X + np.concatenate(list(Att), axis=1) @ self.Wo, self.g1, self.b1)
        return layernorm(h + gelu_approx(h @ self.W1) @ self.W2, self.g2, self.b2)

    # -- block 1 in HE: QKV, then Q K^T on its output ciphertexts --------------
    def he_block1(self, keys, Xc):
        """Xc: the d / k input ciphertexts of X (spatial-first, top level).
        Returns (the 3 d / k QKV output ciphertexts, [Q K^T outputs per head
        group]).  Q's ciphertexts of group g are the A operand and K's the B
        operand (K_h^T in reduce-first packing) of that group's matmul_cc."""
        ctx = self.ctx
        Y = ctx.matmul_cp_plan(keys, self.p_qkv, Xc)
        nq = self.d // self.k
        outs, e0 = [], 0
        for Hg in self.groups:
            n_c = self.cc_qk[Hg].info()["n_c"]
            outs.append(ctx.matmul_cc_plan(keys, self.cc_qk[Hg], Y[e0:e0 + n_c], Y[nq + e0:nq + e0 + n_c]))
            e0 += n_c
        return Y, outs

    # -- the HE parts of segments 3-6 (ciphertexts in, ciphertexts out) --------
    def he_attention(self, keys_big, Hg, Pc, Rc, Vc):
        """Segment 3, one head group (on the big context): the exponentials P
        times the reciprocal row sums R (smul_cc: product and rescale), P V with
        matmul_cc (Sec. 5.1), and the merge of complementary diagonals of the
        padded product (App. C.2).  Returns the merged ciphertexts."""
        big, pl = self.big, self.cc_pv[Hg]
        Pn = [big.rescale(big.mul(keys_big, p_, r_)) for p_, r_ in zip(Pc, Rc)]
        C = big.matmul_cc_plan(keys_big, pl, Pn, Vc)
        half = self.Dh // pl.info()["Kc"]
        return [big.add(C[j], C[j + half]) for j in range(half)]

    def he_output_projection(self, keys_big, merged):
        """Segment 3: Concat(Att_h) W_O on the merged diagonals of every head
        group (the diagonal-input matmul_cp of App. C.2)."""
        return self.big.matmul_cp_plan(keys_big, self.p_o, merged)

    def he_residual_ln_head(self, ctx, keys, Y, Xres):
        """Segments 3 and 5: the residual addition and the LayerNorm head (Alg.
        LayerNorm lines 1-6) on ctx.  Returns (X_mu ciphertexts, [var])."""
        R = [ctx.add(a, b) for a, b in zip(Y, Xres)]
        return ctx.layernorm_head(keys, R, self.L, self.d, len(R))

    def he_ln_tail(self, keys, Xm, Rs, gz, bz):
        """The LayerNorm tail of segments 4 and 6: the centred columns times
        1/sigma (smul_cc), times gamma (ewmul_cp, mul_const), plus beta
        (ewadd_cp)."""
        ctx = self.ctx
        out = []
        for c, x in enumerate(Xm):
            y = ctx.rescale(ctx.mul(keys, x, Rs))
            y = ctx.mul_const(y, gz[c])
            out.append(ctx.add_plain(y, ctx.encode(bz[c], y.level, y.scale)))
        return out

    def he_ffn_up(self, keys, hs):
        """Segment 4 after the LN1 tail: W_1 (matmul_cp) and, on each output
        ciphertext x, the two degree-4 GeLU pieces F0 = e + c x^2 + a x^4 - b x^3
        + (1/2 - d) x and F1 = e + c x^2 + a x^4 + b x^3 + (1/2 + d) x, every term
        brought to x's scale by mul_const.  Returns (U, F0, F1)."""
        ctx = self.ctx
        U = ctx.matmul_cp_plan(keys, self.p_w1, hs)
        a, b, cc, dd, e = GELU
        F0s, F1s = [], []
        for x in U:
            x2 = ctx.rescale(ctx.mul(keys, x, x))
            x1d = ctx.drop_level(x, x2.level)
            x3 = ctx.rescale(ctx.mul(keys, x2, x1d))
            x4 = ctx.rescale(ctx.mul(keys, x2, x2))
            tgt = x.scale
            t4 = ctx.mul_const(x4, a, tgt)
            t3 = ctx.mul_const(x3, b, tgt)
            x2d, x1dd = ctx.drop_level(x2, x3.level), ctx.drop_level(x, x3.level)
            t2 = ctx.mul_const(x2d, cc, tgt)
            tm = ctx.mul_const(x1dd, 0.5 - dd, tgt)
            tp = ctx.mul_const(x1dd, 0.5 + dd, tgt)
            base = ctx.add(t4, t2)
            base = ctx.add_plain(base, ctx.encode(np.full(ctx.N // 2, e), base.level, base.scale))
            F0s.append(ctx.add(ctx.sub(base, t3), tm))
            F1s.append(ctx.add(ctx.add(base, t3), tp))
        return U, F0s, F1s

    # -- the hybrid evaluation --------------------------------------------------
    def forward(self, X, keys, keys_big, mpc, seed=11):
        """X: (L, d) activation (the previous layer's output, as MPC shares).
        Returns (Y, seconds per segment for the HE work, seconds per segment for
        the conversions and the simulated MPC)."""
        ctx, big = self.ctx, self.big
        L, d, H, Dh, f, k, kb = self.L, self.d, self.H, self.Dh, self.f, self.k, self.kb
        br, bb = Bridge(ctx, keys, mpc, seed), Bridge(big, keys_big, mpc, seed + 1)
        he, conv = {}, {}

        def timed(name, fn, store):
            ctx.sync()
            big.sync()
            t0 = time.perf_counter()
            r = fn()
            ctx.sync()
            big.sync()
            store[name] = store.get(name, 0.0) + time.perf_counter() - t0
            return r

        # segment 1: QKV and Q K^T in one HE block; V and the scores go to MPC
        Xc = timed("1 QKV + QK^T", lambda: br.to_ckks(pack_columns(X, L, k), self.top), conv)
        Y, Cs = timed("1 QKV + QK^T", lambda: self.he_block1(keys, Xc), he)
        V = unpack_columns(timed("1 QKV + QK^T", lambda: br.to_mpc(Y[2 * d // k:]), conv), L, k, d)
        V = V.reshape(L, H, Dh).transpose(1, 0, 2)
        S = np.zeros((H, L, L))
        h0 = 0
        for Hg, C in zip(self.groups, Cs):
            Kc = self.cc_qk[Hg].info()["Kc"]
            S[h0:h0 + Hg] = unpack_diagonals(timed("1 QKV + QK^T", lambda: br.to_mpc(C), conv), L, Hg, Kc)
            h0 += Hg
        # MPC: row maxima
        mx = S.max(axis=2)
        # segment 2: exponential, in the diagonal packing
        Xexp = np.zeros((H, L, L))
        h0 = 0
        for Hg in self.groups:
            inf = self.cc_qk[Hg].info()
            Kc, nout = inf["Kc"], inf["nout"]
            Sz = pack_diagonals(S[h0:h0 + Hg], L, Hg, Kc, nout)
            Mz = pack_diagonals(np.repeat(mx[h0:h0 + Hg, :, None], L, axis=2), L, Hg, Kc, nout)
            Sc = timed("2 exp", lambda: br.to_ckks(Sz, self.top), conv)
            Mc = timed("2 exp", lambda: br.to_ckks(Mz, self.top), conv)

            def expo():
                outs = []
                for s_, m_ in zip(Sc, Mc):
                    x = ctx.mul_const(ctx.sub(s_, m_), 1.0 / 64.0)
                    x = ctx.add_plain(x, ctx.encode(np.ones(ctx.N // 2), x.level, x.scale))
                    for _ in range(6):
                        x = ctx.rescale(ctx.mul(keys, x, x))
                    outs.append(x)
                return outs
            E = timed("2 exp", expo, he)
            Ez = timed("2 exp", lambda: br.to_mpc(E), conv)
            Xexp[h0:h0 + Hg] = unpack_diagonals(Ez, L, Hg, Kc)
            h0 += Hg
        # MPC: clipping (cmp + mux), row sums (local), reciprocal
        Xexp = np.where(S - mx[:, :, None] < T_EXP, 0.0, Xexp)
        rinv = 1.0 / Xexp.sum(axis=2)
        # segment 3 (on the big context): normalisation, P V, W_O, residual, LN1 head
        merged, h0 = [], 0
        for Hg in self.groups:
            pl = self.cc_pv[Hg]
            inf = pl.info()
            Kc, n_c = inf["Kc"], inf["n_c"]
            Pz = pack_heads(Xexp[h0:h0 + Hg], L, Hg, Kc, n_c, rows=False)
            Rz = pack_heads(np.repeat(rinv[h0:h0 + Hg, :, None], L, axis=2), L, Hg, Kc, n_c, rows=False)
            Vz = pack_heads(np.concatenate([V[h0:h0 + Hg], np.zeros((Hg, L, L - Dh))], axis=2), L, Hg, Kc, n_c,
                            rows=True)
            Pc = timed("3 attention", lambda: bb.to_ckks(Pz, self.topb), conv)
            Rc = timed("3 attention", lambda: bb.to_ckks(Rz, self.topb), conv)
            Vc = timed("3 attention", lambda: bb.to_ckks(Vz, self.topb - 1), conv)
            merged += timed("3 attention", lambda: self.he_attention(keys_big, Hg, Pc, Rc, Vc), he)
            h0 += Hg
        Eo = timed("3 attention", lambda: self.he_output_projection(keys_big, merged), he)
        Xres = timed("3 attention", lambda: bb.to_ckks(pack_columns(X, L, kb), Eo[0].level, Eo[0].scale), conv)
        Xmu, var = timed("3 attention", lambda: self.he_residual_ln_head(big, keys_big, Eo, Xres), he)
        xmu = unpack_columns(timed("3 attention", lambda: bb.to_mpc(Xmu), conv), L, kb, d)
        v1 = timed("3 attention", lambda: bb.to_mpc(var), conv)[0][:L]
        # MPC: rsqrt
        rs1 = 1.0 / np.sqrt(v1)
        # segment 4: LN1 tail, W_1, GeLU polynomials
        Xm = timed("4 FFN up", lambda: br.to_ckks(pack_columns(xmu, L, k), self.top), conv)
        Rs = timed("4 FFN up", lambda: br.to_ckks(np.tile(rs1, k)[None], self.top), conv)[0]
        g1z, b1z = pack_columns(np.tile(self.g1, (L, 1)), L, k), pack_columns(np.tile(self.b1, (L, 1)), L, k)

        hs_out = []

        def ffn_up():
            hs = self.he_ln_tail(keys, Xm, Rs, g1z, b1z)
            hs_out.extend(hs)
            return self.he_ffn_up(keys, hs)
        U, F0, F1 = timed("4 FFN up", ffn_up, he)
        u = unpack_columns(timed("4 FFN up", lambda: br.to_mpc(U), conv), L, k, f)
        f0 = unpack_columns(timed("4 FFN up", lambda: br.to_mpc(F0), conv), L, k, f)
        f1 = unpack_columns(timed("4 FFN up", lambda: br.to_mpc(F1), conv), L, k, f)
        # MPC: three comparisons and the multiplexer
        g = np.where(u > 2.7, u, np.where(u > 0, f1, np.where(u > -2.7, f0, 0.0)))
        hmid = unpack_columns(timed("4 FFN up", lambda: br.to_mpc(hs_out), conv), L, k, d)   # the LN1 output
        # segment 5: W_2, residual, LN2 head
        Gc = timed("5 FFN down", lambda: br.to_ckks(pack_columns(g, L, k), self.top), conv)
        W2o = timed("5 FFN down", lambda: ctx.matmul_cp_plan(keys, self.p_w2, Gc), he)
        Hc = timed("5 FFN down", lambda: br.to_ckks(pack_columns(hmid, L, k), W2o[0].level, W2o[0].scale), conv)

        Xmu2, var2 = timed("5 FFN down", lambda: self.he_residual_ln_head(ctx, keys, W2o, Hc), he)
        xmu2 = unpack_columns(timed("5 FFN down", lambda: br.to_mpc(Xmu2), conv), L, k, d)
        v2 = timed("5 FFN down", lambda: br.to_mpc(var2), conv)[0][:L]
        rs2 = 1.0 / np.sqrt(v2)
        # segment 6 (the next layer's first block in a stack): LN2 tail
        Xm2 = timed("6 LN2 tail", lambda: br.to_ckks(pack_columns(xmu2, L, k), self.top), conv)
        Rs2 = timed("6 LN2 tail", lambda: br.to_ckks(np.tile(rs2, k)[None], self.top), conv)[0]
        g2z, b2z = pack_columns(np.tile(self.g2, (L, 1)), L, k), pack_columns(np.tile(self.b2, (L, 1)), L, k)

        Yc = timed("6 LN2 tail", lambda: self.he_ln_tail(keys, Xm2, Rs2, g2z, b2z), he)
        Yv = unpack_columns(timed("6 LN2 tail", lambda: br.to_mpc(Yc), conv), L, k, d)
        return Yv, he, conv
