#!/usr/bin/env python
"""Benchmark of the B300 RNS-CKKS linear path (BLB, arXiv 2508.19525).

Workload (one GPU): the BERT-base fused linear block of the paper's ct-pt
matrix products -- an encrypted activation X (128 x 768, U[-1,1]) times the
fused QKV weight (768 x 2304), then the first 768 output columns times the
output projection W_O (768 x 768); N = 2^15, 8 RNS primes (60 + 7 x 40 bits),
3 special primes, dnum = 3, scale 2^40.  One step is the whole hot path for
one sequence of 128 tokens:
  client: encode + encrypt X (6 ciphertexts),
  server: matmul_cp QKV (6 -> 18 ciphertexts), matmul_cp W_O (6 -> 6),
          CKKS->MPC masking of the 18 outputs that leave the block,
  client: decryption of the 18 masked ciphertexts (its additive shares).
The plaintext diagonals of both weight matrices are encoded once, when the
weights are loaded (36.6 GB resident in HBM), like any model weights.

Output: one JSON line (rank 0).  `value` is tokens/s with X already in HBM;
`e2e` is the same step through the C ABI from pinned host buffers (X copied
in, both parties' shares copied out).  `--impl reference` times the CPU
oracle on a bounded sample of the same step instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CKKS fused-matmul tokens/s"
UNIT = "tokens/s"
WORKLOAD = ("bert-base fused linear ct-pt: X 128x768 @ W_QKV 768x2304 then @ W_O 768x768, "
            "N=2^15, 8 primes (60+7x40 bits), 3 special primes, dnum=3, scale 2^40, "
            "he2mpc + client decryption of 18 outputs")
M, D, D_QKV, D_O, B1 = 128, 768, 2304, 768, 16
LEVEL = 7
TOKENS_PER_STEP = 128


def config(world):
    return {"workload": WORKLOAD, "global_batch": world, "seq_len": M,
            "parallelism": f"replicas x{world}" if world > 1 else "single",
            "l2": "working set larger than L2 (25.2 GB of byte-sliced plaintext diagonals read per step)",
            "bsgs_b1": B1,
            "encode_overflow_check": "deferred: read once after the timed steps (blb_ctx_set_deferred_encode_check)"}


# --------------------------------------------------------------------------- clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
            return
        # the timed region starts once the sampler has written its first line
        t0 = time.time()
        while time.time() - t0 < 10 and self.p.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.02)
        self.skip = sum(1 for _ in open(self.f.name))

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines()[getattr(self, "skip", 0):]
                if l.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest value of x over all ranks (elapsed seconds: the job is as slow as
    its slowest replica)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(elapsed_s, units_per_rank, world):
    """Whole-job throughput: units processed by all ranks / max elapsed."""
    t = max_over_ranks(elapsed_s, world)
    return units_per_rank * world / t, t


# --------------------------------------------------------------------------- workload
def pack_columns(X, m, k):
    """Spatial-first packing (Sec. 4.2.1): ciphertext c holds X[i, c k + b] at slot i + m b."""
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
    """Multi-head packing (Sec. 5.1): block beta = h + Hg kappa of ciphertext c holds
    column (rows=False, mats (Hg, L, R)) or row (rows=True, mats (Hg, R, L)) k = c Kc + kappa
    of head h, element i at slot beta L + i."""
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


def unpack_head_diagonals(Z, L, Hg, Kc):
    """Output ciphertext j holds diagonal delta = j Kc + kappa of head h at block
    h + Hg kappa: element i is C_h[i, (i + delta) mod L]."""
    out = np.zeros((Hg, L, L))
    i = np.arange(L)
    for j in range(Z.shape[0]):
        for kappa in range(Kc):
            delta = j * Kc + kappa
            for h in range(Hg):
                b = h + Hg * kappa
                out[h, i, (i + delta) % L] = Z[j, b * L:(b + 1) * L]
    return out


class Workload:
    def __init__(self, device, ntt_split=None, ntt_radix=None):
        import torch
        from paper_2508_19525_b300 import blb
        from paper_2508_19525_b300 import workloads as wl
        self.torch, self.blb = torch, blb
        prm = wl.BERT_CP
        self.stream = torch.cuda.Stream(device=device)
        self.ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, prm.dnum, prm.scale, stream=self.stream)
        self.N = self.ctx.N
        self.k = self.N // 2 // M
        G = self.k // B1
        rots = [b * M for b in range(1, B1)] + [g * B1 * M for g in range(1, G)]
        self.keys = self.ctx.keygen(0, rots)
        self.keys_bytes = len(rots) * prm.dnum * 2 * (len(prm.q_bits) + len(prm.p_bits)) * self.N * 8
        # pick the NTT radix and pass split for this ring on the device before
        # anything is timed (or take the given ones, so that profiles capture
        # known kernels)
        self.ntt_split, self.ntt_radix, self.ntt_us = self.ctx.ntt_autotune(256)
        if ntt_split is not None:
            self.ctx.ntt_set_split(ntt_split)
            self.ntt_split = ntt_split
        if ntt_radix is not None:
            self.ctx.ntt_set_radix(ntt_radix)
            self.ntt_radix = ntt_radix
        self.X, Wqkv, Wo = wl.bert_base_cp(seed=0)
        self.Wqkv, self.Wo = Wqkv, Wo
        self.ref_qkv = self.X @ Wqkv
        self.ref_o = self.ref_qkv[:, :D_O] @ Wo
        t = time.time()
        self.plan_qkv = self.ctx.cp_plan(M, D, Wqkv, D_QKV, LEVEL, B1)
        self.plan_o = self.ctx.cp_plan(M, D, Wo, D_O, LEVEL - 1, B1)
        self.ctx.sync()
        self.plan_s = time.time() - t
        self.plan_bytes = self.plan_qkv.info()["plaintext_bytes"] + self.plan_o.info()["plaintext_bytes"]
        # the step's encodings report an overflow at the next sync instead of
        # each waiting for the device (timed() syncs after the timed steps)
        self.ctx.set_deferred_encode_check(True)
        Z = pack_columns(self.X, M, self.k)
        self.n_in = Z.shape[0]
        self.n_out = 18
        self.Zdev = torch.tensor(Z, dtype=torch.float64, device=device)
        self.Zhost = torch.tensor(Z, dtype=torch.float64).pin_memory()
        self.p0_dev = torch.zeros((self.n_out, self.N), dtype=torch.uint64, device=device)
        self.p1_dev = torch.zeros((self.n_out, self.N), dtype=torch.uint64, device=device)
        self.p0_host = torch.zeros((self.n_out, self.N), dtype=torch.uint64).pin_memory()
        self.p1_host = torch.zeros((self.n_out, self.N), dtype=torch.uint64).pin_memory()
        self.nonce = 1000

    def nonces(self, k):
        self.nonce += k
        return list(range(self.nonce - k + 1, self.nonce + 1))

    def step(self, host=False, keep=False):
        ctx, keys = self.ctx, self.keys
        Z = self.Zhost if host else self.Zdev
        p0 = self.p0_host if host else self.p0_dev
        p1 = self.p1_host if host else self.p1_dev
        cts = ctx.encrypt_batch(keys, ctx.encode_batch(Z, LEVEL), self.nonces(self.n_in))
        Y = ctx.matmul_cp_plan(keys, self.plan_qkv, cts)
        O = ctx.matmul_cp_plan(keys, self.plan_o, Y[:self.n_in])
        outs = Y[self.n_in:] + O
        masked, _ = ctx.he2mpc_batch(keys, outs, self.nonces(len(outs)), share_out=p1)
        ctx.decrypt_batch(keys, masked, coeff_out=p0)
        return (Y, O, cts) if keep else None

    def graph_step(self):
        """The step with its products, masking and P0's decryption replayed from
        a CUDA graph captured once: each step encodes and encrypts the inputs
        eagerly (fresh nonces) into the captured input ciphertexts, then replays
        QKV, W_O, the 18 maskings and the decryption (their masking nonces are
        those of the capture).  Returns the step function."""
        ctx, keys = self.ctx, self.keys
        cts = ctx.encrypt_batch(keys, ctx.encode_batch(self.Zdev, LEVEL), self.nonces(self.n_in))
        mask_nonces = self.nonces(self.n_out)

        def tail():
            Y = ctx.matmul_cp_plan(keys, self.plan_qkv, cts)
            O = ctx.matmul_cp_plan(keys, self.plan_o, Y[:self.n_in])
            masked, _ = ctx.he2mpc_batch(keys, Y[self.n_in:] + O, mask_nonces, share_out=self.p1_dev)
            ctx.decrypt_batch(keys, masked, coeff_out=self.p0_dev)
            return Y, O, masked

        self.graph, self.graph_out = ctx.capture(tail)

        def step():
            fresh = ctx.encrypt_batch(keys, ctx.encode_batch(self.Zdev, LEVEL), self.nonces(self.n_in))
            for dst, src in zip(cts, fresh):
                ctx.ct_copy(dst, src)
            with self.torch.cuda.stream(self.stream):
                self.graph.replay()
        self.graph_inputs = cts
        return step

    def step_batched(self, S):
        """S sequences through the same plans in one batched pass per product."""
        ctx, keys = self.ctx, self.keys
        seqs = [ctx.encrypt_batch(keys, ctx.encode_batch(self.Zdev, LEVEL), self.nonces(self.n_in))
                for _ in range(S)]
        Ys = ctx.matmul_cp_batch(keys, self.plan_qkv, seqs)
        Os = ctx.matmul_cp_batch(keys, self.plan_o, [Y[:self.n_in] for Y in Ys])
        outs = [y for Y, O in zip(Ys, Os) for y in Y[self.n_in:] + O]
        if getattr(self, "bp0", None) is None or self.bp0.shape[0] != len(outs):
            self.bp0 = self.torch.zeros((len(outs), self.N), dtype=self.torch.uint64, device=self.p0_dev.device)
            self.bp1 = self.torch.zeros_like(self.bp0)
        masked, _ = ctx.he2mpc_batch(keys, outs, self.nonces(len(outs)), share_out=self.bp1)
        ctx.decrypt_batch(keys, masked, coeff_out=self.bp0)

    # baby-step counts of the packed forms (fewest rotations at each geometry)
    PACKED_B1 = {2: (16, 8), 4: (8, 8)}

    def packed(self, per=2):
        """`per` sequences per ciphertext: m = per x 128 rows, k = N/(2 m)
        columns, so one set of rotations serves per x 128 tokens (two: 288 +
        168 rotations per pair against 2 x (216 + 132); four: 384 + 240 per
        four).  Plans, keys (the step's secret, seed 0) and the packed inputs
        are made on first use (any other packing is freed first); returns the
        number of ciphertexts per packed input."""
        if getattr(self, "plan_qkv2", None) is not None and self.per2 != per:
            self.free_packed()
        if getattr(self, "plan_qkv2", None) is None:
            b1_qkv, b1_o = self.PACKED_B1[per]
            m2 = per * M
            k2 = self.N // 2 // m2
            rots = sorted({r for b1 in (b1_qkv, b1_o)
                           for r in [b * m2 for b in range(1, b1)] + [g * b1 * m2 for g in range(1, k2 // b1)]})
            self.keys2 = self.ctx.keygen(0, rots)
            self.plan_qkv2 = self.ctx.cp_plan(m2, D, self.Wqkv, D_QKV, LEVEL, b1_qkv)
            self.plan_o2 = self.ctx.cp_plan(m2, D, self.Wo, D_O, LEVEL - 1, b1_o)
            self.k2, self.per2, self.b1_2 = k2, per, (b1_qkv, b1_o)
            Z2 = pack_columns(np.vstack([self.X] * per), m2, k2)
            self.n_in2 = Z2.shape[0]
            self.Z2dev = self.torch.tensor(Z2, dtype=self.torch.float64, device=self.p0_dev.device)
            self.ctx.sync()
        return self.n_in2

    def step_batched_packed(self, S, keep=False):
        """S sequences (a multiple of the packing), `per2` per ciphertext,
        through the packed plans in one batched pass per product, then masking
        and P0's decryption of every output."""
        n_in = self.n_in2
        ctx, keys = self.ctx, self.keys2
        seqs = [ctx.encrypt_batch(keys, ctx.encode_batch(self.Z2dev, LEVEL), self.nonces(n_in))
                for _ in range(S // self.per2)]
        Ys = ctx.matmul_cp_batch(keys, self.plan_qkv2, seqs)
        Os = ctx.matmul_cp_batch(keys, self.plan_o2, [Y[:n_in] for Y in Ys])
        outs = [y for Y, O in zip(Ys, Os) for y in Y[n_in:] + O]
        if getattr(self, "bp0p", None) is None or self.bp0p.shape[0] != len(outs):
            self.bp0p = self.torch.zeros((len(outs), self.N), dtype=self.torch.uint64, device=self.p0_dev.device)
            self.bp1p = self.torch.zeros_like(self.bp0p)
        masked, _ = ctx.he2mpc_batch(keys, outs, self.nonces(len(outs)), share_out=self.bp1p)
        ctx.decrypt_batch(keys, masked, coeff_out=self.bp0p)
        return (Ys, Os) if keep else None

    def packed_accuracy(self):
        """Largest error of the packed form's first packed input: every
        sequence's QKV and W_O outputs decrypted against FP64."""
        per = self.per2
        Ys, Os = self.step_batched_packed(per, keep=True)
        Y, O = Ys[0], Os[0]
        n_in = self.n_in2
        dec = lambda cts: np.stack([self.ctx.decrypt(self.keys2, c, coeffs=False)[1] for c in cts])  # noqa: E731
        got_qkv = unpack_columns(dec(Y), per * M, self.k2, D_QKV)
        got_o = unpack_columns(dec(O), per * M, self.k2, D_O)
        assert len(Y) == -(-D_QKV // self.k2) and len(O) == -(-D_O // self.k2) and n_in == D // self.k2
        ref_qkv = np.vstack([self.ref_qkv] * per)
        ref_o = np.vstack([self.ref_o] * per)
        return float(max(np.abs(got_qkv - ref_qkv).max(), np.abs(got_o - ref_o).max()))

    def free_packed(self):
        for name in ("plan_qkv2", "plan_o2", "keys2"):
            h = getattr(self, name, None)
            if h is not None:
                h.free()
                setattr(self, name, None)
        self.torch.cuda.empty_cache()

    def accuracy(self):
        Y, O, _ = self.step(keep=True)
        got_qkv = unpack_columns(np.stack([self.ctx.decrypt(self.keys, y, coeffs=False)[1] for y in Y]), M, self.k, D_QKV)
        got_o = unpack_columns(np.stack([self.ctx.decrypt(self.keys, y, coeffs=False)[1] for y in O]), M, self.k, D_O)
        err = np.concatenate([(got_qkv - self.ref_qkv).ravel(), (got_o - self.ref_o).ravel()])
        return float(np.max(np.abs(err))), float(np.mean(err ** 2))

    def cp_bytes(self):
        """HBM bytes of the step's two matmul_cp products: the algorithmic
        minimum (compact FP64 weights, input and output ciphertexts, the
        rotation keys once) beside what the implementation streams (the
        pre-encoded byte-plane plaintext diagonals, the baby-step ciphertexts and
        the partial sums of the MAC)."""
        N, w8 = self.N, 8
        ct = lambda lv: 2 * (lv + 1) * N * w8
        keys = self.keys_bytes
        alg = ((D * D_QKV + D * D_O) * w8 + self.n_in * ct(LEVEL) + 18 * ct(LEVEL - 1)
               + self.n_in * ct(LEVEL - 1) + 6 * ct(LEVEL - 2) + keys)
        qkv, o = self.plan_qkv.info(), self.plan_o.info()
        mac = 0
        for info, lv, nY in ((qkv, LEVEL, 18), (o, LEVEL - 1, 6)):
            mac += info["plaintext_bytes"] + (info["nX"] * info["b1"] + nY * info["G"]) * ct(lv)
        return {"algorithmic_min": int(alg), "as_implemented_mac": int(mac),
                "note": "algorithmic = weights d x d' x 8 B + ciphertexts in/out + 22 rotation keys; "
                        "as implemented = byte-plane plaintexts + baby-step ciphertexts + partial sums (MAC only)"}

    def counts(self):
        qkv, o = self.plan_qkv.info(), self.plan_o.info()
        rot = lambda i: i["nX"] * (i["b1"] - 1) + i["nY"] * (i["G"] - 1)
        return {"rotations": rot(qkv) + rot(o),
                "plaintext_products": qkv["nX"] * qkv["nY"] * self.k + o["nX"] * o["nY"] * self.k,
                "rescales": qkv["nY"] + o["nY"], "he2mpc": self.n_out}


def timed_fn(w, fn, steps, world):
    torch = w.torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    ev0.record(w.stream)
    for _ in range(steps):
        fn()
    ev1.record(w.stream)
    torch.cuda.synchronize()
    w.ctx.sync()  # raises if an encoding of the timed steps overflowed
    barrier(world)
    return ev0.elapsed_time(ev1) / 1e3


def attention_cc(steps, groupings=((8, 4), (16,))):
    """BERT-base attention products on ciphertexts (12 heads, 128 tokens, head
    dim 64, N = 2^16, 12 primes, dnum 4): Q_h K_h^T and Softmax x V_h with
    matmul_cc, one sequence per step, for each head grouping in `groupings`:
    the paper's groups of 8 and 4, and one group of 16 (four all-zero heads:
    at N = 2^16 one ciphertext has room for 16 heads of 128 tokens, Kc = 16,
    so one product pair replaces two, at a third more step-2 products).
    Returns tokens/s and ms of the fastest grouping, and every grouping's
    figures."""
    import torch
    from paper_2508_19525_b300 import blb
    from paper_2508_19525_b300 import workloads as wl
    prm = wl.BERT_CC
    stream = torch.cuda.Stream()
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, prm.dnum, prm.scale, stream=stream)
    L, Dh, H, level = 128, 64, 12, ctx.nQ - 1
    Q, K, V, P = wl.attention_operands(L, H, Dh, seed=3)
    res = {}
    for grouping in groupings:
        plans = {Hg: (ctx.cc_plan(L, Hg, Dh, level), ctx.cc_plan(L, Hg, L, level)) for Hg in set(grouping)}
        rots = sorted({r for pq, pv in plans.values() for r in pq.rotations() + pv.rotations()})
        keys = ctx.keygen(1, rots, relin=True)
        inputs = []
        h0 = 0
        for Hg in grouping:
            pq, pv = plans[Hg]
            heads = [h for h in range(h0, h0 + Hg) if h < H]

            def take(M):
                out = np.zeros((Hg,) + M.shape[1:])
                out[:len(heads)] = M[heads]
                return out
            for kind, plan in (("qk", pq), ("pv", pv)):
                info = plan.info()
                if kind == "qk":
                    A, B = take(Q), np.transpose(take(K), (0, 2, 1))
                else:
                    A = take(P)
                    B = np.concatenate([take(V), np.zeros((Hg, L, L - Dh))], axis=2)
                Az = pack_heads(A, L, Hg, info["Kc"], info["n_c"], rows=False)
                Bz = pack_heads(B, L, Hg, info["Kc"], info["n_c"], rows=True)
                Ac = [ctx.encrypt(keys, ctx.encode(z, level), 7 * c) for c, z in enumerate(Az)]
                Bc = [ctx.encrypt(keys, ctx.encode(z, level), 7 * c + 1) for c, z in enumerate(Bz)]
                inputs.append((plan, Ac, Bc, A, B, Hg, info))
            h0 += Hg

        def one():
            for plan, Ac, Bc, *_ in inputs:
                ctx.matmul_cc_plan(keys, plan, Ac, Bc)
        one()
        ctx.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            one()
        ev1.record(stream)
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3 / steps
        # accuracy of the last products against FP64
        err = 0.0
        for plan, Ac, Bc, A, B, Hg, info in inputs:
            C = ctx.matmul_cc_plan(keys, plan, Ac, Bc)
            zs = np.stack([ctx.decrypt(keys, c, coeffs=False)[1] for c in C])
            got = unpack_head_diagonals(zs, L, Hg, info["Kc"])
            err = max(err, float(np.max(np.abs(got - np.einsum("hik,hkj->hij", A, B)))))
        res["+".join(map(str, grouping))] = {
            "value": round(L / sec, 3), "ms_per_step": round(sec * 1e3, 3), "max_abs_err_vs_fp64": err,
            "products": len(inputs), "rotation_keys": len(rots),
            "rotations": sum(len(p.rotations()) for pq, pv in plans.values() for p in (pq, pv))}
        del inputs, keys
        for pq, pv in plans.values():
            pq.free()
            pv.free()
        torch.cuda.empty_cache()
    best = min(res, key=lambda g: res[g]["ms_per_step"])
    return {"value": res[best]["value"], "unit": UNIT, "ms_per_step": res[best]["ms_per_step"],
            "head_groups": best, "max_abs_err_vs_fp64": res[best]["max_abs_err_vs_fp64"],
            "workload": "BERT-base attention: Q_h K_h^T and Softmax x V_h for 12 heads, L=128, head dim 64, "
                        "N=2^16, 12 primes, dnum 4, one sequence per step; head groupings 8+4 (the paper's) "
                        "and 16 (four zero heads)", "groupings": res}


def conversion_bench(w, reps):
    """The parties' local steps of both conversions (Alg. 1 steps 3-4, Alg. 2
    steps 1-2, App. C.3) for one BERT-base step: C2M of the 18 masked outputs
    (field to ring + decoding of shares, both parties) and M2C of 6 slot-share
    vectors back to the next layer's input level (extension + encoding of
    shares + ring to field, both parties), MPC ring l = 43 at scale 2^-13.  The
    wrap-bit comparisons (MPC protocols) run through their simulated ideal
    functionality and are timed apart."""
    torch, ctx = w.torch, w.ctx
    n_out, n_in, N, s = w.n_out, w.n_in, w.N, w.N // 2
    dev = w.p0_dev.device
    u64 = dict(dtype=torch.uint64, device=dev)
    W0, W1 = torch.zeros((n_out, N, 2), **u64), torch.zeros((n_out, N, 2), **u64)
    Y0, Y1 = torch.zeros((n_out, s), **u64), torch.zeros((n_out, s), **u64)
    V0, V1 = torch.zeros((n_in, s, 2), **u64), torch.zeros((n_in, s, 2), **u64)
    M0 = torch.zeros((n_in, LEVEL + 1, N), **u64)
    M1 = torch.zeros_like(M0)
    scale = ctx.scale
    w.step()
    ids = list(range(n_out))

    def sim_c2m():
        ctx.f2r_wrap_sim(w.p0_dev, w.p1_dev, 7, ids, W0, W1)

    def c2m():
        ctx.c2m_local(0, w.p0_dev, W0, scale, 43, 13, out=Y0)
        ctx.c2m_local(1, w.p1_dev, W1, scale, 43, 13, out=Y1)

    def sim_m2c():
        ctx.ext_wrap_sim(Y0[:n_in], Y1[:n_in], s, 43, 7, ids[:n_in], V0, V1)

    def m2c():
        ctx.m2c_local(0, Y0[:n_in], V0, s, LEVEL, scale, 43, 13, out=M0)
        ctx.m2c_local(1, Y1[:n_in], V1, s, LEVEL, scale, 43, 13, out=M1)

    for f in (sim_c2m, c2m, sim_m2c, m2c):
        f()
    ctx.sync()
    ctx.profile(True)
    t = {name: timed_fn(w, f, reps, 1) / reps * 1e3
         for name, f in (("f2r_wrap_sim", sim_c2m), ("c2m", c2m), ("ext_wrap_sim", sim_m2c), ("m2c", m2c))}
    sites = {site: ctx.profile_read(site) for site in ("c2m", "m2c")}
    ctx.profile(False)
    out = {"workload": f"C2M of {n_out} masked outputs (N=2^15, q_0 60 bits) and M2C of {n_in} slot vectors "
                       f"back to level {LEVEL}, both parties, l=43, sf=13, extended ring Z_2^128",
           "ms": {k: round(v, 4) for k, v in t.items()}, "sites": {}}
    for site, (ms, cnt, nbytes) in sites.items():
        if cnt and ms > 0:
            out["sites"][site] = {"ms_per_call": round(ms / cnt, 4), "calls": cnt,
                                  "algorithmic_bytes_per_call": nbytes // cnt,
                                  "achieved_gbs": round(nbytes / (ms / 1e3) / 1e9, 1)}
    return out


def bert_large_batching(n_seqs=8, plain_chunks=6, ms=(32, 128, 256), groups=(1, 2, 4, 8)):
    """Batching of uneven-length BERT-large-shaped sequences of one client:
    n_seqs sequences with lengths U[16, 512] (seeded), hidden 1024, FFN 4096;
    the ct-pt products QKV (1024 x 3072), FFN up (1024 x 4096) and FFN down
    (4096 x 1024) over all their tokens, laid end to end and cut into m-row
    chunks, N = 2^16, 12 primes, dnum autotuned.
    Plain: 32-row chunks (one ciphertext holds a chunk's 1024 features), one
    chunk per call, the b1 fastest for that form.
    Batched: m in `ms` rows per ciphertext (more tokens through the same
    rotations; the plan's plaintexts grow with m), a group of chunks per
    blb_matmul_cp_batch call (every plaintext streamed once per group); m, b1
    (two candidates per m from the rotation count) and the group size are
    autotuned per product by timing every triple on the product itself."""
    import torch
    from paper_2508_19525_b300 import batching as bt
    from paper_2508_19525_b300 import blb
    from paper_2508_19525_b300 import workloads as wl
    prm = wl.BERT_CC
    stream = torch.cuda.Stream()
    # digit count of key switching, timed on the device (the special primes fix
    # alpha = ceil(12 / dnum) <= 3, so dnum in {4, 6, 12})
    dnum, dnum_t = bt.autotune_dnum(
        lambda dn: blb.Context(prm.logN, prm.q_bits, prm.p_bits, dn, prm.scale, stream=stream), (4, 6, 12), 32)
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, dnum, prm.scale, stream=stream)
    ntt_split, ntt_radix, ntt_us = ctx.ntt_autotune(256)
    level, slots = ctx.nQ - 1, ctx.N // 2
    rng = np.random.default_rng(44)
    lengths = rng.integers(16, 513, n_seqs)
    T = int(lengths.sum())
    products = [("qkv", 1024, 3072, 41), ("ffn_up", 1024, 4096, 42), ("ffn_down", 4096, 1024, 43)]
    cands = {(name, m): bt.cp_b1_candidates(m, d, d_out, slots) for name, d, d_out, _ in products for m in ms}
    t0 = time.perf_counter()
    rots = sorted({r for (name, m), bs in cands.items() for b1 in bs for r in bt.cp_rotations(m, slots // m, b1)})
    keys = ctx.keygen(6, rots)
    ctx.sync()
    keygen_s = time.perf_counter() - t0
    out = {"workload": f"{n_seqs} BERT-large-shaped sequences, lengths U[16,512] (total {T} tokens), "
                       f"QKV 1024x3072 + FFN 1024x4096 + 4096x1024 ct-pt products over m-row chunks, "
                       f"N=2^16, 12 primes, dnum autotuned", "lengths": [int(x) for x in lengths], "tokens": T,
           "rotation_keys": len(rots),
           "autotuned": {"dnum": dnum, "dnum_s_per_rotation": {str(k): round(v, 5) for k, v in dnum_t.items()},
                         "ntt_split": ntt_split, "ntt_radix": ntt_radix, "ntt_us_per_row_direction": ntt_us_json(ntt_us)},
           "keygen_s": round(keygen_s, 2), "products": {}}
    tot_b = tot_p = tot_g = 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def encrypt_chunks(X, m):
        k = slots // m
        n_cts = -(-X.shape[1] // k)
        Z = bt.pack_chunks(X, m, k, n_cts)
        return [ctx.encrypt_batch(keys, ctx.encode_batch(Z[c], level), [1000 * c + i for i in range(n_cts)])
                for c in range(len(Z))]

    for name, d, d_out, seed in products:
        X = wl.uniform((T, d), seed=seed)
        W = wl.uniform((d, d_out), seed=seed + 100)
        tune_all, best, pb32 = {}, None, None
        for m in ms:
            # a plan's plaintexts grow as m: skip an m whose plan would take
            # more than half of the device (other products' keys and
            # ciphertexts, and the attention products later, need the rest)
            if pb32 is not None and pb32 * m // 32 > 0.5 * torch.cuda.get_device_properties(0).total_memory:
                continue
            chunks = encrypt_chunks(X, m)
            n_cts = len(chunks[0])
            # baby-step ciphertexts of a call: group x inputs x b1 x 2 polynomials
            grp = [x for x in groups if x * n_cts * max(cands[(name, m)]) * ctx.N * 8 * 2 * ctx.nQ < 40e9] or [1]
            try:
                (b1, g), tune = bt.autotune(ctx, keys, m, d, W, d_out, level, chunks, cands[(name, m)], grp)
            except ValueError:
                continue
            for (b, gg), t in tune.items():
                tune_all[f"m={m},b1={b},group={gg}"] = round(t, 4)
            if m == 32:
                # plain: 32-row chunks, one per call, with the b1 fastest for that form
                b1p = min((b for b, gg in tune if gg == 1), key=lambda b: tune[(b, 1)])
                plan_p = ctx.cp_plan(32, d, W, d_out, level, b1p)
                pb32 = plan_p.info()["plaintext_bytes"]
                npl = min(plain_chunks, len(chunks))
                ctx.matmul_cp_plan(keys, plan_p, chunks[0])
                ev0.record(stream)
                for c in range(npl):
                    ctx.matmul_cp_plan(keys, plan_p, chunks[c])
                ev1.record(stream)
                torch.cuda.synchronize()
                plain_per_chunk = ev0.elapsed_time(ev1) / 1e3 / npl
                n_plain_chunks = len(chunks)
                plan_p.free()
            per_tok = tune[(b1, g)] / m
            if best is None or per_tok < best[0]:
                best = (per_tok, m, b1, g)
            del chunks
            torch.cuda.empty_cache()
        _, m, b1, g = best
        k = slots // m
        chunks = encrypt_chunks(X, m)
        plan = ctx.cp_plan(m, d, W, d_out, level, b1)
        bt.run_batched(ctx, keys, plan, chunks[:g], g)
        ctx.sync()
        ev0.record(stream)
        Y = bt.run_batched(ctx, keys, plan, chunks, g)
        ev1.record(stream)
        torch.cuda.synchronize()
        batched_s = ev0.elapsed_time(ev1) / 1e3
        # the product over every chunk captured once as one CUDA graph (the
        # arenas are already sized by the eager run), replayed and timed
        l0 = blb.kernel_launches()
        graph, Yg = ctx.capture(lambda: bt.run_batched(ctx, keys, plan, chunks, g), warmup=False)
        graph_kernels = blb.kernel_launches() - l0
        with torch.cuda.stream(stream):
            graph.replay()
            ev0.record(stream)
            graph.replay()
            ev1.record(stream)
        torch.cuda.synchronize()
        graph_s = ev0.elapsed_time(ev1) / 1e3
        graph_same = all(np.array_equal(ctx.ct_export(a), ctx.ct_export(b))
                         for c in (0, len(chunks) - 1) for a, b in zip(Yg[c], Y[c]))
        del graph, Yg
        err = 0.0
        for c in (0, len(chunks) - 1):
            got = bt.unpack_chunk([ctx.decrypt(keys, y, coeffs=False)[1] for y in Y[c]], m, k, d_out)
            rows = min(m, T - c * m)
            err = max(err, float(np.abs(got[:rows] - X[c * m:c * m + rows] @ W).max()))
        plain_s = plain_per_chunk * n_plain_chunks
        out["products"][name] = {
            "m": m, "b1": b1, "G": k // b1,
            "autotune_s_per_chunk": tune_all,
            "rotations_per_chunk": bt.cp_rotation_count(m, d, d_out, slots, b1),
            "chunks": len(chunks), "chunks_per_call": g,
            "batched_s": round(batched_s, 3), "batched_tokens_per_s": round(T / batched_s, 1),
            "plain": {"m": 32, "b1": b1p, "chunks": n_plain_chunks, "s_per_chunk": round(plain_per_chunk, 4),
                      "rotations_per_chunk": bt.cp_rotation_count(32, d, d_out, slots, b1p)},
            "plain_tokens_per_s": round(T / plain_s, 1),
            "speedup": round(plain_s / batched_s, 3),
            "graph_s": round(graph_s, 3), "graph_tokens_per_s": round(T / graph_s, 1),
            "graph_kernel_nodes": int(graph_kernels), "graph_equals_eager": bool(graph_same),
            "plaintext_bytes": plan.info()["plaintext_bytes"], "max_abs_err_vs_fp64": err}
        tot_b += batched_s
        tot_g += graph_s
        tot_p += plain_s
        del chunks, Y
        plan.free()
        torch.cuda.empty_cache()
    out["batched_tokens_per_s"] = round(T / tot_b, 1)
    out["graph_tokens_per_s"] = round(T / tot_g, 1)
    out["graph_speedup_vs_plain"] = round(tot_p / tot_g, 3)
    out["plain_tokens_per_s"] = round(T / tot_p, 1)
    out["speedup"] = round(tot_p / tot_b, 3)
    out["peak_device_gb"] = round(torch.cuda.max_memory_allocated() / 1e9, 1)
    del keys
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    att = bert_large_batch_attention(ctx, stream, [int(x) for x in lengths])
    out["attention"] = att
    out["ct_pt_and_attention_tokens_per_s"] = round(T / (tot_b + att["s_total"]), 1)
    out["ct_pt_and_attention_plain_tokens_per_s"] = round(T / (tot_p + att["plain"]["s_total"]), 1)
    return out


def bert_large_batch_attention(ctx, stream, lengths, heads=16, dh=64, seed=45, check=2, packed=True):
    """The ct-ct attention products of the BERT-large-shaped sequences,
    Q_h K_h^T and P_h V_h (matmul_cc, Sec. 5.1), each length padded to a power
    of two L >= 64 (Kc = N/2/(16 L) <= L) with zero rows and columns past the
    sequence's end, V_h padded to L columns for the square diagonal-packed
    output.  Two forms, each with its own plans and Galois keys:
      plain:  one product pair per sequence, its 16 heads in one group;
      packed: the sequences of one padded length S at a time in one product
              pair, as S x 16 heads of one group (batching.cc_pack_groups), so
              that step 3's rotations and the relinearizations are shared.
    Each product is timed with CUDA events after one warm-up product per plan;
    the first `check` sequences are decrypted against FP64 in both forms.  In
    the plain form, for up to 8 sequences, every product is also captured as
    one CUDA graph and a replay is timed (its first product's limbs compared
    with the eager ones)."""
    import torch
    from paper_2508_19525_b300 import batching as bt
    from paper_2508_19525_b300 import layer as ly
    from paper_2508_19525_b300 import workloads as wl
    level = ctx.nQ - 1
    pad = [max(64, 1 << int(np.ceil(np.log2(x)))) for x in lengths]
    slots = ctx.N // 2

    def operands(si, l, Lp):
        Q, K, V, P = wl.attention_operands(Lp, heads, dh, seed=seed + si)
        for M in (Q, K, V):
            M[:, l:] = 0.0
        P[:, l:, :] = 0.0
        P[:, :, l:] = 0.0
        P[:, :l] /= P[:, :l].sum(axis=2, keepdims=True)
        Vp = np.concatenate([V, np.zeros((heads, Lp, Lp - dh))], axis=2)
        return (("qk", Q, np.transpose(K, (0, 2, 1))), ("pv", P, Vp))

    def run(groups, graph_ok):
        plans = {}
        for Lp, idx in groups:
            Hg = heads * len(idx)
            if (Lp, Hg) not in plans:
                plans[(Lp, Hg)] = (ctx.cc_plan(Lp, Hg, dh, level), ctx.cc_plan(Lp, Hg, Lp, level))
        rots = sorted({r for pq, pv in plans.values() for r in pq.rotations() + pv.rotations()})
        t0 = time.perf_counter()
        keys = ctx.keygen(46, rots, relin=True)
        ctx.sync()
        keygen_s = time.perf_counter() - t0
        work = []                      # (sequences, kind, plan, A_cts, B_cts, padded length, Hg, FP64 products)
        for gi, (Lp, idx) in enumerate(groups):
            Hg = heads * len(idx)
            per = [operands(si, lengths[si], Lp) for si in idx]
            for k, plan in enumerate(plans[(Lp, Hg)]):
                A = bt.stack_heads([p[k][1] for p in per])
                B = bt.stack_heads([p[k][2] for p in per])
                info = plan.info()
                Az = ly.pack_heads(A, Lp, Hg, info["Kc"], info["n_c"], rows=False)
                Bz = ly.pack_heads(B, Lp, Hg, info["Kc"], info["n_c"], rows=True)
                n, nonce = info["n_c"], 100000 * gi + 50000 * k
                Ac = ctx.encrypt_batch(keys, ctx.encode_batch(Az, level), [nonce + c for c in range(n)])
                Bc = ctx.encrypt_batch(keys, ctx.encode_batch(Bz, level), [nonce + 20000 + c for c in range(n)])
                want = [np.einsum("hik,hkj->hij", p[k][1], p[k][2]) if si < check else None
                        for si, p in zip(idx, per)]
                work.append((idx, per[0][k][0], plan, Ac, Bc, Lp, Hg, want))
        warm = set()
        for _, _, plan, Ac, Bc, _, _, _ in work:      # one untimed product per plan (arenas)
            if id(plan) not in warm:
                ctx.matmul_cc_plan(keys, plan, Ac, Bc)
                warm.add(id(plan))
        ctx.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        per_len, total, err, eager_first = {}, 0.0, 0.0, None
        for idx, kind, plan, Ac, Bc, Lp, Hg, want in work:
            ev0.record(stream)
            C = ctx.matmul_cc_plan(keys, plan, Ac, Bc)
            ev1.record(stream)
            torch.cuda.synchronize()
            sec = ev0.elapsed_time(ev1) / 1e3
            total += sec
            e = per_len.setdefault(str(Lp), {"sequences": 0, "products": 0, "qk_ms": 0.0, "pv_ms": 0.0})
            e[kind + "_ms"] += sec * 1e3
            if kind == "qk":
                e["sequences"] += len(idx)
                e["products"] += 1
            if any(x is not None for x in want):
                Z = np.stack([ctx.decrypt(keys, c, coeffs=False)[1] for c in C])
                got = bt.split_heads(ly.unpack_diagonals(Z, Lp, Hg, plan.info()["Kc"]), len(idx))
                for g_, w_ in zip(got, want):
                    if w_ is not None:
                        err = max(err, float(np.abs(g_ - w_).max()))
            if eager_first is None:
                eager_first = [ctx.ct_export(c) for c in C]
            del C
        # every product captured as one CUDA graph, then replayed (up to 8
        # sequences: the graph's pool keeps every product's temporaries)
        graph_s = graph_same = None
        if graph_ok:
            torch.cuda.empty_cache()
            graph, Cg = ctx.capture(lambda: [ctx.matmul_cc_plan(keys, w_[2], w_[3], w_[4]) for w_ in work],
                                    warmup=False)
            with torch.cuda.stream(stream):
                graph.replay()
                ev0.record(stream)
                graph.replay()
                ev1.record(stream)
            torch.cuda.synchronize()
            graph_s = ev0.elapsed_time(ev1) / 1e3
            graph_same = all(np.array_equal(ctx.ct_export(a), b) for a, b in zip(Cg[0], eager_first))
            del graph, Cg
        del work
        for e in per_len.values():
            e["qk_ms_per_sequence"] = round(e.pop("qk_ms") / e["sequences"], 2)
            e["pv_ms_per_sequence"] = round(e.pop("pv_ms") / e["sequences"], 2)
        info = {f"L={Lp},Hg={Hg}": {k: v for k, v in pv.info().items() if k in ("Kc", "n_c", "b1s1", "b1s2",
                                                                                   "c_chunk", "t_chunk")}
                for (Lp, Hg), (_, pv) in plans.items()}
        for pq, pv in plans.values():
            pq.free()
            pv.free()
        del keys
        torch.cuda.empty_cache()
        T = int(sum(lengths))
        return {"rotation_keys": len(rots), "keygen_s": round(keygen_s, 2), "per_padded_length": per_len,
                "pv_plans": info, "s_total": round(total, 4), "tokens_per_s": round(T / total, 1),
                "graph_s": None if graph_s is None else round(graph_s, 4),
                "graph_tokens_per_s": None if graph_s is None else round(T / graph_s, 1),
                "graph_equals_eager": None if graph_same is None else bool(graph_same),
                "max_abs_err_vs_fp64": err}

    plain = run([(Lp, [i]) for i, Lp in enumerate(pad)], len(lengths) <= 8)
    out = {"workload": f"{len(lengths)} sequences, Q K^T and P V, {heads} heads of dim {dh}, lengths padded to "
                       f"powers of two >= 64, N=2^16, 12 primes",
           "padded_lengths": pad, "plain": plain}
    if packed:
        groups = bt.cc_pack_groups(pad, heads, slots)
        pk = run(groups, False)
        pk["sequences_per_product"] = [len(i) for _, i in groups]
        out["packed"] = pk
        out["packed_speedup_vs_plain"] = round(plain["s_total"] / pk["s_total"], 3)
    best = out.get("packed", plain)
    out["s_total"] = best["s_total"]
    out["tokens_per_s"] = best["tokens_per_s"]
    out["peak_device_gb"] = round(torch.cuda.max_memory_allocated() / 1e9, 1)
    return out


def layer_bench():
    """One BERT-base encoder layer the hybrid way (paper_2508_19525_b300/layer.py):
    the linear operators in fused HE blocks (QKV + Q K^T, softmax exponential,
    normalisation + P V + W_O + residual + LN1 head, LN1 tail + W_1 + GeLU
    polynomials, W_2 + residual + LN2 head, LN2 tail) with CKKS <-> MPC
    conversions at every boundary; MPC nonlinear steps simulated.  Returns the
    seconds per segment (HE kernels; conversions + simulated MPC) and the error
    against the FP64 layer with the same approximations."""
    import torch
    from paper_2508_19525_b300 import blb
    from paper_2508_19525_b300 import layer as ly
    from paper_2508_19525_b300 import workloads as wl
    ctx = blb.Context(*[getattr(wl.BERT_CP, a) for a in ("logN", "q_bits", "p_bits", "dnum", "scale")])
    big = blb.Context(*[getattr(wl.BERT_CC, a) for a in ("logN", "q_bits", "p_bits", "dnum", "scale")])
    t0 = time.perf_counter()
    lay = ly.BertLayer(ctx, big)
    rs, rb = lay.rotations()
    keys, keysb = ctx.keygen(21, rs, relin=True), big.keygen(22, rb, relin=True)
    ctx.sync()
    setup_s = time.perf_counter() - t0
    X = np.random.default_rng(23).uniform(-1, 1, (lay.L, lay.d))
    lay.forward(X, keys, keysb, ly.Mpc(24))                     # warm-up
    Y, he, conv = lay.forward(X, keys, keysb, ly.Mpc(25))
    err = float(np.abs(Y - lay.reference(X)).max())
    del lay, keys, keysb
    torch.cuda.empty_cache()
    return {"workload": "BERT-base encoder layer (128 tokens, 768 hidden, 12 heads, FFN 3072): fused HE blocks "
                        "on N=2^15 / 8 primes and N=2^16 / 12 primes, CKKS<->MPC conversions at every boundary, "
                        "MPC nonlinear steps simulated",
            "he_s": {k: round(v, 4) for k, v in he.items()}, "conversion_and_mpc_s": {k: round(v, 4) for k, v in conv.items()},
            "he_total_s": round(sum(he.values()), 4), "conversion_total_s": round(sum(conv.values()), 4),
            "setup_s": round(setup_s, 2), "rotation_keys": [len(rs), len(rb)], "max_abs_err_vs_fp64": err}


def layernorm_bench(steps, seqs=(1, 8)):
    """The HE steps of the secure LayerNorm before rsqrt (Alg. LayerNorm lines
    1-6) on BERT-base activations: 128 tokens x 768 features packed
    spatial-first in 6 ciphertexts of 128 columns at N = 2^15, level 7: row
    sums by rotate-and-sum (7 rotations, no mask: Sec. 4.2.1's sum -> scalar
    fusion), mean, centring, squares, variance.  Timed for one sequence and
    for a batch of sequences per call."""
    import torch
    from paper_2508_19525_b300 import blb
    from paper_2508_19525_b300 import workloads as wl
    prm = wl.BERT_CP
    stream = torch.cuda.Stream()
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, prm.dnum, prm.scale, stream=stream)
    s, L = ctx.N // 2, M
    k = s // L
    nc = D // k
    keys = ctx.keygen(2, [L << i for i in range(int(np.log2(k)))], relin=True)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (L, D))
    Z = np.zeros((nc, s))
    for c in range(nc):
        Z[c] = X[:, c * k:(c + 1) * k].T.reshape(-1)
    cts = ctx.encrypt_batch(keys, ctx.encode_batch(Z, LEVEL), list(range(nc)))
    out = {"workload": f"LayerNorm head (Alg. LayerNorm lines 1-6): {L} tokens x {D} features in {nc} "
                       f"ciphertexts, N=2^15, level {LEVEL} -> 4, {int(np.log2(k))} rotations per sum", "per_call": {}}
    for S in seqs:
        X_in = cts * S
        ctx.layernorm_head(keys, X_in, L, D, nc)
        ctx.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            ctx.layernorm_head(keys, X_in, L, D, nc)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        out["per_call"][str(S)] = {"ms": round(ms, 3), "tokens_per_s": round(S * L / (ms / 1e3), 1)}
    _, var = ctx.layernorm_head(keys, cts, L, D, nc)
    v = ctx.decrypt(keys, var[0], coeffs=False)[1].reshape(k, L)
    out["max_abs_err_var_vs_fp64"] = float(np.abs(v - X.var(axis=1)[None, :]).max())
    return out


def serving_bench(n_requests=64, rate=20.0, sat_rate=400.0, budget_gb=24, max_batch=8):
    """Continuous batching of encrypted linear-layer requests (one client and key
    set per request) against one request per launch; BERT-base-shaped and
    GPT2-base-shaped weights (hidden 768), sequence lengths U[16, 128] padded to
    32 / 64 / 128, N=2^15, 8 primes.  Poisson arrivals (seeded)."""
    import torch
    from paper_2508_19525_b300 import blb
    from paper_2508_19525_b300 import workloads as wl
    from paper_2508_19525_b300.serving import GpuEngine, Request, Server, bucket, percentile
    prm = wl.BERT_CP
    stream = torch.cuda.Stream()
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, prm.dnum, prm.scale, stream=stream)
    buckets = (32, 64, 128)
    rng = np.random.default_rng(2024)
    plans = {}
    for name, seed in (("bert", 0), ("gpt2", 1)):
        Wq = rng.uniform(-1, 1, (D, D_QKV))
        Wo = rng.uniform(-1, 1, (D, D_O))
        for m in buckets:
            k = ctx.N // 2 // m
            b1 = 1
            while b1 * b1 < k:
                b1 *= 2
            rots = [b * m for b in range(1, b1)] + [g * b1 * m for g in range(1, k // b1)]
            plans[(name, m)] = (ctx.cp_plan(m, D, Wq, D_QKV, LEVEL, b1), ctx.cp_plan(m, D, Wo, D_O, LEVEL - 1, b1), rots)
    ctx.sync()

    def requests(rate_rps, seed):
        r = np.random.default_rng(seed)
        t, out = 0.0, []
        for i in range(n_requests):
            t += r.exponential(1.0 / rate_rps)
            seq = int(r.integers(16, max(buckets) + 1))
            out.append(Request(rid=i, client_seed=10_000 + i, model="bert" if i % 2 else "gpt2", seq=seq,
                               m=bucket(seq, buckets), arrival=t, X=r.uniform(-1, 1, (seq, D))))
        return out

    def run(rate_rps, mb):
        reqs = requests(rate_rps, seed=int(rate_rps))
        srv = Server(GpuEngine(ctx, plans, LEVEL, D, D_QKV), budget_bytes=budget_gb << 30, max_batch=mb)
        t0 = time.perf_counter()
        done = srv.run(reqs)
        span = time.perf_counter() - t0
        lat = [r.latency * 1e3 for r in done]
        return {"p50_ms": round(percentile(lat, 50), 2), "p99_ms": round(percentile(lat, 99), 2),
                "tokens_per_s": round(sum(r.seq for r in done) / span, 1),
                "mean_batch": round(float(np.mean([n for _, n in srv.iterations])), 2),
                "iterations": len(srv.iterations)}

    run(rate, max_batch)  # warm-up (plans, kernels, allocator)
    out = {"workload": f"{n_requests} requests, Poisson {rate:g} req/s, half BERT-base- and half GPT2-base-shaped "
                       "weights (768 -> 2304 then 768 -> 768, masking of every output), sequence lengths "
                       "U[16,128] padded to 32/64/128, each request its own client key set; N=2^15, 8 primes",
           "budget_gb": budget_gb, "max_batch": max_batch,
           "batched": run(rate, max_batch), "plain": run(rate, 1),
           "saturated": {"rate_rps": sat_rate, "batched": run(sat_rate, max_batch), "plain": run(sat_rate, 1)}}
    ctx.sync()
    return out


def serving_n65536_bench(n_requests=32, rate=20.0, light_rate=2.0, n_light=12, budget_gb=80, max_batch=4, group=4,
                       m=32, b1=32, m_batched=128, b1_batched=32):
    """Continuous batching at the serving configuration's own parameters:
    N = 2^16, 12 primes, dnum 4; Poisson arrivals at `rate` req/s, half
    GPT2-base-shaped requests (hidden 768, lengths U[32, 1024]) and half
    BERT-base-shaped ones (U[16, 512]), each its own client key set.  Every
    request is cut into chunks of rows, one plan pair per model (QKV 768 ->
    2304, output projection 768 -> 768).  Plain: m-row chunks (k = 1024
    columns per ciphertext hold a chunk's 768 features), one request per
    iteration and one chunk per product.  Batched: m_batched-row chunks (more
    of a request's tokens through each ciphertext's rotations), a stage of up
    to `max_batch` requests as cross-client products over `group` chunks
    each.  The two forms run one after the other, each with its own plans.  A
    second, shorter run at `light_rate` req/s (below what one GPU serves) shows
    the batched form's latency without queueing."""
    import torch
    from paper_2508_19525_b300 import blb
    from paper_2508_19525_b300 import batching as bt
    from paper_2508_19525_b300 import workloads as wl
    from paper_2508_19525_b300.serving import ChunkEngine, Request, Server, percentile
    prm = wl.BERT_CC
    stream = torch.cuda.Stream()
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, 4, prm.scale, stream=stream)
    level = ctx.nQ - 1
    rng = np.random.default_rng(2025)
    weights = {name: (rng.uniform(-1, 1, (D, D_QKV)), rng.uniform(-1, 1, (D, D_O))) for name in ("bert", "gpt2")}

    def make_plans(mm, bb):
        rots = bt.cp_rotations(mm, ctx.N // 2 // mm, bb)
        t0 = time.perf_counter()
        plans = {name: (ctx.cp_plan(mm, D, Wq, D_QKV, level, bb), ctx.cp_plan(mm, D, Wo, D_O, level - 1, bb), rots)
                 for name, (Wq, Wo) in weights.items()}
        ctx.sync()
        gb = sum(p.info()["plaintext_bytes"] for q, o, _ in plans.values() for p in (q, o)) / 1e9
        return plans, time.perf_counter() - t0, gb

    def free_plans(plans):
        for q, o, _ in plans.values():
            q.free()
            o.free()
        torch.cuda.empty_cache()

    def requests(n, seed, mm, rps=rate):
        r = np.random.default_rng(seed)
        t, out = 0.0, []
        for i in range(n):
            t += r.exponential(1.0 / rps)
            gpt = i % 2 == 0
            seq = int(r.integers(32, 1025)) if gpt else int(r.integers(16, 513))
            out.append(Request(rid=i, client_seed=20_000 + i, model="gpt2" if gpt else "bert", seq=seq, m=mm,
                               arrival=t, X=r.uniform(-1, 1, (seq, D))))
        return out

    def run(plans, mm, reqs, mb, grp):
        srv = Server(ChunkEngine(ctx, plans, level, D, D_QKV, mm, group=grp), budget_bytes=budget_gb << 30,
                     max_batch=mb)
        t0 = time.perf_counter()
        done = srv.run(reqs)
        span = time.perf_counter() - t0
        lat = [r.latency * 1e3 for r in done]
        return {"p50_ms": round(percentile(lat, 50), 1), "p99_ms": round(percentile(lat, 99), 1),
                "tokens_per_s": round(sum(r.seq for r in done) / span, 1), "span_s": round(span, 2),
                "mean_batch": round(float(np.mean([n for _, n in srv.iterations])), 2),
                "iterations": len(srv.iterations)}

    reqs = requests(n_requests, seed=7, mm=m)
    out = {"workload": f"{n_requests} requests, Poisson {rate:g} req/s, half GPT2-base-shaped (lengths U[32,1024]) "
                       f"and half BERT-base-shaped (U[16,512]); QKV 768x2304 then output projection 768x768 and "
                       f"masking of every output; N=2^16, 12 primes, dnum 4, each request its own client key set",
           "tokens": int(sum(r.seq for r in reqs)), "budget_gb": budget_gb, "max_batch": max_batch,
           "chunks_per_product": group}
    plans, enc_s, gb = make_plans(m_batched, b1_batched)
    rots = plans["bert"][2]
    run(plans, m_batched, requests(4, seed=1, mm=m_batched), max_batch, group)  # warm-up (kernels, arenas)
    out["batched"] = run(plans, m_batched, requests(n_requests, seed=7, mm=m_batched), max_batch, group)
    out["batched"].update(m=m_batched, b1=b1_batched, plaintext_gb=round(gb, 1), encode_s=round(enc_s, 2),
                          rotation_keys_per_client=len(rots),
                          key_gb_per_client=round(len(rots) * ctx.key_bytes() / 1e9, 1))
    light = requests(n_light, seed=11, mm=m_batched, rps=light_rate)
    out["light"] = {"rate_rps": light_rate, "requests": n_light, "tokens": int(sum(r.seq for r in light)),
                    "batched": run(plans, m_batched, light, max_batch, group)}
    free_plans(plans)
    plans, enc_s, gb = make_plans(m, b1)
    rots = plans["bert"][2]
    run(plans, m, requests(2, seed=1, mm=m), 1, 1)  # warm-up
    out["plain"] = run(plans, m, requests(n_requests, seed=7, mm=m), 1, 1)
    out["plain"].update(m=m, b1=b1, plaintext_gb=round(gb, 1), encode_s=round(enc_s, 2),
                        rotation_keys_per_client=len(rots), key_gb_per_client=round(len(rots) * ctx.key_bytes() / 1e9, 1))
    free_plans(plans)
    out["speedup"] = round(out["batched"]["tokens_per_s"] / out["plain"]["tokens_per_s"], 3)
    return out


def timed(w, steps, host, world):
    torch = w.torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0.record(w.stream)
    for _ in range(steps):
        w.step(host=host)
    ev1.record(w.stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    w.ctx.sync()  # raises if an encoding of the timed steps overflowed
    barrier(world)
    return ev0.elapsed_time(ev1) / 1e3, wall


def traffic_ratio(path):
    """The `traffic_ratio:` line of an ncu summary (DRAM bytes per algorithmic byte)."""
    try:
        for ln in open(path):
            if ln.startswith("traffic_ratio:"):
                return float(ln.split(":", 1)[1])
    except OSError:
        pass
    return None


def measure_int_peaks(q, stream):
    """This GPU's integer-pipe rates for the ALU rooflines (the register-only
    butterfly and 128-bit multiply-add kernels of libblb_peaks.so,
    include/blb_peaks.h), on the workload's stream."""
    import ctypes
    from paper_2508_19525_b300 import build
    f = ctypes.CDLL(build.build_peaks()).blb_peaks_int_rates
    f.argtypes = [ctypes.c_uint64, ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_double)] * 4
    v = [ctypes.c_double() for _ in range(4)]
    rc = f(q, stream, *[ctypes.byref(x) for x in v])
    if rc:
        raise RuntimeError(f"blb_peaks_int_rates failed ({rc})")
    g = ctypes.CDLL(build.build_peaks()).blb_peaks_reduce_rate
    g.argtypes = [ctypes.c_uint64, ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_double)] * 2
    red = [ctypes.c_double() for _ in range(2)]
    rc = g(q, stream, *[ctypes.byref(x) for x in red])
    if rc:
        raise RuntimeError(f"blb_peaks_reduce_rate failed ({rc})")
    return {"bfly_per_s": v[0].value, "mad128_per_s": v[1].value, "reduce128_per_s": red[0].value,
            "bfly_per_sm_cycle": v[2].value, "mad128_per_sm_cycle": v[3].value,
            "reduce128_per_sm_cycle": red[1].value}


def run_blb(args):
    world, rank, local = dist_env()
    import torch
    dist_init(world, "nccl")
    torch.cuda.set_device(local)
    from paper_2508_19525_b300 import blb
    w = Workload(torch.device("cuda", local))
    for _ in range(args.warmup):
        w.step()
    # device-resident timed region, with CUDA events around the dominant
    # kernel's launches (cp_mac) and clock samples
    clocks = Clocks(local)
    w.ctx.profile(True, only="cp_mac")
    launches0 = blb.kernel_launches()
    clocks.start()
    dev_s, _ = timed(w, args.steps, False, world)
    clk = clocks.stop()
    launches = blb.kernel_launches() - launches0
    sites = {"cp_mac": w.ctx.profile_read("cp_mac")}
    # the other launch sites from a second pass of the same steps with every
    # site bracketed (their events cost the step about 1.5 %, so the timed
    # region above brackets only cp_mac)
    w.ctx.profile(True)
    prof_s, _ = timed(w, args.steps, False, world)
    sites.update({s: w.ctx.profile_read(s) for s in ("keyswitch", "ntt", "intt", "intt_gather")})
    ks_ops = w.ctx.profile_read_ops("keyswitch")
    w.ctx.profile(False)
    int_peaks = measure_int_peaks(w.ctx.primes[0], w.stream.cuda_stream)
    value, dev_max = aggregate(dev_s, TOKENS_PER_STEP * args.steps, world)
    # end to end from pinned host buffers
    for _ in range(max(1, args.warmup // 2)):
        w.step(host=True)
    _, e2e_wall = timed(w, args.steps, True, world)
    e2e_value, _ = aggregate(e2e_wall, TOKENS_PER_STEP * args.steps, world)
    max_err, mse = w.accuracy()
    # batched: several sequences share each plaintext stream
    batched = None
    if args.batch > 1:
        w.step_batched(args.batch)
        bsteps = max(1, min(10, args.steps // 2))
        bsec = timed_fn(w, lambda: w.step_batched(args.batch), bsteps, world)
        bval, _ = aggregate(bsec, TOKENS_PER_STEP * args.batch * bsteps, world)
        # where a batched step's time goes (CUDA events per launch site, one step)
        w.ctx.profile(True)
        w.step_batched(args.batch)
        w.ctx.sync()
        bsites = {s_: round(w.ctx.profile_read(s_)[0], 3) for s_ in ("cp_mac", "keyswitch", "ntt", "intt")}
        w.ctx.profile(False)
        same = {"value": round(bval, 3), "unit": UNIT,
                "ms_per_step": round(bsec * 1e3 / bsteps, 3), "speedup_vs_plain": round(bval / value, 3),
                "site_ms_one_step": bsites,
                "form": "one sequence per ciphertext (the plain form's plans, m = 128), every plaintext streamed "
                        "once for all sequences",
                "mac_kernel": "automatic: mma.sync in 4-sequence launches for these plans (nine and three 16-output "
                              "blocks); the tcgen05 kernel is chosen for single-block plans at 8 sequences"}
        batched = {"sequences_per_step": args.batch, "same_packing": same}
        from paper_2508_19525_b300.batching import cp_rotation_count as bt_rot
        for per, name in ((2, "two_per_ciphertext"), (4, "four_per_ciphertext")):
            if args.batch % per:
                continue
            # several sequences per ciphertext (m = per x 128): one set of rotations per packed input
            w.packed(per)
            w.step_batched_packed(args.batch)
            psec = timed_fn(w, lambda: w.step_batched_packed(args.batch), bsteps, world)
            pval, _ = aggregate(psec, TOKENS_PER_STEP * args.batch * bsteps, world)
            w.ctx.profile(True)
            w.step_batched_packed(args.batch)
            w.ctx.sync()
            psites = {s_: round(w.ctx.profile_read(s_)[0], 3) for s_ in ("cp_mac", "keyswitch", "ntt", "intt")}
            w.ctx.profile(False)
            k2 = w.k2
            batched[name] = {
                "value": round(pval, 3), "unit": UNIT, "ms_per_step": round(psec * 1e3 / bsteps, 3),
                "speedup_vs_plain": round(pval / value, 3), "site_ms_one_step": psites,
                "max_abs_err_vs_fp64": w.packed_accuracy(),
                "form": f"{per} sequences per ciphertext (m = {per * M} rows, k = {k2} columns; b1 = {w.b1_2[0]} for "
                        f"QKV, {w.b1_2[1]} for W_O), plaintexts {per}x, streamed once for all packed inputs",
                "rotations_per_packed_input": [bt_rot(per * M, D, D_QKV, w.N // 2, w.b1_2[0]),
                                               bt_rot(per * M, D, D_O, w.N // 2, w.b1_2[1])],
                "plaintext_bytes": w.plan_qkv2.info()["plaintext_bytes"] + w.plan_o2.info()["plaintext_bytes"]}
            w.free_packed()
        best = max((v for v in batched.values() if isinstance(v, dict)), key=lambda v: v["value"])
        batched.update(value=best["value"], unit=UNIT, ms_per_step=best["ms_per_step"],
                       speedup_vs_plain=best["speedup_vs_plain"])
    # the same step with its products, masking and decryption replayed from a
    # CUDA graph (inputs encrypted eagerly every step)
    gstep = w.graph_step()
    for _ in range(args.warmup):
        gstep()
    gsec = timed_fn(w, gstep, args.steps, world)
    gval, _ = aggregate(gsec, TOKENS_PER_STEP * args.steps, world)
    graph = {"value": round(gval, 3), "unit": UNIT, "ms_per_step": round(gsec * 1e3 / args.steps, 3),
             "speedup_vs_eager": round(gval / value, 3),
             "form": "encode + encrypt eager per step, then one CUDA graph replay of QKV, W_O, 18 maskings "
                     "(nonces fixed at capture) and P0's decryption"}
    del w.graph, w.graph_out, w.graph_inputs
    conv = conversion_bench(w, 20) if args.conversion else None
    # the BERT-base step is done: keep its figures, free its plans and keys
    # (25 GB) before the larger workloads below
    w_counts, w_cp_bytes = w.counts(), w.cp_bytes()
    for h in (w.plan_qkv, w.plan_o, w.keys):
        h.free()
    torch.cuda.empty_cache()
    def section(run, fn):
        """A further workload's figures; a library error in it (an allocation
        the device cannot hold, say) is reported in its place instead of
        ending the run before the line is printed."""
        if not run or world != 1:
            return None
        try:
            return fn()
        except (blb.BlbError, torch.OutOfMemoryError) as e:
            torch.cuda.empty_cache()
            return {"error": str(e)[:300]}

    bl_batch = section(args.bert_large_seqs, lambda: bert_large_batching(args.bert_large_seqs))
    lnorm = section(args.layernorm, lambda: layernorm_bench(max(2, min(10, args.steps // 5))))
    layer = section(args.layer, layer_bench)
    attn = section(args.attention, lambda: attention_cc(max(1, min(5, args.steps // 4))))
    serving = section(args.serving, serving_bench)
    serving5 = section(args.serving_n65536, serving_n65536_bench)
    if rank != 0:
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    peak_note = "measured" if "hbm_gbs" in peaks else "fallback"
    roof = {}
    for s, (ms, cnt, nbytes) in sites.items():
        if cnt and ms > 0:
            gbs = nbytes / (ms / 1e3) / 1e9
            roof[s] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                       "frac": round(gbs / hbm, 4), "ms_total": round(ms, 3), "launch_sites": cnt,
                       "share_of_step": round(ms / ((dev_s if s == "cp_mac" else prof_s) * 1e3), 4),
                       "measured_in": "the timed region" if s == "cp_mac" else
                                      "a second pass of the same steps with every site bracketed",
                       "algorithmic_bytes_per_call": nbytes // cnt, "peak_kind": peak_note}
    # ALU roofline of the NTT sites: butterflies (rows x N/2 x log2 N; the site
    # records 16 B per coefficient per row, 32 for the gather-fused inverse) per
    # second against the measured register-only butterfly rate of the same
    # instruction mix
    logn = int(np.log2(w.N))
    for s_, word_bytes in (("ntt", 16), ("intt", 16), ("intt_gather", 32)):
        if s_ in roof:
            ms, cnt, nbytes = sites[s_]
            bfly = nbytes / word_bytes * logn / 2
            ach = bfly / (ms / 1e3)
            roof[s_]["alu"] = {"bound": "alu", "achieved": round(ach / 1e9, 2), "peak": round(int_peaks["bfly_per_s"] / 1e9, 2),
                               "unit": "Gbutterfly/s", "frac": round(ach / int_peaks["bfly_per_s"], 4),
                               "peak_kind": "measured (register-only lazy butterfly, libblb_peaks.so)"}
    # ALU roofline of the key-switch site: its counted arithmetic (128-bit
    # multiply-adds, 128-bit reductions, butterflies of its NTTs and Shoup
    # products) at the measured register-only rate of each, summed (they share
    # the integer pipes), is the least time the site could take; frac = that
    # time / the measured time.  The binding roofline is the larger fraction.
    if "keyswitch" in roof and ks_ops[0]:
        ms = sites["keyswitch"][0]
        t_min = (ks_ops[0] / int_peaks["mad128_per_s"] + ks_ops[1] / int_peaks["reduce128_per_s"]
                 + ks_ops[2] / int_peaks["bfly_per_s"])
        alu_frac = t_min / (ms / 1e3)
        roof["keyswitch"]["alu"] = {
            "bound": "alu", "frac": round(alu_frac, 4), "min_ms_total": round(t_min * 1e3, 3),
            "ops_total": {"mad128": ks_ops[0], "reduce128": ks_ops[1], "butterflies": ks_ops[2]},
            "peak_kind": "measured (register-only rates of each unit, libblb_peaks.so)"}
        roof["keyswitch"]["binding"] = "alu" if alu_frac > roof["keyswitch"]["frac"] else "hbm"
    # the dominant single-kernel site (the key-switch site is a pipeline of kernels)
    kernel_sites = [s for s in ("cp_mac", "ntt", "intt") if s in roof]
    dominant = max(kernel_sites, key=lambda s: roof[s]["ms_total"]) if kernel_sites else None
    # DRAM bytes per launch site of the dominant kernel: the measured ratio of
    # DRAM traffic to algorithmic bytes from the committed ncu summary of the
    # same kernel on a smaller matrix, times this workload's algorithmic bytes
    traffic = None
    if dominant == "cp_mac":
        ratio = traffic_ratio(os.path.join(ROOT, "profiles", "ncu_cp_mac_tc_128x768x256_N32768.md"))
        if ratio:
            traffic = int(ratio * roof[dominant]["algorithmic_bytes_per_call"])
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dev_max * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64 (RNS residues; FP64 encode/decode)",
        "data": "synthetic (seeded U[-1,1] BERT-base-shaped operands)", "config": config(world),
        "clocks": clk,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT,
                "h2d_bytes_per_step": int(w.Zhost.numel() * 8),
                "d2h_bytes_per_step": int(w.p0_host.numel() * 8 + w.p1_host.numel() * 8)},
        "gpu_launches": int(launches),
        "roofline": dict(roof[dominant], kernel=dominant, traffic=traffic) if dominant else None,
        "roofline_sites": roof,
        "ntt_autotune": {"split": w.ntt_split, "radix": w.ntt_radix, "us_per_row_direction": ntt_us_json(w.ntt_us)},
        "int_peaks": {k: (round(v / 1e9, 2) if k.endswith("_s") else round(v, 3)) for k, v in int_peaks.items()},
        "accuracy": {"max_abs_err_vs_fp64": max_err, "mse": mse, "bound": 1e-4},
        "batched": batched,
        "graph_step": graph,
        "attention_cc": attn,
        "serving": serving,
        "serving_n65536": serving5,
        "layernorm_head": lnorm,
        "encoder_layer": layer,
        "bert_large_batching": bl_batch,
        "conversion": dict(conv, sites={k: dict(v, frac_of_hbm=round(v["achieved_gbs"] / hbm, 4), peak_kind=peak_note)
                                        for k, v in conv["sites"].items()}) if conv else None,
        "counts_per_step": w_counts,
        "matmul_cp_bytes_per_step": w_cp_bytes,
        "weights": {"plaintext_bytes": w.plan_bytes, "encode_s": round(w.plan_s, 2), "timed": False},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- CPU oracle
class OracleSample:
    """The CPU oracle's own matmul_cp method, phase by phase (orc_cp_baby_steps,
    orc_cp_inner_sum, orc_rotate_sum, orc_rescale: the calls orc_matmul_cp is
    made of), on a bounded sample of the BERT-base step with the weights'
    plaintext diagonals encoded once outside the timed region (as the GPU arm's
    plans are).  One sample times, at level 7 (N = 2^15, 8 primes): the hoisted
    baby steps of input 0 (15 rotations), the inner sum of QKV output block 0's
    giant step 0 over all 6 inputs (96 plaintext products), that block's 7
    giant-step rotations summed with one ModDown and its rescale, one
    encryption, and one masking + decryption.  The step is extrapolated by its
    own counts: QKV = 6 x baby steps + 18 x (8 inner sums + giant sum + rescale);
    W_O at level 6 = 6 x baby steps + 6 x (the same), scaled by its limb count
    (7/8); 6 encryptions; 18 maskings + decryptions.  (The giant sum's inputs
    are 7 copies of the inner sum: its cost does not depend on the values.)"""

    def __init__(self):
        import oracle
        from paper_2508_19525_b300 import workloads as wl
        prm = wl.BERT_CP
        self.o = o = oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum)
        self.scale = prm.scale
        self.sk = o.keygen_secret(0)
        self.k = (o.N // 2) // M
        self.G = G = self.k // B1
        self.baby_rots = [b * M for b in range(1, B1)]
        self.giant_rots = [g * B1 * M for g in range(1, G)]
        self.gal = {o.galois_elt(r): o.keygen_galois(0, self.sk, o.galois_elt(r))
                    for r in self.baby_rots + self.giant_rots}
        X, Wqkv, _ = wl.bert_base_cp(0)
        self.Z = pack_columns(X, M, self.k)
        self.cts = np.stack([o.encrypt(self.sk, o.encode(z, LEVEL, prm.scale), 0, c) for c, z in enumerate(self.Z)])
        self.baby = o.cp_baby_steps(self.cts, M, B1, self.gal)           # all inputs, once
        self.pts = o.cp_encode_diagonals(LEVEL, M, D, Wqkv, D_QKV, B1, [0])[0, 0]  # block 0, giant step 0

    def run(self):
        o = self.o
        t0 = time.perf_counter()
        o.cp_baby_steps(self.cts[:1], M, B1, self.gal)
        t_baby = time.perf_counter() - t0
        t0 = time.perf_counter()
        T = o.cp_inner_sum(self.baby, self.pts)
        t_inner = time.perf_counter() - t0
        t0 = time.perf_counter()
        acc = o.rotate_sum(T, np.stack([T] * (self.G - 1)), self.giant_rots,
                           [self.gal[o.galois_elt(r)] for r in self.giant_rots])
        y = o.rescale(acc)
        t_giant = time.perf_counter() - t0
        t0 = time.perf_counter()
        o.encrypt(self.sk, o.encode(self.Z[0], LEVEL, self.scale), 0, 99)
        t_enc = time.perf_counter() - t0
        t0 = time.perf_counter()
        masked, _ = o.he2mpc(y, 0, 1)
        o.decrypt(self.sk, masked)
        t_mask = time.perf_counter() - t0
        block = self.G * t_inner + t_giant
        est = (6 * t_baby + 18 * block) + (7 / 8) * (6 * t_baby + 6 * block) + 6 * t_enc + 18 * t_mask
        return est, {"baby_steps_one_input_s": round(t_baby, 3), "inner_sum_s": round(t_inner, 3),
                     "giant_sum_and_rescale_s": round(t_giant, 3), "encrypt_s": round(t_enc, 4),
                     "mask_decrypt_s": round(t_mask, 4)}

    @staticmethod
    def describe():
        return ("oracle calls of matmul_cp's phases on the BERT-base step (N=2^15, level 7, plaintexts pre-encoded): "
                "orc_cp_baby_steps (input 0, 15 hoisted rotations), orc_cp_inner_sum (QKV block 0, giant step 0: 96 "
                "plaintext products), orc_rotate_sum (7 giant rotations, one ModDown) + orc_rescale, 1 encryption, "
                "1 he2mpc + decryption; extrapolated as QKV = 6 baby + 18 x (8 inner sums + giant sum), "
                "W_O = 7/8 x (6 baby + 6 x the same), 6 encryptions, 18 maskings")

    def threads(self):
        """OpenMP threads the sample keeps busy: the oracle's limb loops (8 limbs
        at level 7, 11 with the special primes in key switching)."""
        n = os.environ.get("OMP_NUM_THREADS")
        avail = int(n) if n and n.isdigit() else (os.cpu_count() or 1)
        return min(avail, LEVEL + 1)


def cpu_baseline():
    smp = OracleSample()
    est, parts = smp.run()
    return {"value": round(TOKENS_PER_STEP / est, 6), "unit": UNIT, "cores": smp.threads(),
            "host_cores": os.cpu_count(), "kind": "oracle", "sample": smp.describe(),
            "sample_parts_s": parts, "est_s_per_step": round(est, 2)}


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    smp = OracleSample()
    for _ in range(args.warmup):
        smp.run()
    ests = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e, parts = smp.run()
        ests.append(e)
    wall = time.perf_counter() - t0
    est = sum(ests) / len(ests)
    value = TOKENS_PER_STEP / est
    line = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(est * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64 (RNS residues; FP64 encode/decode)",
            "data": "synthetic (seeded U[-1,1] BERT-base-shaped operands)", "config": config(1),
            "impl": "reference",
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": smp.threads(),
                             "host_cores": os.cpu_count(), "kind": "oracle", "sample": smp.describe(),
                             "sample_parts_s": parts},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_wall_s": round(wall, 1)}
    print(json.dumps(line), flush=True)


def ntt_us_json(us):
    """{(radix, split): microseconds} of the NTT autotuner as JSON keys
    "r<radix>/<split>"."""
    return {f"r{r}/{sp}": round(v, 4) for (r, sp), v in sorted(us.items())}


def ncu_case(seqs=1, ntt_split=None, ntt_radix=None, d_out=256):
    """Small profiling case of the same kernels for `ncu --profile-from-start off`:
    N = 2^15, 8 primes, matmul_cp 128x768 @ 768x256 (96 plaintext terms per
    output as in the BERT-base products, 2.2 GB of byte-sliced diagonals, larger
    than L2) for `seqs` sequences; one call bracketed by cudaProfilerStart/Stop
    after a warm-up call."""
    import torch
    from paper_2508_19525_b300 import blb
    from paper_2508_19525_b300 import workloads as wl
    prm = wl.BERT_CP
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, prm.dnum, prm.scale)
    if ntt_split is not None:
        ctx.ntt_set_split(ntt_split)
    if ntt_radix is not None:
        ctx.ntt_set_radix(ntt_radix)
    k = ctx.N // 2 // M
    rots = [b * M for b in range(1, B1)] + [g * B1 * M for g in range(1, k // B1)]
    keys = ctx.keygen(0, rots)
    X, W = wl.cp_operands(M, D, d_out, seed=1)
    plan = ctx.cp_plan(M, D, W, d_out, LEVEL, B1)
    seq = [[ctx.encrypt(keys, ctx.encode(z, LEVEL), 100 * s + i) for i, z in enumerate(pack_columns(X, M, k))]
           for s in range(seqs)]
    run = (lambda: ctx.matmul_cp_plan(keys, plan, seq[0])) if seqs == 1 else \
        (lambda: ctx.matmul_cp_batch(keys, plan, seq))
    run()
    ctx.sync()
    torch.cuda.profiler.start()
    run()
    ctx.sync()
    torch.cuda.profiler.stop()
    print(json.dumps({"ncu_case": f"matmul_cp 128x768 @ 768x{d_out}, N=2^15, level 7, {seqs} sequence(s)",
                      "plan": plan.info()}))


def ncu_step(ntt_split=None, ntt_radix=None):
    """One BERT-base step bracketed by cudaProfilerStart/Stop (after one warm-up
    step), for a launch list with `ncu --profile-from-start off`."""
    import torch
    w = Workload(torch.device("cuda", 0), ntt_split, ntt_radix)
    w.step()
    w.ctx.sync()
    torch.cuda.profiler.start()
    w.step()
    w.ctx.sync()
    torch.cuda.profiler.stop()
    print(json.dumps({"ncu_step": WORKLOAD}))


def ncu_conv(count=18):
    """Profiling case of the conversion kernels: C2M and M2C of `count`
    random share vectors at N = 2^15 (the BERT-base matmul_cp parameters),
    both parties, once."""
    import torch
    from paper_2508_19525_b300 import blb
    from paper_2508_19525_b300 import workloads as wl
    prm = wl.BERT_CP
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, prm.dnum, prm.scale)
    N, s, q = ctx.N, ctx.N // 2, ctx.primes[0]
    g = torch.Generator(device="cuda").manual_seed(1)
    t0 = torch.randint(0, q, (count, N), generator=g, device="cuda", dtype=torch.int64)
    t1 = torch.randint(0, q, (count, N), generator=g, device="cuda", dtype=torch.int64)
    u64 = dict(dtype=torch.int64, device="cuda")
    W0, W1 = torch.zeros((count, N, 2), **u64), torch.zeros((count, N, 2), **u64)
    Y0, Y1 = torch.zeros((count, s), **u64), torch.zeros((count, s), **u64)
    ctx.f2r_wrap_sim(t0, t1, 3, list(range(count)), W0, W1)
    ctx.c2m_local(0, t0, W0, prm.scale, 43, 13, out=Y0)
    ctx.c2m_local(1, t1, W1, prm.scale, 43, 13, out=Y1)
    V0, V1 = torch.zeros((count, s, 2), **u64), torch.zeros((count, s, 2), **u64)
    M = torch.zeros((count, ctx.nQ, N), **u64)
    ctx.ext_wrap_sim(Y0, Y1, s, 43, 3, list(range(count)), V0, V1)
    ctx.m2c_local(0, Y0, V0, s, ctx.nQ - 1, prm.scale, 43, 13, out=M)
    ctx.m2c_local(1, Y1, V1, s, ctx.nQ - 1, prm.scale, 43, 13, out=M)
    ctx.sync()
    print(json.dumps({"ncu_conv": count}))


def ncu_cc(L, kind="pv", params="large", dh=64):
    """Profiling case of matmul_cc: one Q K^T (kind "qk", inner dimension 64) or
    P V ("pv", inner dimension L) product at L tokens; params "large": the
    BERT-large attention shape (16 heads in one group, N = 2^16, 12 primes,
    dnum 4), "base": 8 heads at the BERT-base ct-pt parameters (N = 2^15,
    8 primes, dnum 3), small enough for full ncu captures.  One untimed
    product, then one bracketed by cudaProfilerStart/Stop."""
    import torch
    from paper_2508_19525_b300 import blb
    from paper_2508_19525_b300 import layer as ly
    from paper_2508_19525_b300 import workloads as wl
    prm, heads, dnum = (wl.BERT_CC, 16, 4) if params == "large" else (wl.BERT_CP, 8, wl.BERT_CP.dnum)
    stream = torch.cuda.Stream()
    ctx = blb.Context(prm.logN, prm.q_bits, prm.p_bits, dnum, prm.scale, stream=stream)
    level = ctx.nQ - 1
    plan = ctx.cc_plan(L, heads, dh if kind == "qk" else L, level)
    keys = ctx.keygen(46, plan.rotations(), relin=True)
    Q, K, V, P = wl.attention_operands(L, heads, dh, seed=1)
    if kind == "qk":
        A, B = Q, np.transpose(K, (0, 2, 1))
    else:
        A, B = P, np.concatenate([V, np.zeros((heads, L, L - dh))], axis=2)
    info = plan.info()
    Az = ly.pack_heads(A, L, heads, info["Kc"], info["n_c"], rows=False)
    Bz = ly.pack_heads(B, L, heads, info["Kc"], info["n_c"], rows=True)
    Ac = ctx.encrypt_batch(keys, ctx.encode_batch(Az, level), list(range(info["n_c"])))
    Bc = ctx.encrypt_batch(keys, ctx.encode_batch(Bz, level), [1000 + c for c in range(info["n_c"])])
    C = ctx.matmul_cc_plan(keys, plan, Ac, Bc)
    ctx.sync()
    del C
    l0 = blb.kernel_launches()
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    C = ctx.matmul_cc_plan(keys, plan, Ac, Bc)
    ctx.sync()
    sec = time.perf_counter() - t0
    torch.cuda.profiler.stop()
    print(json.dumps({"ncu_cc": f"{kind} L={L} heads={heads} N={ctx.N}", "s": round(sec, 4),
                      "launches": blb.kernel_launches() - l0, "plan": info}))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["blb", "reference"], default="blb")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", action="store_true", help="run the small profiling case and exit")
    ap.add_argument("--ncu-seqs", type=int, default=1, help="sequences in the profiling case")
    ap.add_argument("--ncu-dout", type=int, default=256, help="output columns of the profiling case (2304: QKV)")
    ap.add_argument("--ncu-step", action="store_true", help="run one profiled BERT-base step and exit")
    ap.add_argument("--ncu-conv", action="store_true", help="run the conversion profiling case and exit")
    ap.add_argument("--ncu-cc", type=int, default=0, metavar="L",
                    help="run one profiled BERT-large matmul_cc product at L tokens and exit")
    ap.add_argument("--ncu-cc-kind", choices=("qk", "pv"), default="pv")
    ap.add_argument("--ncu-cc-params", choices=("large", "base"), default="large")
    ap.add_argument("--ntt-split", type=int, default=None, choices=(-1, 0, 1),
                    help="fix the NTT pass split of the profiling cases (default: autotuned)")
    ap.add_argument("--ntt-radix", type=int, default=None, choices=(8, 16),
                    help="fix the NTT radix of the profiling cases (default: autotuned)")
    ap.add_argument("--batch", type=int, default=8, help="sequences per batched step (1 = skip)")
    ap.add_argument("--no-attention", dest="attention", action="store_false",
                    help="skip the matmul_cc attention measurement")
    ap.add_argument("--bert-large-seqs", type=int, default=32,
                    help="BERT-large uneven-length sequences of the batching measurement (0 = skip; 32 = the full config)")
    ap.add_argument("--no-layer", dest="layer", action="store_false",
                    help="skip the hybrid encoder-layer measurement")
    ap.add_argument("--no-layernorm", dest="layernorm", action="store_false",
                    help="skip the LayerNorm-head (rotate-and-sum) measurement")
    ap.add_argument("--no-conversion", dest="conversion", action="store_false",
                    help="skip the CKKS <-> MPC conversion measurement")
    ap.add_argument("--no-serving-n65536", dest="serving_n65536", action="store_false",
                    help="skip the continuous-batching measurement at N=2^16 (lengths up to 1024, chunked)")
    ap.add_argument("--no-serving", dest="serving", action="store_false",
                    help="skip the continuous-batching serving measurement")
    args = ap.parse_args()
    if args.ncu_case:
        return ncu_case(args.ncu_seqs, args.ntt_split, args.ntt_radix, args.ncu_dout)
    if args.ncu_step:
        return ncu_step(args.ntt_split, args.ntt_radix)
    if args.ncu_conv:
        return ncu_conv()
    if args.ncu_cc:
        return ncu_cc(args.ncu_cc, args.ncu_cc_kind, args.ncu_cc_params)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_blb(args)


if __name__ == "__main__":
    main()
