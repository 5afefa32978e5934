"""Continuous-batching server for encrypted linear-layer requests.

Each request belongs to its own client (its own secret and key set) and asks
for one layer's fused linear products on its encrypted activation: the QKV
product, then the output projection on the first d columns of the result
(matmul_cp, Sec. 4.2.1 / 5.2), then CKKS -> MPC masking of every output
(Alg. 1).  Sequence lengths are padded to a power of two m (the spatial-first
packing needs m | N/2); the server holds one pair of weight plans per
(model, m).

Scheduling.  Requests are admitted in arrival order while the HBM budget
(the client's rotation keys plus its ciphertexts) and the number of requests
in flight allow.  Work advances stage by stage (0: QKV, 1: output projection
and masking); one iteration runs, for the group (model, m, stage) holding the
oldest waiting request, one batched product over up to `max_batch` requests of
that group (`blb_matmul_cp_multi`: the plaintext diagonals stream once for all
of them, every key switch uses its own client's key).  Requests that arrive
while others are in flight are admitted as memory frees up and join the next
iteration of their group, so requests at different stages interleave on the
device.  Every result is bit-identical to the same request served alone.

The scheduler is independent of the GPU: `Server` drives an engine with the
methods `admit`, `run` and `release` (`GpuEngine` and `ChunkEngine` below; the
tests use a fake engine on CPU).  `GpuEngine` packs a whole request into one
product of its padded length; `ChunkEngine` cuts every request into m-row
chunks (one plan pair per model serves every length) and runs a stage of a
batch as cross-client products over groups of chunks.
"""
from dataclasses import dataclass, field
import time

import numpy as np

STAGES = 2  # 0: QKV product; 1: output projection + masking


@dataclass
class Request:
    rid: int
    client_seed: int
    model: str
    seq: int                # true sequence length
    m: int                  # padded length (bucket)
    arrival: float          # seconds after the start of the run
    X: np.ndarray = None    # (seq, d) activation (client side, FP64)
    stage: int = 0
    admitted: float = None
    done: float = None
    state: dict = field(default_factory=dict)

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


def bucket(seq, buckets):
    """Smallest bucket m >= seq."""
    for m in sorted(buckets):
        if seq <= m:
            return m
    raise ValueError(f"sequence length {seq} exceeds the largest bucket {max(buckets)}")


class Server:
    """Admission by memory budget and continuous batching over (model, m, stage) groups."""

    def __init__(self, engine, budget_bytes, max_batch=8, max_inflight=64):
        self.engine = engine
        self.budget = budget_bytes
        self.max_batch = max_batch
        self.max_inflight = max_inflight
        self.used = 0
        self.waiting = []       # arrived, not admitted (FIFO)
        self.inflight = []      # admitted, not done
        self.finished = []
        self.iterations = []    # (group, batch size) per iteration

    def _admit(self, now):
        while self.waiting and len(self.inflight) < self.max_inflight:
            r = self.waiting[0]
            need = self.engine.footprint(r)
            if need > self.budget:
                raise ValueError(f"request {r.rid} needs {need} bytes, more than the whole budget")
            if self.used + need > self.budget:
                break
            self.waiting.pop(0)
            self.used += need
            r.admitted = now
            self.engine.admit(r)
            self.inflight.append(r)

    def _pick(self):
        """The group of the oldest in-flight request and up to max_batch of its members."""
        if not self.inflight:
            return None, []
        oldest = min(self.inflight, key=lambda r: (r.admitted, r.rid))
        key = (oldest.model, oldest.m, oldest.stage)
        members = sorted((r for r in self.inflight if (r.model, r.m, r.stage) == key),
                         key=lambda r: (r.admitted, r.rid))[: self.max_batch]
        return key, members

    def run(self, requests, clock=None):
        """Serve requests (sorted by arrival); clock() returns seconds since the
        start (real time by default).  Returns the finished requests."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        t0 = time.perf_counter()
        clock = clock or (lambda: time.perf_counter() - t0)
        while pending or self.waiting or self.inflight:
            now = clock()
            while pending and pending[0].arrival <= now:
                self.waiting.append(pending.pop(0))
            self._admit(now)
            key, batch = self._pick()
            if not batch:
                # idle until the next arrival
                if pending:
                    self.engine.idle(pending[0].arrival - now)
                continue
            self.engine.run(key, batch)
            self.iterations.append((key, len(batch)))
            now = clock()
            for r in batch:
                r.stage += 1
                if r.stage == STAGES:
                    r.done = now
                    self.inflight.remove(r)
                    self.used -= self.engine.footprint(r)
                    self.engine.release(r)
                    self.finished.append(r)
        return self.finished


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(np.ceil(p / 100.0 * len(xs))) - 1))
    return xs[i]


class GpuEngine:
    """Runs the stages on the CUDA library.  plans[(model, m)] = (plan_qkv,
    plan_o, rotations); every request gets its own key set at admission (the
    client's keys arriving with its request) and freed at completion."""

    def __init__(self, ctx, plans, level, d, d_out_qkv, sync=True, keep_outputs=False):
        self.ctx = ctx
        self.keep_outputs = keep_outputs  # keep keys and unmasked outputs (for checking)
        self.plans = plans
        self.level = level
        self.d = d
        self.d_out_qkv = d_out_qkv
        self.sync = sync
        self.key_bytes = ctx.key_bytes()

    def footprint(self, r):
        """Bytes the request holds while in flight: its rotation keys and its
        input, intermediate and output ciphertexts."""
        qkv, o, rots = self.plans[(r.model, r.m)]
        n = self.level + 1
        ct = lambda lv: 2 * (lv + 1) * self.ctx.N * 8
        i, io = qkv.info(), o.info()
        cts = i["nX"] * ct(self.level) + i["nY"] * ct(self.level - 1) + io["nY"] * ct(self.level - 2)
        return len(rots) * self.key_bytes + cts + 2 * io["nY"] * self.ctx.N * 8

    def admit(self, r):
        ctx = self.ctx
        qkv, o, rots = self.plans[(r.model, r.m)]
        r.state["keys"] = ctx.keygen(r.client_seed, rots)
        k = (ctx.N // 2) // r.m
        Xp = np.zeros((r.m, self.d))
        Xp[: r.seq] = r.X
        nX = qkv.info()["nX"]
        Z = np.zeros((nX, r.m * k))
        for c in range(nX):
            blk = Xp[:, c * k:(c + 1) * k]
            Z[c, :blk.shape[1] * r.m] = blk.T.reshape(-1)
        base = 1_000_000 + 100 * r.rid
        r.state["in"] = ctx.encrypt_batch(r.state["keys"], ctx.encode_batch(Z, self.level),
                                         [base + c for c in range(nX)])

    def run(self, key, batch):
        ctx = self.ctx
        model, m, stage = key
        qkv, o, _ = self.plans[(model, m)]
        keys = [r.state["keys"] for r in batch]
        if stage == 0:
            outs = ctx.matmul_cp_multi(keys, qkv, [r.state["in"] for r in batch])
            nX = qkv.info()["nX"]
            for r, Y in zip(batch, outs):
                r.state["qkv"] = Y
                r.state["o_in"] = Y[:nX]
                del r.state["in"]
        else:
            outs = ctx.matmul_cp_multi(keys, o, [r.state["o_in"] for r in batch])
            for r, O in zip(batch, outs):
                Y = r.state.pop("qkv")[qkv.info()["nX"]:]
                del r.state["o_in"]
                outs_r = Y + O
                if self.keep_outputs:
                    r.state["outs"] = outs_r
                # the two outputs of different levels are masked per level
                masked, shares = [], []
                for lv in sorted({c.level for c in outs_r}):
                    cs = [c for c in outs_r if c.level == lv]
                    base = 2_000_000 + 100 * r.rid + 50 * (lv % 2)
                    mk, sh = ctx.he2mpc_batch(r.state["keys"], cs, [base + j for j in range(len(cs))])
                    masked += mk
                    shares.append(sh)
                r.state["masked"] = masked
                r.state["shares"] = np.concatenate(shares, axis=0)
        if self.sync:
            ctx.sync()

    def release(self, r):
        # the masked outputs and P1's shares stay with the request; keys go
        keys = r.state["keys"] if self.keep_outputs else r.state.pop("keys")
        r.state["p0"] = self.ctx.decrypt_batch(keys, r.state["masked"])[0]
        if not self.keep_outputs:
            keys.free()

    def idle(self, seconds):
        time.sleep(max(0.0, min(seconds, 0.002)))


class ChunkEngine:
    """Token-chunked requests: a request of `seq` tokens is cut into
    ceil(seq / m) chunks of m rows (the last zero-padded), each packed
    spatial-first into ceil(d / k) ciphertexts (k = N / (2 m) columns per
    ciphertext), so one plan pair per model, plans[model] = (plan_qkv, plan_o,
    rotations), serves every sequence length.  A stage of a batch of requests
    runs as `blb_matmul_cp_multi` calls over up to `group` chunks each, every
    chunk key-switched with its own client's keys; chunk c of a request returns
    the limbs of its single product.  The requests' `m` is the chunk size.
    Masking covers, per chunk, the QKV output ciphertexts after the first
    ceil(d / k) and the output projection."""

    def __init__(self, ctx, plans, level, d, d_out_qkv, m, group=4, sync=True, keep_outputs=False):
        self.ctx = ctx
        self.plans = plans
        self.level = level
        self.d = d
        self.d_out_qkv = d_out_qkv
        self.m = m
        self.k = ctx.N // 2 // m
        self.nX = -(-d // self.k)
        self.group = group
        self.sync = sync
        self.keep_outputs = keep_outputs
        self.key_bytes = ctx.key_bytes()

    def chunks(self, r):
        return -(-r.seq // self.m)

    def footprint(self, r):
        qkv, o, rots = self.plans[r.model]
        ct = lambda lv: 2 * (lv + 1) * self.ctx.N * 8
        i, io = qkv.info(), o.info()
        per_chunk = (i["nX"] * ct(self.level) + i["nY"] * ct(self.level - 1) + io["nY"] * ct(self.level - 2)
                     + 2 * (i["nY"] - i["nX"] + io["nY"]) * self.ctx.N * 8)
        return len(rots) * self.key_bytes + self.chunks(r) * per_chunk

    def admit(self, r):
        from .batching import pack_chunks
        ctx = self.ctx
        _, _, rots = self.plans[r.model]
        keys = ctx.keygen(r.client_seed, rots)
        r.state["keys"] = keys
        Z = pack_chunks(r.X, self.m, self.k, self.nX).reshape(-1, self.m * self.k)
        base = 1_000_000 + 10_000 * r.rid
        cts = ctx.encrypt_batch(keys, ctx.encode_batch(Z, self.level), [base + i for i in range(len(Z))])
        r.state["in"] = [cts[c * self.nX:(c + 1) * self.nX] for c in range(self.chunks(r))]

    def run(self, key, batch):
        ctx = self.ctx
        model, _, stage = key
        qkv, o, _ = self.plans[model]
        items = [(r, c) for r in batch for c in range(self.chunks(r))]
        for g0 in range(0, len(items), self.group):
            part = items[g0:g0 + self.group]
            keys = [r.state["keys"] for r, _ in part]
            if stage == 0:
                outs = ctx.matmul_cp_multi(keys, qkv, [r.state["in"][c] for r, c in part])
                for (r, c), Y in zip(part, outs):
                    r.state.setdefault("qkv", {})[c] = Y
            else:
                outs = ctx.matmul_cp_multi(keys, o, [r.state["qkv"][c][:self.nX] for r, c in part])
                for (r, c), O in zip(part, outs):
                    r.state.setdefault("o", {})[c] = O
        for r in batch:
            if stage == 0:
                del r.state["in"]
                continue
            outs_r = []
            for c in range(self.chunks(r)):
                outs_r += r.state["qkv"][c][self.nX:] + r.state["o"][c]
            del r.state["qkv"], r.state["o"]
            if self.keep_outputs:
                r.state["outs"] = outs_r
            masked, shares = [], []
            for lv in sorted({c.level for c in outs_r}):
                cs = [c for c in outs_r if c.level == lv]
                base = 2_000_000 + 10_000 * r.rid + 5_000 * (lv % 2)
                mk, sh = ctx.he2mpc_batch(r.state["keys"], cs, [base + j for j in range(len(cs))])
                masked += mk
                shares.append(sh)
            r.state["masked"] = masked
            r.state["shares"] = np.concatenate(shares, axis=0)
        if self.sync:
            ctx.sync()

    def release(self, r):
        keys = r.state["keys"] if self.keep_outputs else r.state.pop("keys")
        r.state["p0"] = self.ctx.decrypt_batch(keys, r.state["masked"])[0]
        if not self.keep_outputs:
            keys.free()

    def idle(self, seconds):
        time.sleep(max(0.0, min(seconds, 0.002)))
