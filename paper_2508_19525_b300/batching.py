"""Batched ciphertext-plaintext products over many uneven-length sequences of
one client.

matmul_cp (Sec. 4.2.1 / 5.2) multiplies every row (token) of the activation
by the same weight matrix, independently of the other rows, so the tokens of
all sequences of a batch are laid end to end and cut into chunks of m rows:
chunk c holds tokens [c m, (c+1) m) of the concatenation (the last chunk is
zero-padded).  Every chunk is packed spatial-first like one m-row activation
(ciphertext i holds columns [i k, (i+1) k), k = N/(2m), column j of the chunk
at slots [j m, (j+1) m) of its ciphertext), so one plan serves every chunk,
whatever the sequence lengths, and the batched product
(blb_matmul_cp_batch) streams each plaintext diagonal once for a whole group
of chunks.

Attention (matmul_cc) mixes the rows of one sequence, so its products cannot
be chunked; but the heads of one head group are independent products that
multi-head packing (Sec. 5.1) places side by side in one ciphertext, and the
heads of several sequences of one client with the same padded length are
independent in the same way.  `cc_pack_groups` packs S such sequences into one
product as S x heads heads of one group: the rotations of step 3 and the
relinearizations (L of each per product) are then shared by the S sequences,
and steps 1-2 need fewer rotations per sequence (Kc = s/(L S heads) shrinks,
the input ciphertexts per operand grow by S), while the step-2 tensor products
per sequence stay the same.

The rows per ciphertext m (a power of two; 32 to 256 at N = 2^16 for the
1024-feature products) set how many tokens share one ciphertext's rotations:
the rotations per token fall about as 1/m (`cp_rotation_count`) while the
plan's plaintexts grow as m.  The split of each product's rotations into baby
and giant steps (b1, G with b1 G = k) and the number of chunks per batched
call are chosen by `autotune`:
every b1 candidate is encoded and every (b1, group) pair timed on the product
itself, the fastest kept.  The group size matters because the plaintext MAC
reads each plaintext once per call but its epilogue work grows with the number
of chunks per call: for products with few terms per output a large group
turns the MAC from memory-bound into compute-bound.
"""
import time

import numpy as np


def chunk_layout(lengths, m):
    """Token t of sequence s -> (chunk, row).  Returns (starts, n_chunks):
    starts[s] is the global index of the sequence's first token."""
    starts = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    total = int(np.sum(lengths))
    return starts, -(-total // m)


def pack_chunks(X, m, k, n_cts):
    """X: (T, d) tokens -> (n_chunks, n_cts, m k) slot vectors."""
    T, d = X.shape
    n_chunks = -(-T // m)
    Z = np.zeros((n_chunks, n_cts, m * k))
    Xp = np.zeros((n_chunks * m, n_cts * k))
    Xp[:T, :d] = X
    for c in range(n_chunks):
        blk = Xp[c * m:(c + 1) * m]                  # m x (n_cts k)
        for i in range(n_cts):
            Z[c, i] = blk[:, i * k:(i + 1) * k].T.reshape(-1)
    return Z


def unpack_chunk(slots, m, k, d_out):
    """slots: (n_out_cts, m k) of one chunk -> (m, d_out)."""
    cols = [z.reshape(k, m).T for z in slots]
    return np.concatenate(cols, axis=1)[:, :d_out]


def cp_rotations(m, k, b1):
    """Rotations of one plan: baby steps b m (b < b1), giant steps g b1 m."""
    G = k // b1
    return [b * m for b in range(1, b1)] + [g * b1 * m for g in range(1, G)]


def cp_rotation_count(m, d, d_out, slots, b1):
    """Rotations of one m-row product on ciphertexts of k = slots/m columns:
    b1 - 1 hoisted baby steps per input ciphertext and G - 1 giant steps per
    output ciphertext (b1 G = k).  Per token it falls as m grows: a ciphertext
    of more rows carries more tokens through the same rotations."""
    k = slots // m
    nX, nY = -(-d // k), -(-d_out // k)
    return nX * (b1 - 1) + nY * (k // b1 - 1)


def cp_b1_candidates(m, d, d_out, slots, n=2):
    """Baby-step counts b1 (powers of two below k) to time: the n with the
    fewest rotations by cp_rotation_count and the next larger power of two
    (baby steps are hoisted, so they cost less than giant steps and the
    fastest b1 tends to lie above the count's optimum), ascending."""
    k = slots // m
    cands = [1 << i for i in range(1, k.bit_length()) if (1 << i) < k]
    ranked = sorted(cands, key=lambda b1: (cp_rotation_count(m, d, d_out, slots, b1), b1))
    pick = set(ranked[:n])
    if 2 * max(pick) < k:
        pick.add(2 * max(pick))
    return sorted(pick)


def run_batched(ctx, keys, plan, chunks, group):
    """chunks: list of per-chunk input ciphertext lists.  Runs the product in
    groups of `group` chunks; returns the per-chunk output lists."""
    out = []
    for g0 in range(0, len(chunks), group):
        part = chunks[g0:g0 + group]
        out += ctx.matmul_cp_batch(keys, plan, part) if len(part) > 1 else [ctx.matmul_cp_plan(keys, plan, part[0])]
    return out


def autotune(ctx, keys, m, d, W, d_out, level, chunks, b1_candidates, group_candidates, reps=1):
    """Encode the plan for every baby-step count b1 (powers of two dividing
    k = N/(2m)) and time the product on `chunks` for every group size (chunks
    per call; 1 is the plain product); return ((b1, group), {(b1, group):
    seconds per chunk})."""
    from .blb import BlbError
    timings = {}
    for b1 in b1_candidates:
        try:
            plan = ctx.cp_plan(m, d, W, d_out, level, b1)
        except BlbError:
            continue                                             # shape the library refuses
        for group in group_candidates:
            g = min(group, len(chunks))
            try:
                run_batched(ctx, keys, plan, chunks[:g], g)      # warm-up
            except BlbError:
                break
            ctx.sync()
            t0 = time.perf_counter()
            for _ in range(reps):
                run_batched(ctx, keys, plan, chunks[:g], g)
            ctx.sync()
            timings[(b1, group)] = (time.perf_counter() - t0) / (reps * g)
        plan.free()
    if not timings:
        raise ValueError("no candidate (b1, group) runs on this product")
    best = min(timings, key=timings.get)
    return best, timings


def autotune_dnum(make_ctx, candidates, m, reps=3, rotations=8):
    """Key-switch digit count: for every dnum in `candidates` build a context
    (make_ctx(dnum)), keys for `rotations` rotations by multiples of m slots,
    and time rotations of one ciphertext at the top level (each one a full
    key switch: decomposition, ModUp, inner product, ModDown).  Returns (best dnum, {dnum:
    seconds per rotation}).  Candidates the library refuses (more primes per
    digit than special primes) are skipped."""
    from .blb import BlbError
    timings = {}
    for dnum in candidates:
        try:
            ctx = make_ctx(dnum)
        except BlbError:
            continue
        rots = [b * m for b in range(1, rotations + 1)]
        keys = ctx.keygen(7, rots)
        level = ctx.nQ - 1
        ct = ctx.encrypt(keys, ctx.encode(np.ones(ctx.N // 2) * 0.5, level), 1)
        for r in rots:                                    # warm-up
            ctx.rotate(keys, ct, r)
        ctx.sync()
        t0 = time.perf_counter()
        for _ in range(reps):
            for r in rots:
                ctx.rotate(keys, ct, r)
        ctx.sync()
        timings[dnum] = (time.perf_counter() - t0) / (reps * len(rots))
        del keys, ct
        ctx.free()
    best = min(timings, key=timings.get)
    return best, timings


def cc_pack_groups(pads, heads, slots, max_pack=None):
    """Group the sequences (padded lengths `pads`) of one client into matmul_cc
    products of S sequences each: S a power of two, all of one padded length
    L, with L x S x heads dividing `slots` (Kc >= 1; `heads` a power of two).
    Greedy per length: the largest S (at most `max_pack`) that the remaining
    sequences fill.  Returns [(L, [sequence indices])] covering every sequence
    once, in order of L."""
    if heads & (heads - 1):
        raise ValueError("heads must be a power of two to pack several sequences into one head group")
    by_len = {}
    for i, Lp in enumerate(pads):
        by_len.setdefault(int(Lp), []).append(i)
    groups = []
    for Lp in sorted(by_len):
        idx = by_len[Lp]
        smax = max(1, slots // (Lp * heads))
        if max_pack:
            smax = min(smax, max_pack)
        while idx:
            S = 1
            while 2 * S <= min(smax, len(idx)):
                S *= 2
            groups.append((Lp, idx[:S]))
            idx = idx[S:]
    return groups


def stack_heads(mats):
    """Per-sequence head stacks (heads, rows, cols) -> one stack of S x heads
    heads, sequence j's head h at index j heads + h."""
    return np.concatenate(mats, axis=0)


def split_heads(stack, S):
    """Inverse of stack_heads for S sequences."""
    return np.split(stack, S, axis=0)
