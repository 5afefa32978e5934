/*
 * blb.h -- C ABI of the B300 RNS-CKKS linear path of BLB ("Breaking the Layer
 * Barrier", arXiv 2508.19525): ciphertext x plaintext matrix products
 * (matmul_cp, Sec. 4.2.1 / 5.2 with the baby-step giant-step split of App. C.1),
 * the CKKS primitives they are built on (Sec. 2.4, Eq. 2) and the secure
 * CKKS-to-MPC masking step (Alg. 1, Sec. 6.3).  Both parties of the protocol
 * run in one process: "sending" a ciphertext is handing over a handle.
 *
 * Conventions
 *  - Every entry point returns 0 (BLB_OK) or a negative BLB_ERR_* code and never
 *    throws; blb_last_error() gives a message for the calling thread.
 *  - Objects (context, keys, plaintexts, ciphertexts, cp plans) are opaque,
 *    library-owned and device-resident; free them with the matching *_free.
 *    Their device memory comes from the allocator installed with
 *    blb_set_allocator (default: cudaMalloc / cudaFree).
 *  - All device work of a context runs in order on the CUDA stream given to
 *    blb_ctx_create (NULL = the legacy default stream).  Calls that return data
 *    into host memory synchronize that stream before returning.
 *  - Pointers marked "host or device" are classified with
 *    cudaPointerGetAttributes; unregistered pointers are treated as host memory.
 *  - Polynomials are stored limb-major: limb i holds N residues mod q_i in the
 *    evaluation (NTT) domain.  Exports in coefficient form give the canonical
 *    representation: residues in [0, q_i), limb-major, (level+1) x N words per
 *    polynomial, polynomial-major for ciphertexts.
 *  - Levels: a ciphertext at level l has the l+1 primes q_0..q_l.  Rescaling
 *    drops q_l.
 */
#ifndef BLB_H
#define BLB_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BLB_OK = 0,
    BLB_ERR_ARG = -1,     /* invalid argument: null pointer, size, shape, range */
    BLB_ERR_LEVEL = -2,   /* no level left (rescale at level 0, product needs one) */
    BLB_ERR_SCALE = -3,   /* operands carry different scales */
    BLB_ERR_NO_KEY = -4,  /* the rotation / relinearization key is missing */
    BLB_ERR_OOM = -5,     /* allocation failed */
    BLB_ERR_CUDA = -6,    /* a CUDA runtime call failed (message has the details) */
    BLB_ERR_TIMEOUT = -7, /* a bounded device wait expired */
    BLB_ERR_PARAM = -8    /* parameter set rejected (no prime of a requested size) */
};

typedef struct blb_ctx blb_ctx;
typedef struct blb_keys blb_keys;
typedef struct blb_pt blb_pt;
typedef struct blb_ct blb_ct;
typedef struct blb_cp_plan blb_cp_plan;
typedef struct blb_cc_plan blb_cc_plan;

/* Parameter set.  q_bits[0..nQ) are the bit sizes of the ciphertext primes,
 * p_bits[0..nP) those of the special primes of hybrid key switching; dnum is
 * the number of key-switching digits (alpha = ceil(nQ/dnum) primes each; nP must
 * be >= alpha).  Prime rule: for each size b, in the order q_0, q_1, ..., p_0,
 * ..., the largest prime below 2^b that is 1 mod 2N and not already taken.
 * scale is the default encoding scale Delta (informational). */
typedef struct {
    uint32_t logN;
    uint32_t nQ, nP;
    const uint32_t* q_bits;
    const uint32_t* p_bits;
    uint32_t dnum;
    double scale;
} blb_params;

/* Baby-step giant-step split for matmul_cp: b1 baby steps, G = k/b1 giant
 * steps (k = N/2/m columns per ciphertext); b1 must divide k.  b1 = 0 picks
 * the power of two nearest sqrt(k) (rounded up). */
typedef struct {
    uint32_t b1;
} blb_sched;

/* ---- library ---------------------------------------------------------------
 * Allocator used for all device memory of objects created afterwards.
 * alloc(bytes, stream, user) returns a device pointer or NULL; free(ptr, bytes,
 * stream, user).  Pass NULLs to restore cudaMalloc / cudaFree. */
typedef void* (*blb_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*blb_free_fn)(void* ptr, size_t bytes, void* stream, void* user);
int blb_set_allocator(blb_alloc_fn alloc, blb_free_fn free_fn, void* user);
const char* blb_last_error(void);
const char* blb_version(void);

/* Host-only: the primes a parameter set selects (no GPU needed).
 * out receives nQ + nP words (q_0..q_{nQ-1}, p_0..p_{nP-1}). */
int blb_params_primes(const blb_params* params, uint64_t* out);

/* ---- context ----------------------------------------------------------------
 * Builds primes, NTT / base-conversion / encoding tables on the device.
 * stream: a cudaStream_t (NULL = default stream). */
int blb_ctx_create(const blb_params* params, void* stream, blb_ctx** out);
void blb_ctx_free(blb_ctx* ctx);
int blb_ctx_info(const blb_ctx* ctx, uint32_t* logN, uint32_t* nQ, uint32_t* nP, uint32_t* dnum);
int blb_ctx_primes(const blb_ctx* ctx, uint64_t* out /* host, nQ + nP words */);
int blb_ctx_sync(blb_ctx* ctx);
/* Device memory currently held by this context and its objects (bytes). */
uint64_t blb_ctx_bytes_in_use(const blb_ctx* ctx);
/* Bounded device waits (failure detection; no counterpart in the paper, whose
 * protocols assume kernels that finish).  The plaintext-product pipeline of
 * matmul_cp (copy ring, fragment builder, tensor-core consumers) waits on
 * shared-memory barriers; each wait gives up after limit_ns nanoseconds
 * (0 = the default, 2 s), ends its thread block early, and makes the next
 * blb_ctx_sync return BLB_ERR_TIMEOUT (and clear the condition).  The outputs
 * of the calls since the previous sync are then invalid; the context stays
 * usable.  Copies already in flight are always waited for (up to 2 s) before a
 * block exits, whatever the limit.  Applies to calls made after it. */
int blb_ctx_set_wait_limit(blb_ctx* ctx, uint64_t limit_ns);
/* Deferred encoding checks.  By default an encoding (blb_encode,
 * blb_encode_batch, and the plaintext encodings inside other calls) waits for
 * its kernels and returns BLB_ERR_ARG when a coefficient exceeds 2^63 (value x
 * scale too large).  With on != 0 encodings do not wait: the overflow
 * condition of every encoding accumulates on the device, and the next
 * blb_ctx_sync returns BLB_ERR_ARG (and clears it) if any overflowed; the
 * outputs of the calls since the previous sync are then invalid.  This keeps
 * the host from stalling on the device once per encoding.  on = 0 restores
 * the default for later calls. */
int blb_ctx_set_deferred_encode_check(blb_ctx* ctx, int on);
/* Test hook for that error path: with withhold != 0 the pipeline's copy
 * stage issues no copies, so the consumers' waits run out (after the limit
 * above) instead of completing.  Products computed meanwhile are invalid.
 * 0 restores normal operation. */
int blb_ctx_test_withhold_copies(blb_ctx* ctx, int withhold);
/* Kernel of the plaintext products of batched matmul_cp calls (2, 4 or 8
 * sequences per launch; single sequences always use the mma.sync kernel):
 * 0 = automatic (tcgen05 for 8 sequences of a plan with one 16-output block,
 * where it measured faster; mma.sync otherwise), 1 = the
 * mma.sync kernel, 2 = the tcgen05 kernel (tensor-memory accumulators) where
 * its operands fit shared memory.  Both give the same limbs. */
int blb_ctx_set_batch_mac(blb_ctx* ctx, int kind);

/* ---- keys (Sec. 2.4: rotations and products need switching keys) -----------
 * Secret key s (ternary) and switching keys drawn from Philox4x32-10 with key
 * `seed`: relinearization key (s^2 -> s) if relin != 0, and one Galois key per
 * left-rotation amount rot_steps[i] (negative = right rotation).  Each key has
 * dnum digits over all nQ + nP primes. */
int blb_keygen(blb_ctx* ctx, uint64_t seed, const int32_t* rot_steps, uint32_t n_rot, int relin,
               blb_keys** out);
void blb_keys_free(blb_keys* keys);
/* Export in coefficient form to host memory.  which = 0: secret key, N signed
 * words (int64).  which = 1: relinearization key; which = 2: Galois key for
 * left rotation `rot`; both as dnum x 2 x (nQ+nP) x N words (b then a). */
int blb_keys_export(blb_ctx* ctx, const blb_keys* keys, int which, int32_t rot, void* host_out);

/* ---- encode / decode (Sec. 6.1, Eq. 2) -------------------------------------
 * Encode n <= N/2 real slot values (host or device doubles; missing slots are
 * 0) at `level` with `scale`: round(scale * pi^-1(z)) (round half to even),
 * reduced mod q_0..q_level, stored in the NTT domain. */
int blb_encode(blb_ctx* ctx, const double* vals, uint64_t n, uint32_t level, double scale,
               blb_pt** out);
void blb_pt_free(blb_pt* pt);
/* Plaintext in coefficient form to host: (level+1) x N words. */
int blb_pt_export(blb_ctx* ctx, const blb_pt* pt, uint64_t* host_out);

/* ---- ciphertexts -------------------------------------------------------------
 * Secret-key encryption (-a s + m + e, a); `nonce` selects the Philox stream of
 * a and e (key = the keygen seed).  Only the low 32 bits of nonce are used. */
int blb_encrypt(blb_ctx* ctx, const blb_keys* keys, const blb_pt* pt, uint64_t nonce, blb_ct** out);
void blb_ct_free(blb_ct* ct);
int blb_ct_info(const blb_ct* ct, uint32_t* level, uint32_t* npolys, double* scale);
/* Export in coefficient form: npolys x (level+1) x N words into host or device
 * memory. */
int blb_ct_export(blb_ctx* ctx, const blb_ct* ct, uint64_t* out);
/* Import a ciphertext given in coefficient form (host or device words,
 * npolys x (level+1) x N, residues in [0, q_i)). */
int blb_ct_import(blb_ctx* ctx, const uint64_t* coeffs, uint32_t level, uint32_t npolys,
                  double scale, blb_ct** out);
/* Overwrite dst's limbs (and scale) with src's, in the context's stream order
 * (both of one level and size).  Useful to feed new inputs to ciphertexts a
 * captured CUDA graph reads. */
int blb_ct_copy(blb_ctx* ctx, blb_ct* dst, const blb_ct* src);
/* Decrypt (m = c0 + c1 s [+ c2 s^2]).  coeff_limbs (nullable, host or device):
 * (level+1) x N words, coefficient form.  slots (nullable, host or device):
 * N/2 doubles, the decoding of the q_0 limb lifted to (-q_0/2, q_0/2] and divided
 * by the ciphertext's scale (exact while |message| < q_0/2). */
int blb_decrypt(blb_ctx* ctx, const blb_keys* keys, const blb_ct* ct, uint64_t* coeff_limbs,
                double* slots);

/* ---- homomorphic operations (Sec. 2.4) ------------------------------------- */
/* Rot_l^steps (left by steps slots; negative = right) with hybrid key switching. */
int blb_rotate(blb_ctx* ctx, const blb_keys* keys, const blb_ct* in, int32_t steps, blb_ct** out);
/* Divide by the last prime with rounding; drops one level, scale /= q_l. */
int blb_rescale(blb_ctx* ctx, blb_ct* inout);
int blb_add(blb_ctx* ctx, const blb_ct* a, const blb_ct* b, blb_ct** out);
int blb_mul_plain(blb_ctx* ctx, const blb_ct* a, const blb_pt* b, blb_ct** out);
/* a - b (one level, size and scale). */
int blb_sub(blb_ctx* ctx, const blb_ct* a, const blb_ct* b, blb_ct** out);
/* The same message at a lower level: the limbs past `level` are dropped
 * (modulus switching without scaling; the scale is kept). */
int blb_drop_level(blb_ctx* ctx, const blb_ct* a, uint32_t level, blb_ct** out);
/* a times the slot vector vals (n values: n = 1 broadcasts the one value to
 * every slot, otherwise slots past n are 0), then rescaled: the constant is
 * encoded at scale target_scale q_level / scale(a), so the result (one level
 * down) has scale target_scale; this aligns the scales of terms that went
 * through different numbers of rescales before they are added (the
 * ewmul_cp / smul_cp operators of Sec. 4.1 with a chosen output scale). */
int blb_mul_const(blb_ctx* ctx, const blb_ct* a, const double* vals, uint64_t n, double target_scale,
                  blb_ct** out);
/* ct x ct: tensor product (3 polynomials) followed by relinearization when
 * relin != 0 (needs the relinearization key). */
int blb_mul(blb_ctx* ctx, const blb_keys* keys, const blb_ct* a, const blb_ct* b, int relin,
            blb_ct** out);
int blb_relinearize(blb_ctx* ctx, const blb_keys* keys, const blb_ct* in, blb_ct** out);
/* Key switching of one polynomial d (coefficient form, host or device, (level+1)
 * x N words) with the Galois key of rotation `rot`: writes (k0, k1) in
 * coefficient form, 2 x (level+1) x N words, to out (host or device).
 * Exposed for parity testing of the key-switch pipeline. */
int blb_keyswitch_coeffs(blb_ctx* ctx, const blb_keys* keys, int32_t rot, const uint64_t* d,
                         uint32_t level, uint64_t* out);

/* Allocation-free form of blb_keyswitch_coeffs (same arguments, same result).
 * The paper has no counterpart: this exists for callers that may not
 * allocate device memory while they run, such as a serving process whose
 * memory manager reserved the whole device budget up front, a latency-critical
 * loop that cannot afford cudaMalloc's device-wide synchronization, or code
 * running inside the allocator callbacks of blb_set_allocator.  All temporaries
 * live in one fixed 32 MiB device array compiled into the library: every GPU
 * that loads the library holds it until the process exits.  The call needs
 * (3(l+1) + (l+1) + beta (l+1+nP) + 2 (l+1+nP) + 2 (l+1)) N words, beta =
 * ceil((l+1)/alpha), and returns BLB_ERR_ARG when that exceeds 32 MiB (for
 * example N = 2^16 with 12 primes); N = 2^15 with 8 primes and 3 special primes
 * fits at every level.  blb_ctx_create, with the context's device current,
 * looks up the array's device address (loading the array with the library's
 * module, under lazy module loading too) and loads this call's kernels, so the
 * call itself neither allocates nor loads anything.  All calls on a GPU share the array and it keeps the previous
 * call's contents (nothing in it needs to start at zero): calls that can
 * overlap on the GPU -- other streams, other contexts, other threads -- race
 * and must be serialized by the caller.  d and out may be host or device
 * memory; with host memory the call synchronizes the context's stream. */
int blb_keyswitch_noalloc(blb_ctx* ctx, const blb_keys* keys, int32_t rot, const uint64_t* d,
                          uint32_t level, uint64_t* out);

/* ---- matmul_cp: encrypted X (m x d) times plaintext W (d x d_out) ------------
 * Spatial-first packing (Sec. 4.2.1): with k = N/2/m, input ciphertext c holds
 * X[i][c k + b] at slot i + m b (nX = ceil(d/k) ciphertexts); output e holds
 * Y[i][e k + b] likewise (nY = ceil(d_out/k)).  Diagonal method with
 * baby-step giant-step (App. C.1): nX(b1-1) + nY(G-1) rotations,
 * nX nY k plaintext products, one rescale per output.  The output is at
 * level-1 with the input's scale (plaintexts are encoded with scale q_level).
 * Needs Galois keys for left rotations b m (0 < b < b1) and g b1 m (0 < g < G).
 *
 * blb_cp_plan_create encodes all plaintext diagonals of W (host or device,
 * row-major d x d_out doubles) once, for inputs at `level`; plans are reused
 * across calls (model weights).  blb_matmul_cp_plan runs the product for nX
 * input ciphertexts and writes nY new handles into Y.  blb_matmul_cp is the
 * one-shot form (plan, run, free). */
int blb_cp_plan_create(blb_ctx* ctx, uint32_t m, uint32_t d, const double* W, uint32_t d_out,
                       uint32_t level, const blb_sched* sched, blb_cp_plan** out);
void blb_cp_plan_free(blb_cp_plan* plan);
int blb_cp_plan_info(const blb_cp_plan* plan, uint32_t* nX, uint32_t* nY, uint32_t* b1,
                     uint32_t* G, uint64_t* plaintext_bytes);
/* Plan of the diagonal-input product (App. C.2): E = Concat_h(Att_h) W for
 * Att_h (L x Dh, L = 2 Dh) in matmul_cc's multi-head diagonal packing.  The
 * input, per head group g (Hg[g] heads, Kc = N/2/(L Hg[g])), is the Dh/Kc
 * dense-diagonal ciphertexts of matmul_cc's output with V_h padded to L
 * columns: outputs j and j + Dh/Kc added (blb_add), so that block h + Hg kappa
 * of ciphertext j holds Att_h[i][(i + delta) mod Dh], delta = j Kc + kappa.  W
 * is (sum Hg) Dh x d_out, row-major (host or device).  The product runs with
 * blb_matmul_cp_plan on the groups' ciphertexts in order; E comes back
 * spatial-first (L rows, N/2/L columns per ciphertext) at level - 1. */
int blb_cp_plan_create_diag(blb_ctx* ctx, uint32_t L, uint32_t n_groups, const uint32_t* Hg, uint32_t Dh,
                            const double* W, uint32_t d_out, uint32_t level, const blb_sched* sched,
                            blb_cp_plan** out);
int blb_matmul_cp_plan(blb_ctx* ctx, const blb_keys* keys, const blb_cp_plan* plan,
                       blb_ct* const* X, uint32_t nX, blb_ct** Y);
/* Batched form: n_seq sequences (same m and d, e.g. the sequences of one
 * client's batch) through one plan.  X: n_seq x nX handles, sequence-major;
 * Y: n_seq x nY.  Every plaintext word is read from HBM once per batch and
 * applied to all sequences; results equal n_seq calls of blb_matmul_cp_plan. */
int blb_matmul_cp_batch(blb_ctx* ctx, const blb_keys* keys, const blb_cp_plan* plan,
                        blb_ct* const* X, uint32_t n_seq, blb_ct** Y);
/* The same product for sequences of different clients: keys[s] is the key set
 * of sequence s (Galois keys for the plan's rotations, same context).  The
 * plaintext diagonals are shared, so they stream from HBM once for the whole
 * batch; each key switch uses its own client's key.  Member s's outputs are
 * bit-identical to blb_matmul_cp_plan with keys[s]. */
int blb_matmul_cp_multi(blb_ctx* ctx, const blb_keys* const* keys, const blb_cp_plan* plan, blb_ct* const* X,
                        uint32_t n_seq, blb_ct** Y /* n_seq x nY handles */);
int blb_matmul_cp(blb_ctx* ctx, const blb_keys* keys, blb_ct* const* X, uint32_t nX, uint32_t m,
                  uint32_t d, const double* W, uint32_t d_out, const blb_sched* sched, blb_ct** Y);

/* ---- matmul_cc: encrypted A_h (L x R) times encrypted B_h (R x L), Hg heads ----
 * Sec. 5.1 (three steps, multi-head packing) with the baby-step giant-step split
 * of App. C.1.  Packing: N/2 slots in blocks of L; block h + Hg kappa of input
 * ciphertext c holds column k = c Kc + kappa of A_h (spatial-first) or row k of
 * B_h (reduce-first), element i at slot (h + Hg kappa) L + i, Kc = N/2/(L Hg)
 * (Kc <= L, n_c = ceil(R/Kc) ciphertexts per operand).  Output ciphertext j of
 * L/Kc holds diagonal delta = j Kc + kappa of C_h at block h + Hg kappa:
 * element i = C_h[i][(i + delta) mod L] (diagonal packing).
 * Schedule (both sides of the parity tests implement the same):
 *   1. pre-rotate row k of block kappa of B by kappa (masks, BSGS split b1s1 | Kc);
 *   2. for t = g b1s2 + b: V = masks x {Rot^b, Rot^{b-L}}(B'), tensor with
 *      Rot^{-g b1s2}(A), sum over input ciphertexts, relinearize, rescale;
 *   3. one rotation Rot^{g b1s2 - (t mod Kc) Hg L} per t, two routing masks.
 * Depth 4: inputs at `level` (>= 4), outputs at level-4 with scale
 * scale(A) scale(B) / q_{level-2}.  Needs the relinearization key and the Galois
 * keys of blb_cc_plan_rotations.  Masks are encoded once per plan: the 2 Kc
 * step-1 and 2 L step-2 masks, and the distinct step-3 masks (at most 2 Kc: a
 * step-3 mask is constant on each block and splits the blocks at kappa = t mod Kc).
 * Steps 1-2 run over chunks of c_chunk input ciphertexts and, inside, t_chunk
 * diagonals, their tensor products summed mod q (the result does not depend on
 * the chunking); by default the chunks are the largest whose workspace stays
 * within workspace_bytes (0 = 24 GiB), the whole product when it fits. */
typedef struct {
    uint32_t b1s1, b1s2;      /* 0 = about sqrt(Kc/2), sqrt(L/2) */
    uint32_t c_chunk, t_chunk; /* 0 = from the workspace budget */
    uint64_t workspace_bytes;  /* 0 = 24 GiB */
} blb_cc_sched;
int blb_cc_plan_create(blb_ctx* ctx, uint32_t L, uint32_t Hg, uint32_t R, uint32_t level,
                       const blb_cc_sched* sched, blb_cc_plan** out);
void blb_cc_plan_free(blb_cc_plan* plan);
int blb_cc_plan_info(const blb_cc_plan* plan, uint32_t* n_c, uint32_t* Kc, uint32_t* nout, uint32_t* b1s1,
                     uint32_t* b1s2, uint64_t* mask_bytes, uint32_t* c_chunk, uint32_t* t_chunk);
/* Left-rotation amounts the plan needs keys for; out may be NULL to query count. */
int blb_cc_plan_rotations(const blb_cc_plan* plan, int32_t* out, uint32_t cap, uint32_t* count);
int blb_matmul_cc_plan(blb_ctx* ctx, const blb_keys* keys, const blb_cc_plan* plan, blb_ct* const* A,
                       blb_ct* const* B, uint32_t n_in, blb_ct** C /* L/Kc handles */);
int blb_matmul_cc(blb_ctx* ctx, const blb_keys* keys, blb_ct* const* A, blb_ct* const* B, uint32_t n_in,
                  uint32_t L, uint32_t R, uint32_t Hg, const blb_cc_sched* sched, blb_ct** C);

/* ---- CKKS -> MPC (Alg. 1 steps 1-2, Sec. 6.3) --------------------------------
 * P1 reduces the ciphertext to level 0, adds a mask r drawn uniformly from
 * Z_{q_0}[X]/(X^N+1) (Philox stream `nonce`, key = the keygen seed) and keeps
 * -r mod q_0 as its share: p1_share (host or device) receives N words in
 * coefficient form.  masked_for_p0 receives a new level-0 ciphertext; P0's share
 * is its decryption (blb_decrypt, coeff_limbs).  The two shares sum to the
 * message plus noise mod q_0. */
int blb_he2mpc(blb_ctx* ctx, const blb_keys* keys, const blb_ct* ct, uint64_t nonce,
               blb_ct** masked_for_p0, uint64_t* p1_share);

/* ---- rotate-and-sum packing (Sec. 4.2.1) -------------------------------------
 * Spatial-first packing puts block b (L consecutive slots) of a ciphertext at
 * slots [b L, (b+1) L).  For each of the count input ciphertexts (one level,
 * two polynomials): m^0 = m, m^i = m^{i-1} + Rot^{2^{i-1} L}(m^{i-1}) for
 * i = 1..log2 D, with left rotations (dir = 0: sum) or right rotations
 * (dir = 1: broadcast).  Block b then holds the sum of blocks b .. b+D-1
 * (left) or b-D+1 .. b (right), indices mod N/(2L).  mask != 0 (sum only)
 * multiplies by the plaintext [1 (L slots), 0, ...] encoded at scale q_level and
 * rescales: only block 0 remains, one level lower.  D must be a power of two
 * with L D <= N/2; the keys must hold the rotations +-2^i L.  out[k] receives
 * new ciphertexts (all NULL on error).  Errors: BLB_ERR_ARG, BLB_ERR_NO_KEY,
 * BLB_ERR_OOM, BLB_ERR_CUDA. */
int blb_rotate_sum_packing(blb_ctx* ctx, const blb_keys* keys, blb_ct* const* in, uint32_t count, uint32_t L,
                           uint32_t D, int dir, int mask, blb_ct** out);
/* The HE steps of the secure LayerNorm before rsqrt (Alg. LayerNorm lines 1-6)
 * for count sequences, each L rows x D columns packed spatial-first in nc
 * ciphertexts X[j nc + c] of k = N/(2L) columns (k a power of two) at one
 * level >= 3:
 *   X_sum = the nc ciphertexts added, then rotate-and-sum over the k blocks
 *           without mask (the sum feeds a scalar operator, so every block
 *           keeping the row sums is the broadcast, Sec. 4.2.1);
 *   mu    = X_sum times the plaintext 1/D (scale q_level), rescaled;
 *   X_mu[j nc + c] = X[j nc + c] one level down, minus mu;
 *   X_mu^2: tensor product, relinearization, rescale;
 *   var[j] = the rotate-and-sum of the nc squares, times 1/D, rescaled
 *            (level - 3, scale scale^2 / q_{level-1}, every block holding the
 *            row variances).
 * Needs the relinearization key and the rotations 2^i L, i < log2 k.  With
 * zero-padded columns (D < nc k) each padded column adds mu^2 to the sum of
 * squares.  Outputs are new ciphertexts (all NULL on error). */
int blb_layernorm_head(blb_ctx* ctx, const blb_keys* keys, blb_ct* const* X, uint32_t count, uint32_t nc,
                       uint32_t L, uint32_t D, blb_ct** X_mu, blb_ct** var);

/* ---- local steps of the conversions between CKKS and shares -----------------
 * (Alg. 1 steps 3-4, Alg. 2, Sec. 6.3, App. C.3.)  Both parties' local
 * computations; the interactive comparisons inside the ring/field extensions
 * (Pi_Ext) are MPC protocols outside this library, and the *_wrap_sim calls
 * stand in for their ideal functionality.
 *
 * Rings: the MPC ring Z_{2^l} with fixed-point scale 2^-sf (the paper uses
 * l = 43, sf = 13; here sf <= 26 and sf + 2 <= l <= 62), values stored one per
 * uint64 word; the extended ring Z_{2^128}, each element two words (low,
 * high), arrays 16-byte aligned.  Shares are additive: x = x_0 + x_1 in the
 * ring.  Probabilistic truncation (SecureML): party 0 shifts its share (read
 * as a signed integer) right, party 1 takes the ceiling, so the sum is
 * floor(m / 2^k) + u with Pr[u = 1] = (m mod 2^k) / 2^k; it is wrong (by about
 * 2^(128-k)) only when the signed shares overflow, probability |m| / 2^128.
 * Fixed point of the share FFTs: roots round(2^30 zeta^k), data at 2^-26.
 *
 * Every array may be host or device memory; `count` members are stored one
 * after another.  Needs 2^12 <= N <= 2^17.  Errors: BLB_ERR_ARG for bad
 * sizes, ring widths, party or alignment, BLB_ERR_LEVEL, BLB_ERR_OOM.
 *
 * blb_f2r_wrap_sim: ideal functionality of the comparison inside field to
 * ring (signed Pi_Ext^{q_0, 2^128}).  t0, t1: count x N shares mod q_0 (party
 * 0 and 1) of centered coefficients.  Outputs w0, w1 (count x N x 2 words):
 * arithmetic shares of w = [(t0 + (q_0-1)/2 mod q_0) + t1 >= q_0], P0's share
 * rho the 128-bit Philox draw (i, 0, nonces[k] low 32 bits, purpose 7) keyed
 * by seed, P1's w - rho. */
int blb_f2r_wrap_sim(blb_ctx* ctx, const uint64_t* t0, const uint64_t* t1, uint32_t count, uint64_t seed,
                     const uint64_t* nonces, uint64_t* w0, uint64_t* w1);
/* blb_c2m_local (Alg. 1 steps 3-4): party's share t (count x N residues mod
 * q_0 in coefficient form: P0 the decryption of the masked ciphertext, P1 the
 * share blb_he2mpc returned) and its wrap-bit shares wsh (count x N x 2 words)
 * -> out (count x N/2 words mod 2^l): its share of the decoded slots at scale
 * 2^-sf.  Steps: field to ring; division by Delta / 2^26 (Delta = `scale`,
 * the ciphertext's scale) by truncation; the twist by zeta^t; the decoding FFT
 * with every root product truncated; slot j = real part at k_j = (5^j - 1)/4,
 * truncated to 2^-sf. */
int blb_c2m_local(blb_ctx* ctx, uint32_t party, const uint64_t* t, const uint64_t* wsh, uint32_t count,
                  double scale, uint32_t l, uint32_t sf, uint64_t* out);
/* blb_ext_wrap_sim: ideal functionality of the comparison inside the signed
 * extension Pi_Ext^{2^l, 2^128}: x0, x1 count x n shares mod 2^l, w0, w1 (count
 * x n x 2 words) shares of w = [(x0 + 2^(l-1) mod 2^l) + x1 >= 2^l]; Philox as
 * for blb_f2r_wrap_sim. */
int blb_ext_wrap_sim(blb_ctx* ctx, const uint64_t* x0, const uint64_t* x1, uint32_t n, uint32_t count, uint32_t l,
                     uint64_t seed, const uint64_t* nonces, uint64_t* w0, uint64_t* w1);
/* blb_m2c_local (Alg. 2 steps 1-2): party's shares x (count x n <= N/2 slot
 * values mod 2^l at scale 2^-sf; missing slots are 0) and wrap-bit shares wsh
 * (count x n x 2 words) -> out (count x (level+1) x N residues, coefficient
 * form): its share of Encode(x) = round(scale pi^-1(x)) mod q_0..q_level.
 * Steps: extension; the inverse FFT with each butterfly halved by a
 * truncation; the twist by scale zeta^-t; ring to field (each share read as a
 * signed 128-bit integer, reduced mod q_i).  P0 then encrypts its share
 * (blb_pt_import, blb_encrypt) and P1 adds its own (blb_pt_import,
 * blb_add_plain): Alg. 2 steps 3-4. */
int blb_m2c_local(blb_ctx* ctx, uint32_t party, const uint64_t* x, const uint64_t* wsh, uint32_t n, uint32_t count,
                  uint32_t level, double scale, uint32_t l, uint32_t sf, uint64_t* out);
/* Plaintext from (level+1) x N residues in coefficient form (host or device). */
int blb_pt_import(blb_ctx* ctx, const uint64_t* coeffs, uint32_t level, double scale, blb_pt** out);
/* a + b for a plaintext at the ciphertext's level or above (first polynomial
 * only); the scales must match. */
int blb_add_plain(blb_ctx* ctx, const blb_ct* a, const blb_pt* b, blb_ct** out);

/* ---- CUDA graphs ---------------------------------------------------------------
 * Every call that runs only kernels on device data (the matmul_cp / matmul_cc
 * products and their batched forms, key switching, rescale, the element-wise
 * operations, the batched masking and decryption into device buffers) can be
 * captured into a CUDA graph on the context's stream, with the capture in
 * relaxed mode and an allocator that serves stream-ordered allocations of the
 * capture from a private pool (the binding does this with PyTorch's graph
 * capture).  During a capture every table the library builds on the host goes
 * to a device buffer of its own (freed with the context), so a replay never
 * reads host memory; the key-switch arena must already be large enough, so run
 * the call once before capturing it (BLB_ERR_ARG otherwise).  During a capture
 * these return BLB_ERR_ARG before doing anything: a host input or output
 * buffer, encoding (it reads its overflow flag back), plan creation, the first
 * conversion of a context or with a new scale (they cache tables), blb_ntt and
 * blb_keyswitch_noalloc on host data.  Ciphertexts created during the capture
 * hold the results of the latest replay and must outlive the graph. */

/* ---- batches of the calls above -----------------------------------------------
 * Each computes, for every member, exactly what the single call computes (same
 * Philox streams, bit-identical limbs), but runs each step once over the whole
 * batch.  Handles in out/masked are new objects owned by the caller; on error
 * none is returned (all entries NULL).
 *
 * blb_encode_batch: vals holds count x n doubles (member k at vals + k n, host
 * or device), all at `level` and `scale`.
 * blb_encrypt_batch: pts share one level; nonces[k] is member k's nonce. */
int blb_encode_batch(blb_ctx* ctx, const double* vals, uint64_t n, uint32_t count, uint32_t level,
                     double scale, blb_pt** out);
int blb_encrypt_batch(blb_ctx* ctx, const blb_keys* keys, const blb_pt* const* pts, uint32_t count,
                      const uint64_t* nonces, blb_ct** out);
/* Masking of count ciphertexts (any levels): p1_shares receives count x N words
 * (member k at p1_shares + k N), masked[k] a new level-0 ciphertext. */
int blb_he2mpc_batch(blb_ctx* ctx, const blb_keys* keys, const blb_ct* const* cts, uint32_t count,
                     const uint64_t* nonces, blb_ct** masked, uint64_t* p1_shares);
/* Decryption of count ciphertexts of one level and size: coeff_limbs (nullable)
 * receives count x (level+1) x N words, slots (nullable) count x N/2 doubles. */
int blb_decrypt_batch(blb_ctx* ctx, const blb_keys* keys, const blb_ct* const* cts, uint32_t count,
                      uint64_t* coeff_limbs, double* slots);

/* ---- low-level transforms (parity testing) ------------------------------------
 * Forward / inverse negacyclic NTT of `rows` limbs of N words in place (host or
 * device).  Limb r uses prime q_{prime_idx[r]} (host array).  Forward output
 * order: A[k] = a(psi^(2 bitrev(k) + 1)) with psi the context's root for that
 * prime (first x = 2, 3, ... whose power x^((q-1)/2N) has order 2N). */
int blb_ntt(blb_ctx* ctx, uint64_t* data, uint32_t rows, const uint32_t* prime_idx, int inverse);
/* Transforms above 4096 points run in two passes over 4096-word tiles: a
 * column pass over 2^L1-point sub-transforms and a row pass over the rest.
 * split -1 / 0 / +1 puts L1 one below, at, or one above log2(N)/2.  Inside a
 * tile the butterfly stages run in register rounds of up to 3 stages (radix
 * 8, four CTAs per SM) or up to 4 (radix 16, three CTAs per SM).  Every split
 * and radix computes the same butterflies, so the limbs are identical.
 * blb_ntt_autotune times forward + inverse transforms of `rows` rows for each
 * radix and split, keeps the fastest pair for the context and returns it
 * (split_out, radix_out) with the time of each per row and direction in
 * microseconds (us_per_row[6]: radix 8 at splits -1, 0, +1, then radix 16 at
 * the same; 0 where a ring has one pass); all nullable.  Refused inside a
 * graph capture.  blb_ntt_set_split / blb_ntt_set_radix fix one by hand
 * (BLB_ERR_ARG outside {-1, 0, 1} / {8, 16}). */
int blb_ntt_autotune(blb_ctx* ctx, uint32_t rows, int* split_out, int* radix_out, double* us_per_row);
int blb_ntt_set_split(blb_ctx* ctx, int split);
int blb_ntt_set_radix(blb_ctx* ctx, int radix);

/* ---- measurement ------------------------------------------------------------
 * Total kernel launches issued by this library in this process. */
uint64_t blb_kernel_launches(void);
/* When enabled, CUDA events on the context's stream bracket each launch site
 * ("ntt", "intt", "intt_gather", "keyswitch", "cp_mac"; "intt_gather" is the
 * key switch's inverse transform of its sources with the automorphism's
 * gather in its first pass, kept apart from "intt" so that the latter counts
 * plain transforms only); blb_profile_read synchronizes the
 * stream and returns, since profiling was enabled, the summed milliseconds, the
 * number of bracketed calls and their algorithmic bytes (the minimum HBM
 * traffic of the operation: NTT one read and one write per word, 32 bytes per
 * word for "intt_gather" with the gather's read and digit write; key switch
 * its input, the used key digits and its output; cp_mac every plaintext, every
 * baby-step ciphertext and every partial sum once).  Enabling resets the sums. */
int blb_profile_enable(blb_ctx* ctx, int on);
int blb_profile_read(blb_ctx* ctx, const char* site, double* ms, uint64_t* count, uint64_t* bytes);
/* Bracket only the named site while profiling (NULL: every site, the default).
 * Each bracket is a pair of CUDA events on the stream, which also keeps the
 * next kernel from being scheduled early (programmatic dependent launch), so
 * fewer sites perturb the timed work less. */
int blb_profile_select(blb_ctx* ctx, const char* site);
/* The arithmetic of the calls bracketed at `site` since profiling was enabled,
 * for an ALU roofline beside the bytes: 64 x 64 -> 128-bit multiply-adds,
 * reductions of a 128-bit sum mod a prime, and NTT butterflies (a Shoup product
 * by a constant counted as one).  Counted by the "keyswitch" site (its ModUp,
 * inner products, ModDown and the NTTs between them); other sites report 0.
 * Outputs are nullable host pointers; BLB_ERR_ARG for a null ctx or site. */
int blb_profile_read_ops(blb_ctx* ctx, const char* site, uint64_t* mad128, uint64_t* reductions,
                         uint64_t* butterflies);

#ifdef __cplusplus
}
#endif
#endif
