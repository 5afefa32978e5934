// Plaintext-ciphertext multiply-accumulate of matmul_cp for batches of
// sequences on the 5th-generation tensor cores (tcgen05.mma, accumulators in
// tensor memory).
//
// The contraction is the one of mac_tc.cu (the inner sums of the BSGS
// diagonal method, Sec. 4.2 / Eq. 2): for limb i and coefficient j,
//
//     T[s][eg][p][i][j] = sum_t  D[eg][t][i][j] * X[s][t][p][i][j]   (mod q_i),
//
// computed exactly from byte planes, D = sum_a 2^{8a} D_a, X = sum_b 2^{8b} X_b.
// Per item (coefficient j, block of 16 outputs eg) one UMMA of shape
// M = 128 x N x K = 16 KT forms every plane product at once:
//
//     A (M x K):  row 8 e + a = byte plane a of output e's diagonal (rows
//                 with a >= NB are zero), K = the terms t,
//     B (N x K):  row b 2S + 2s + p = byte plane b of X[s][t][p],
//     C (M x N):  fp32 sums  sum_t D_a[e][t] X_b[s][t][p].
//
// The bytes enter as fp16 subnormals (the bit pattern 0x00XX is XX 2^-24), so
// every product is exact and every sum of at most 128 of them is n 2^-48 with
// an integer n < 2^23, exact in fp32.  The epilogue reads each accumulator
// row (one TMEM lane per thread), turns the fp32 sums back into the integers
// n (the bit pattern of x + 2^-25 is a fixed bias plus n), recombines them with
// their weights 2^{8(a+b)} into 128-bit sums, adds the 8 rows of each output
// across the lanes that hold them (a transposing shuffle, so each lane keeps a
// share of the sums), removes the bias and reduces mod q_i (Barrett).
//
// Roles (one CTA per SM, persistent over tiles of CT coefficients):
//   warp 0   : streams each item's plaintext bytes (one contiguous range in
//              the plan) into a ring of shared-memory stages (cp.async.bulk
//              completed on mbarriers);
//   warp 1   : allocates the tensor memory and issues the UMMAs (one elected
//              thread), double-buffered accumulators, tcgen05.commit to
//              mbarriers;
//   warps 2-9: build the tile's B operands (CT coefficients) from the
//              baby-step ciphertexts and convert each item's plaintext bytes
//              into the A operand, both in the canonical K-major layout of
//              8 x 16-byte core matrices (no swizzle);
//   warps 10-17: the epilogue above, two warpgroups that take half of the
//              (sequence, polynomial) columns each (warp w reads TMEM lanes
//              32 (w % 4) ...).
// Every wait is bounded (the context's wait limit): an expired wait sets an
// abort word that ends the other roles and the status word that
// blb_ctx_sync reports; copies and UMMAs in flight are waited for before the
// tensor memory is freed and the CTA exits.
#include "common.cuh"

#include <atomic>

namespace {

constexpr int UM_BUILD = 256;     // operand builders (warps 2-9)
constexpr int UM_THREADS = 576;   // + producer, UMMA issuer, 8 epilogue warps
constexpr uint64_t UM_DRAIN_NS = 2000000000ull;  // the final drains always allow 2 s
constexpr float UM_BIAS = 2.98023223876953125e-08f;  // 2^-25
constexpr uint32_t UM_BIAS_BITS = 0x33000000u;

struct UmArgs {
    uint64_t* T;
    const uint64_t* baby;
    const uint8_t* ptb;
    const uint64_t* q;
    const uint64_t* bar;
    uint32_t* status;
    uint64_t nN, seq_words, wait_ns;
    uint32_t N, terms, KT, neg, NEB, CT;
    uint32_t tiles_per_limb, tiles, withhold, R;
    uint32_t nacc, accw;  // tensor-memory accumulators and their column stride
    uint32_t limb[64];
    uint64_t off[64];
};

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mb_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// wait for the phase of the given parity; false after limit_ns or once another
// thread of the CTA has given up (abort word)
__device__ __forceinline__ bool mb_wait(uint32_t bar, uint32_t parity, volatile uint32_t* abort, uint64_t limit_ns)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; it++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it == 0) {
            t0 = gtime();
        } else if ((it & 63) == 0) {
            if (*abort || gtime() - t0 > limit_ns) {
                *abort = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// shared-memory matrix descriptor: canonical K-major layout without swizzle,
// lbo = byte distance of core matrices adjacent along K, sbo = along M / N
// (here the row-group stride: kc core matrices plus 16 bytes of padding, so
// that the builders' stores to the 8 row groups hit different banks)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// byte offset of element (row, k) in a canonical K-major tile with kc core
// matrices along K and a padded row-group stride
__device__ __forceinline__ uint32_t canon(uint32_t row, uint32_t k, uint32_t kc)
{
    return (row >> 3) * (kc * 128u + 16u) + (k >> 3) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

__device__ __forceinline__ uint64_t reduce128u(uint64_t lo, uint64_t hi, uint64_t q, uint64_t r0, uint64_t r1)
{
    const uint64_t h = barrett128(hi, 0, q, r0, r1);  // hi mod q: (h, lo) < q 2^64
    return barrett128(lo, h, q, r0, r1);
}

template <int S, int NB>
struct UmShape {
    static constexpr int SP = 2 * S;                    // (sequence, polynomial) columns per byte plane
    static constexpr int NCOL = NB * SP;                // rows of B that carry data
    static constexpr int NPAD = (NCOL + 15) / 16 * 16;  // UMMA N
    static_assert(NPAD <= 128, "B operand too wide");
    static_assert(NB >= 3 && NB <= 8, "byte planes");
};

template <int S, int NB, int NA>
__global__ void __launch_bounds__(UM_THREADS, 1) k_cp_mac_umma(const __grid_constant__ UmArgs A)
{
    using G_ = UmShape<S, NB>;
    constexpr int SP = G_::SP, NPAD = G_::NPAD;
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t KC = A.KT * 2;
    const uint32_t item_bytes = A.KT * NB * 256;
    const uint32_t a_bytes = 16 * (KC * 128 + 16);             // one A operand (16 row groups)
    const uint32_t b_bytes = (uint32_t)(NPAD / 8) * (KC * 128 + 16);  // one coefficient's B operand
    const uint32_t IPT = A.CT * A.NEB;
    // layout: ring | A[NA] | B[2][CT] | barriers
    uint8_t* ring = smem;
    uint8_t* abuf = ring + A.R * item_bytes;
    uint8_t* bbuf = abuf + NA * a_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(bbuf + 2 * A.CT * b_bytes);
    // full[R] empty[R] afull[NA] afree[NA] bfull[2] bdone[2] accfull[2] accempty[2] fin
    const uint32_t UM_R = A.R;
    const uint32_t full0 = su32(bars), empty0 = full0 + 8 * UM_R, afull0 = empty0 + 8 * UM_R,
                   afree0 = afull0 + 8 * NA, bfull0 = afree0 + 8 * NA, bdone0 = bfull0 + 16, accf0 = bdone0 + 16,
                   acce0 = accf0 + 8 * A.nacc, fin = acce0 + 8 * A.nacc;
    const uint32_t NACC = A.nacc;
    volatile uint32_t* abort = reinterpret_cast<volatile uint32_t*>(bars + 2 * UM_R + 2 * NA + 2 * NACC + 5);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * UM_R + 2 * NA + 2 * NACC + 6);

    // zero A and B (padding rows and terms stay zero)
    for (uint32_t x = threadIdx.x; x < (NA * a_bytes + 2 * A.CT * b_bytes) / 16; x += UM_THREADS)
        reinterpret_cast<uint4*>(abuf)[x] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        for (uint32_t r = 0; r < UM_R; r++) {
            mb_init(full0 + 8 * r, 1);
            mb_init(empty0 + 8 * r, 8);  // every builder warp
        }
        for (int b = 0; b < NA; b++) {
            mb_init(afull0 + 8 * b, 8);
            mb_init(afree0 + 8 * b, 1);
        }
        for (int b = 0; b < 2; b++) {
            mb_init(bfull0 + 8 * b, 8);
            mb_init(bdone0 + 8 * b, 1);
        }
        for (uint32_t b = 0; b < NACC; b++) {
            mb_init(accf0 + 8 * b, 1);
            mb_init(acce0 + 8 * b, 8);
        }
        mb_init(fin, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {  // 256 columns: two accumulators of up to 128 fp32 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeroed operands
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint64_t wlim = A.wait_ns;

    if (warp == 0) {
        // ---- plaintext stream (lane 0)
        if (lane == 0) {
            uint32_t issued = 0;
            for (uint32_t lt = 0, tau = blockIdx.x; !A.withhold && tau < A.tiles && !*abort; lt++, tau += gridDim.x) {
                const uint32_t gi = tau / A.tiles_per_limb, j0 = (tau % A.tiles_per_limb) * A.CT;
                const uint8_t* src = A.ptb + A.off[gi] + (size_t)j0 * A.NEB * item_bytes;
                for (uint32_t it = 0; it < IPT; it++) {
                    const uint32_t g = lt * IPT + it, st = g % UM_R;
                    if (g >= UM_R && !mb_wait(empty0 + 8 * st, ((g / UM_R) - 1) & 1, abort, wlim)) break;
                    mb_expect_tx(full0 + 8 * st, item_bytes);
                    bulk_g2s(su32(ring + st * item_bytes), src + (size_t)it * item_bytes, item_bytes, full0 + 8 * st);
                    issued = g + 1;
                }
            }
            // the copies started here land in shared memory whatever the other roles do
            for (uint32_t g = issued > UM_R ? issued - UM_R : 0; g < issued; g++) {
                uint32_t dummy = 0;
                mb_wait(full0 + 8 * (g % UM_R), (g / UM_R) & 1, &dummy, UM_DRAIN_NS);
            }
        }
    } else if (warp == 1) {
        // ---- UMMA issue (lane 0)
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | ((uint32_t)(NPAD >> 3) << 17) | ((128u >> 4) << 24);
            bool any = false;
            for (uint32_t lt = 0, tau = blockIdx.x; tau < A.tiles && !*abort; lt++, tau += gridDim.x) {
                const uint32_t bb = lt & 1;
                if (!mb_wait(bfull0 + 8 * bb, (lt >> 1) & 1, abort, wlim)) break;
                bool ok = true;
                for (uint32_t it = 0; it < IPT && ok; it++) {
                    const uint32_t g = lt * IPT + it, ab = g % NACC, jj = it / A.NEB, an = g % NA;
                    ok = mb_wait(afull0 + 8 * an, (g / NA) & 1, abort, wlim);
                    if (ok && g >= NACC) ok = mb_wait(acce0 + 8 * ab, ((g / NACC) - 1) & 1, abort, wlim);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = su32(abuf + an * a_bytes), b0 = su32(bbuf + (bb * A.CT + jj) * b_bytes);
                    const uint32_t d = tmem + ab * A.accw;
                    for (uint32_t ks = 0; ks < A.KT; ks++) {
                        const uint64_t ad = sdesc(a0 + ks * 256, 128, KC * 128 + 16);
                        const uint64_t bd = sdesc(b0 + ks * 256, 128, KC * 128 + 16);
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(ks)
                            : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     accf0 + 8 * ab)
                                 : "memory");
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     afree0 + 8 * an)
                                 : "memory");
                    any = true;
                }
                if (!ok) break;
                // the tile's B operands are free once its last products complete
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 bdone0 + 8 * bb)
                             : "memory");
            }
            // no product may still read shared memory or write tensor memory
            // when the CTA frees them
            if (any) {
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(fin)
                             : "memory");
                uint32_t dummy = 0;
                mb_wait(fin, 0, &dummy, UM_DRAIN_NS);
            }
        }
        __syncwarp();
    } else if (warp < 10) {
        // ---- operand builders (256 threads, warps 2-9).  Each warp's lane 0
        // waits on the barriers for its warp, and each warp arrives on the
        // barriers of what it built (counts of 8).
        const uint32_t c = threadIdx.x - 64;
        const uint32_t TPR = (A.terms + 1) >> 1;
        for (uint32_t lt = 0, tau = blockIdx.x; tau < A.tiles; lt++, tau += gridDim.x) {
            const uint32_t gi = tau / A.tiles_per_limb, i = A.limb[gi], j0 = (tau % A.tiles_per_limb) * A.CT;
            const uint32_t bb = lt & 1;
            bool w0 = true;
            if (lane == 0 && lt >= 2) w0 = mb_wait(bdone0 + 8 * bb, ((lt >> 1) - 1) & 1, abort, wlim);
            if (!__shfl_sync(0xffffffffu, w0, 0)) break;
            // B: rows (b, s, p), terms t, t + 1 as one fp16 pair, CT coefficients;
            // two rows (s, t pair, p) per thread and round, all their loads first
            const uint32_t nf = (uint32_t)S * TPR * 2;
            for (uint32_t f0 = c; f0 < nf; f0 += 2 * UM_BUILD) {
                uint64_t w[2][2][4];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const uint32_t f = f0 + u * UM_BUILD;
                    const uint32_t p = f & 1, tp = (f >> 1) % TPR, s = (f >> 1) / TPR, t = 2 * tp;
                    const bool in = f < nf, has1 = in && t + 1 < A.terms;
                    const uint64_t* x0 = A.baby + (size_t)s * A.seq_words + ((size_t)t * 2 + p) * A.nN + (size_t)i * A.N + j0;
                    const uint64_t* x1 = x0 + 2 * A.nN;
#pragma unroll
                    for (int jj = 0; jj < 4; jj++) w[u][0][jj] = w[u][1][jj] = 0;
                    if (A.CT == 4) {
                        if (in) {
                            const ulonglong2 a0 = __ldg(reinterpret_cast<const ulonglong2*>(x0));
                            const ulonglong2 a1 = __ldg(reinterpret_cast<const ulonglong2*>(x0) + 1);
                            w[u][0][0] = a0.x, w[u][0][1] = a0.y, w[u][0][2] = a1.x, w[u][0][3] = a1.y;
                        }
                        if (has1) {
                            const ulonglong2 b0 = __ldg(reinterpret_cast<const ulonglong2*>(x1));
                            const ulonglong2 b1 = __ldg(reinterpret_cast<const ulonglong2*>(x1) + 1);
                            w[u][1][0] = b0.x, w[u][1][1] = b0.y, w[u][1][2] = b1.x, w[u][1][3] = b1.y;
                        }
                    } else if (A.CT == 2) {
                        if (in) {
                            const ulonglong2 a0 = __ldg(reinterpret_cast<const ulonglong2*>(x0));
                            w[u][0][0] = a0.x, w[u][0][1] = a0.y;
                        }
                        if (has1) {
                            const ulonglong2 b0 = __ldg(reinterpret_cast<const ulonglong2*>(x1));
                            w[u][1][0] = b0.x, w[u][1][1] = b0.y;
                        }
                    } else {
                        if (in) w[u][0][0] = __ldg(x0);
                        if (has1) w[u][1][0] = __ldg(x1);
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const uint32_t f = f0 + u * UM_BUILD;
                    if (f >= nf) break;
                    const uint32_t p = f & 1, tp = (f >> 1) % TPR, s = (f >> 1) / TPR, t = 2 * tp;
#pragma unroll
                    for (int jj = 0; jj < 4; jj++) {
                        if (jj >= (int)A.CT) break;
                        uint8_t* Bj = bbuf + (bb * A.CT + jj) * b_bytes;
#pragma unroll
                        for (int b = 0; b < NB; b++) {
                            const uint32_t lo = (uint32_t)(w[u][0][jj] >> (8 * b)) & 0xFFu;
                            const uint32_t hi = (uint32_t)(w[u][1][jj] >> (8 * b)) & 0xFFu;
                            *reinterpret_cast<uint32_t*>(Bj + canon(b * SP + 2 * s + p, t, KC)) = lo | (hi << 16);
                        }
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mb_arrive(bfull0 + 8 * bb);
            bool ok = true;
            for (uint32_t it = 0; it < IPT; it++) {
                const uint32_t g = lt * IPT + it, st = g % UM_R, an = g % NA;
                bool w = true;
                if (lane == 0) {
                    // the A buffer is free once the products of item g - NA completed
                    if (g >= NA) w = mb_wait(afree0 + 8 * an, ((g / NA) - 1) & 1, abort, wlim);
                    if (w) w = mb_wait(full0 + 8 * st, (g / UM_R) & 1, abort, wlim);
                }
                ok = __shfl_sync(0xffffffffu, w, 0);
                if (!ok) break;
                // A: fragment-ordered plaintext bytes (see mac_tc.cu) -> rows 8 e + a
                const uint8_t* src = ring + st * item_bytes;
                uint8_t* Ad = abuf + an * a_bytes;
                for (uint32_t x = c; x < A.KT * NB * 32; x += UM_BUILD) {
                    const uint32_t l = x & 31, kta = x >> 5, a = kta % NB, kt = kta / NB;
                    const uint2 v = *reinterpret_cast<const uint2*>(src + (size_t)x * 8);
                    const uint32_t g8 = l >> 2, h4 = l & 3, kb = kt * 16 + 2 * h4;
                    // bytes 0,1: (g, 2h..), 2,3: (g + 8, 2h..), 4,5: (g, 2h + 8..), 6,7: (g + 8, 2h + 8..)
                    *reinterpret_cast<uint32_t*>(Ad + canon(g8 * 8 + a, kb, KC)) = __byte_perm(v.x, 0, 0x4140);
                    *reinterpret_cast<uint32_t*>(Ad + canon((g8 + 8) * 8 + a, kb, KC)) = __byte_perm(v.x, 0, 0x4342);
                    *reinterpret_cast<uint32_t*>(Ad + canon(g8 * 8 + a, kb + 8, KC)) = __byte_perm(v.y, 0, 0x4140);
                    *reinterpret_cast<uint32_t*>(Ad + canon((g8 + 8) * 8 + a, kb + 8, KC)) = __byte_perm(v.y, 0, 0x4342);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mb_arrive(empty0 + 8 * st);
                    mb_arrive(afull0 + 8 * an);
                }
            }
            if (!ok) break;
        }
    } else {
        // ---- epilogue (warps 10-17): TMEM lane row = 32 (warp % 4) + lane =
        // 8 e + a; warpgroup h takes columns sp in [h SH, (h + 1) SH) of every plane
        constexpr int SH = SP / 2;
        const uint32_t quarter = warp & 3, h = (warp - 10) >> 2;
        const uint32_t row = quarter * 32 + lane, e = row >> 3, a = row & 7;
        // every plane sum entered as UM_BIAS_BITS + n: the 8 rows of an output
        // (padding rows included) bring sum_{a < 8, b < NB} UM_BIAS_BITS 2^{8(a+b)}
        uint64_t bias_lo = 0, bias_hi = 0;
#pragma unroll
        for (int aa = 0; aa < 8; aa++)
#pragma unroll
            for (int b = 0; b < NB; b++) {
                const int sh = 8 * (aa + b);
                const uint64_t lo = sh < 64 ? (uint64_t)UM_BIAS_BITS << sh : 0;
                const uint64_t hi = sh == 0 ? 0 : sh < 64 ? (uint64_t)UM_BIAS_BITS >> (64 - sh)
                                                          : (uint64_t)UM_BIAS_BITS << (sh - 64);
                const uint64_t l2 = bias_lo + lo;
                bias_hi += hi + (l2 < lo);
                bias_lo = l2;
            }
        for (uint32_t lt = 0, tau = blockIdx.x; tau < A.tiles; lt++, tau += gridDim.x) {
            const uint32_t gi = tau / A.tiles_per_limb, i = A.limb[gi], j0 = (tau % A.tiles_per_limb) * A.CT;
            const uint64_t q = A.q[i], r0 = A.bar[2 * i], r1 = A.bar[2 * i + 1];
            bool ok = true;
            for (uint32_t it = 0; it < IPT; it++) {
                const uint32_t g = lt * IPT + it, ab = g % NACC, jj = it / A.NEB, eblk = it % A.NEB;
                ok = mb_wait(accf0 + 8 * ab, (g / NACC) & 1, abort, wlim);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                uint64_t P0[SH], P1[SH];
#pragma unroll
                for (int u = 0; u < SH; u++) P0[u] = P1[u] = 0;
                const uint32_t taddr = tmem + ((quarter * 32u) << 16) + ab * A.accw + h * SH;
                uint32_t r[NB][SH];
#pragma unroll
                for (int b = 0; b < NB; b++) {
                    if constexpr (SH == 8) {
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                     : "=r"(r[b][0]), "=r"(r[b][1]), "=r"(r[b][2]), "=r"(r[b][3]), "=r"(r[b][4]),
                                       "=r"(r[b][5]), "=r"(r[b][6]), "=r"(r[b][7])
                                     : "r"(taddr + b * SP));
                    } else if constexpr (SH == 4) {
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                                     : "=r"(r[b][0]), "=r"(r[b][1]), "=r"(r[b][2]), "=r"(r[b][3])
                                     : "r"(taddr + b * SP));
                    } else {
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
                                     : "=r"(r[b][0]), "=r"(r[b][1])
                                     : "r"(taddr + b * SP));
                    }
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // the accumulator may be overwritten once every warp has read it
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mb_arrive(acce0 + 8 * ab);
#pragma unroll
                for (int b = 0; b < NB; b++)
#pragma unroll
                    for (int u = 0; u < SH; u++) {
                        const uint32_t n = __float_as_uint(__uint_as_float(r[b][u]) + UM_BIAS);
                        if (b < 4) P0[u] += (uint64_t)n * (1ull << (8 * b));
                        else P1[u] += (uint64_t)n * (1ull << (8 * (b - 4)));
                    }
                // this lane's 128-bit share: (P0 + P1 2^32) 2^{8a}
                acc128 v[SH];
                const uint32_t sh = 8 * a;
#pragma unroll
                for (int u = 0; u < SH; u++) {
                    uint64_t lo = P0[u] + (P1[u] << 32);
                    uint64_t hi = (P1[u] >> 32) + (lo < P0[u]);
                    if (sh) {
                        hi = (hi << sh) | (lo >> (64 - sh));
                        lo <<= sh;
                    }
                    v[u] = {lo, hi};
                }
                // add the 8 lanes of each output (a = 0..7), each lane keeping
                // a share of the SH sums: halves exchanged over lane masks 4, 2, 1
                uint32_t base = 0;
                int cnt = SH;
#pragma unroll
                for (int m = 4; m >= 1; m >>= 1) {
                    if (cnt >= 2) {
                        const int half = cnt / 2;
                        const bool up = lane & m;
#pragma unroll
                        for (int u = 0; u < SH / 2; u++) {
                            if (u >= half) break;
                            const acc128 send = up ? v[u] : v[u + half];
                            const acc128 keep = up ? v[u + half] : v[u];
                            const uint64_t olo = __shfl_xor_sync(0xffffffffu, send.lo, m);
                            const uint64_t ohi = __shfl_xor_sync(0xffffffffu, send.hi, m);
                            const uint64_t l2 = keep.lo + olo;
                            v[u] = {l2, keep.hi + ohi + (l2 < olo)};
                        }
                        if (up) base += half;
                        cnt = half;
                    } else {
                        const uint64_t olo = __shfl_xor_sync(0xffffffffu, v[0].lo, m);
                        const uint64_t ohi = __shfl_xor_sync(0xffffffffu, v[0].hi, m);
                        const uint64_t l2 = v[0].lo + olo;
                        v[0] = {l2, v[0].hi + ohi + (l2 < olo)};
                    }
                }
                // SH = 8: every lane holds one distinct sum; SH = 4 / 2: lane
                // pairs / quads hold the same sum, and one of them stores it
                const bool store = SH >= 8 || (lane & (8 / SH - 1)) == 0;
                const uint32_t eg = eblk * 16 + e;
                if (store && eg < A.neg) {
                    const uint64_t lo = v[0].lo - bias_lo;
                    const uint64_t hi = v[0].hi - bias_hi - (v[0].lo < bias_lo);
                    const uint32_t sp = h * SH + base;
                    A.T[((size_t)((sp >> 1) * A.neg + eg) * 2 + (sp & 1)) * A.nN + (size_t)i * A.N + j0 + jj] =
                        reduce128u(lo, hi, q, r0, r1);
                }
            }
            if (!ok) break;
        }
    }
    // every role sets the status word if the CTA gave up
    if (lane == 0 && *abort) atomicExch(A.status, 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// shared memory of one CTA: ring, two A operands, two tiles of CT B operands, barriers
size_t umma_smem(uint32_t S, uint32_t NB, uint32_t KT, uint32_t CT, uint32_t NA = 2, uint32_t R = 4)
{
    const size_t grp = (size_t)KT * 2 * 128 + 16, npad = (NB * 2 * S + 15) / 16 * 16;  // padded row-group stride
    return R * (size_t)KT * NB * 256 + NA * 16 * grp + 2 * CT * (npad / 8) * grp + 8 * (2 * R + 2 * NA + 2 * 8 + 7);
}
constexpr size_t UM_SMEM_MAX = 225u << 10;

template <int S, int NB>
int launch_umma(blb_ctx* c, UmArgs& a, uint32_t nlimbs, bool* used)
{
    // shared memory, in order of priority: B tiles of up to four coefficients
    // (whole 32-byte sectors of the baby-step rows), four ring stages, a third
    // A buffer (measured on the B300: deeper rings gave nothing)
    uint32_t R = 4, NA = 2;
    a.CT = 4;
    while (a.CT > 1 && umma_smem(S, NB, a.KT, a.CT, NA, R) > UM_SMEM_MAX) a.CT >>= 1;
    while (R > 2 && umma_smem(S, NB, a.KT, a.CT, NA, R) > UM_SMEM_MAX) R--;
    if (umma_smem(S, NB, a.KT, a.CT, NA, R) > UM_SMEM_MAX) return BLB_OK;  // not used: the operands do not fit
    if (umma_smem(S, NB, a.KT, a.CT, 3, R) <= UM_SMEM_MAX) NA = 3;
    a.R = R;
    const bool three = NA == 3;
    // accumulators: as many as the 512 tensor-memory columns hold, up to 8, at
    // a power-of-two column stride
    a.accw = 32;
    while (a.accw < (uint32_t)UmShape<S, NB>::NPAD) a.accw <<= 1;
    a.nacc = std::min<uint32_t>(8, 512 / a.accw);
    a.tiles_per_limb = c->N / a.CT;
    a.tiles = a.tiles_per_limb * nlimbs;
    static std::atomic<bool> attr[64];
    int dev = 0, sms = 0;
    BLB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return blb_fail(BLB_ERR_ARG, "device ordinal beyond 64");
    if (!attr[dev].load()) {
        BLB_CUDA(cudaFuncSetAttribute(k_cp_mac_umma<S, NB, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 << 10));
        BLB_CUDA(cudaFuncSetAttribute(k_cp_mac_umma<S, NB, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 << 10));
        attr[dev].store(true);
    }
    BLB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint32_t grid = std::min<uint32_t>(a.tiles, (uint32_t)sms);
    // one CTA per SM (it allocates all 512 tensor-memory columns): the request
    // never lets a second CTA fit next to it
    const size_t smem = std::max<size_t>(umma_smem(S, NB, a.KT, a.CT, three ? 3 : 2, R), 120u << 10);
    if (three) k_cp_mac_umma<S, NB, 3><<<grid, UM_THREADS, smem, c->stream>>>(a);
    else k_cp_mac_umma<S, NB, 2><<<grid, UM_THREADS, smem, c->stream>>>(a);
    BLB_LAUNCHED();
    *used = true;
    return BLB_OK;
}

template <int S>
int launch_umma_nb(blb_ctx* c, UmArgs& a, uint32_t nb, uint32_t nlimbs, bool* used)
{
    switch (nb) {
    case 3: return launch_umma<S, 3>(c, a, nlimbs, used);
    case 4: return launch_umma<S, 4>(c, a, nlimbs, used);
    case 5: return launch_umma<S, 5>(c, a, nlimbs, used);
    case 6: return launch_umma<S, 6>(c, a, nlimbs, used);
    case 7: return launch_umma<S, 7>(c, a, nlimbs, used);
    case 8: return launch_umma<S, 8>(c, a, nlimbs, used);
    default: return BLB_OK;
    }
}

}  // namespace

// The batched MAC on tcgen05 for S = 2, 4 or 8 sequences, when every limb group
// fits it (at most 128 terms per output: one exact fp32 accumulation; 64 for
// primes above 2^60).  *used tells whether it ran; otherwise the caller runs
// the mma.sync kernel.  Limb groups and algorithmic bytes as launch_cp_mac.
int launch_cp_mac_umma(blb_ctx* c, const blb_cp_plan* P, const uint64_t* baby, uint64_t* T, uint32_t S, bool* used)
{
    *used = false;
    if (S != 2 && S != 4 && S != 8) return BLB_OK;
    const uint32_t n = P->level + 1, N = c->N;
    for (uint32_t i = 0; i < n; i++)  // one exact accumulation per item, and every limb group's operands fit
        if (P->KT > (c->q[i] >= (1ull << 60) ? 4u : 8u) || P->nb[i] < 3 || P->nb[i] > 8 ||
            umma_smem(S, P->nb[i], P->KT, 1, 2, 2) > UM_SMEM_MAX)
            return BLB_OK;
    UmArgs a{};
    a.T = T;
    a.baby = baby;
    a.ptb = P->d_ptb;
    a.q = c->d_q;
    a.bar = c->d_bar;
    a.status = c->d_status;
    a.wait_ns = c->wait_ns ? c->wait_ns : 2000000000ull;
    a.withhold = c->mac_withhold;
    a.nN = (uint64_t)n * N;
    a.terms = P->nX * P->b1;
    a.seq_words = (uint64_t)a.terms * 2 * a.nN;
    a.N = N;
    a.KT = P->KT;
    a.neg = P->nY * P->G;
    a.NEB = P->NEB;
    for (uint32_t nb = 3; nb <= 8; nb++) {
        uint32_t cnt = 0;
        for (uint32_t i = 0; i < n; i++)
            if (P->nb[i] == nb) {
                if (cnt == 64) return blb_fail(BLB_ERR_PARAM, "too many limbs");
                a.limb[cnt] = i;
                a.off[cnt] = P->off[i];
                cnt++;
            }
        if (!cnt) continue;
        bool u = false;
        int rc;
        switch (S) {
        case 2: rc = launch_umma_nb<2>(c, a, nb, cnt, &u); break;
        case 4: rc = launch_umma_nb<4>(c, a, nb, cnt, &u); break;
        default: rc = launch_umma_nb<8>(c, a, nb, cnt, &u); break;
        }
        if (rc) return rc;
        if (!u) return blb_fail(BLB_ERR_ARG, "tcgen05 MAC: operands do not fit shared memory");
    }
    *used = true;
    return BLB_OK;
}
