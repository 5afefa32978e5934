// Plaintext-ciphertext multiply-accumulate of matmul_cp (the inner sums of the
// BSGS diagonal method, Sec. 4.2 / Eq. 2) on the tensor cores.
//
// For one RNS limb i and one coefficient j (NTT domain, so every coefficient is
// independent) the step computes, for S sequences,
//
//     T[s][eg][p][i][j] = sum_t  D[eg][t][i][j] * X[s][t][p][i][j]   (mod q_i)
//
// with eg = (e, g) the output/giant-step pair, t = (c, b) the input/baby-step
// pair and p the ciphertext polynomial.  Per coefficient this is a dense
// (outputs x terms) . (terms x 2S) contraction.  Both operands are split into
// bytes, D = sum_a 2^{8a} D_a and X = sum_b 2^{8b} X_b, so that every byte
// product is exact in fp16 and every 16-term block sum of byte products stays
// below 2^24, exact in the fp32 accumulators of mma.sync.m16n8k16:
//
//     sum_t D X = sum_{a,b} 2^{8(a+b)} (sum_t D_a X_b).
//
// The bytes of D and X enter as fp16 subnormals (XX 2^-24, one byte permute
// per pair), so the fp32 sums come out scaled by 2^-48, still exact.
// The byte planes of D are the GEMM's M dimension (rows (a, eg)), those of X
// are part of N (columns (b, s, p)).  The epilogue reads the exact fp32 sums
// back as integers, adds them with their shifts 2^{8(a+b)} into four 64-bit
// columns of weight 2^{32c} (no carries on the way), assembles the 128-bit sum
// and, once the lanes that hold other byte planes of the same sums have added
// theirs (a transposing shuffle), reduces it mod q_i (Barrett).  Segments of at
// most 8 term tiles (4 for primes above 2^60) keep the fp32 sums below 2^23
// and the 128-bit sums exact.
//
// Plan layout (bytes): for limb i a region at off[i]; inside it, for each
// coefficient j, each 16-output block, each 16-term tile kt and each byte
// plane a (nb_i = ceil(bits(q_i)/8) planes), one 256-byte mma A fragment: lane
// l = 4 g + h holds 8 bytes for (row, col) = (g + 8 ((e >> 1) & 1),
// 2 h + (e & 1) + 8 (e >> 2)), e = 0..7.  The items (coefficient, output
// block) of a tile of CT coefficients are therefore one contiguous byte range.
//
// Persistent CTAs (as many as fit on the SMs) walk the tiles.  A builder warp
// turns each tile's baby-step ciphertexts into mma B fragments, one tile ahead,
// in one of two shared buffers; a streamer warp copies the tiles' plaintext
// ranges into a ring of shared-memory stages with cp.async.bulk copies
// completed on mbarriers, without pausing between tiles; the consumer warps
// (8 for one sequence, 4 for batches, one ring stage each) take the items in
// turn, hand each stage back right after its last mma, and run the epilogue
// while the next copies land.  Every wait is
// bounded: an expired wait sets a CTA abort word that ends the other waits,
// and the status word the host reads in blb_ctx_sync.
#include "common.cuh"

#include <cuda_fp16.h>

#include <atomic>

namespace {

// Consumer warps per CTA (W, plus a plaintext streamer and a B builder): 8 for
// one sequence, 4 for batches (measured on B300 at the BERT-base products); the
// ring has one stage per consumer and a B buffer holds 16 KB (more for batches
// whose tiles the launcher widens, as long as two CTAs still fit on an SM).
constexpr int mac_consumers(int S) { return S == 1 ? 8 : 4; }
constexpr int mac_threads(int S) { return 32 * (mac_consumers(S) + 2); }
constexpr uint32_t MAC_BBUF_BYTES = 16u << 10;
constexpr int MAC_MAX_GROUP = 64;  // limbs per launch
constexpr uint32_t MAC_MAX_BBUFS = 4;
constexpr uint64_t MAC_WAIT_NS = 2000000000ull;  // bounded waits: 2 s by default

struct MacArgs {
    uint64_t* T;
    const uint64_t* baby;
    const uint8_t* ptb;
    const uint64_t* q;
    const uint64_t* bar;
    uint32_t* status;
    uint64_t nN, seq_words;
    uint32_t N, terms, KT, neg, NEB, CT, kseg, R, jstride;
    uint32_t tiles_per_limb, tiles;  // coefficient tiles of CT per limb, over all limbs of the launch
    uint32_t nbb;                    // B fragment buffers (2 .. MAC_MAX_BBUFS)
    uint32_t selfb;                  // batches of one item per tile: each consumer builds its own B
    uint32_t withhold;               // test hook: the streamer issues no copy, so the consumers' waits run out
    uint64_t wait_ns;                // limit of the pipeline's waits (the final drain always allows MAC_WAIT_NS)
    uint32_t limb[MAC_MAX_GROUP];
    uint64_t off[MAC_MAX_GROUP];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Wait for the phase of the given parity to complete.  Returns false after
// limit_ns, or as soon as another thread of the CTA has given up (abort word
// in shared memory), so that one expired wait ends the whole CTA quickly.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile uint32_t* abort, uint64_t limit_ns)
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
            t0 = globaltimer();
        } else if ((it & 63) == 0) {
            if (*abort || globaltimer() - t0 > limit_ns) {
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

// 8 bytes -> 4 registers of fp16 pairs (low half = lower byte), one byte
// permute per pair: the bit pattern 0x00XX is the subnormal fp16 number
// XX 2^-24 (exact: the tensor cores take fp16 subnormals as they are, and the
// scale only moves the exponent of every fp32 partial sum)
__device__ __forceinline__ void bytes_to_f16x2(uint2 v, uint32_t (&f)[4])
{
    f[0] = __byte_perm(v.x, 0, 0x4140);
    f[1] = __byte_perm(v.x, 0, 0x4342);
    f[2] = __byte_perm(v.y, 0, 0x4140);
    f[3] = __byte_perm(v.y, 0, 0x4342);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint2 b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ uint64_t reduce128(uint64_t lo, uint64_t hi, uint64_t q, uint64_t r0, uint64_t r1)
{
    const uint64_t h = barrett128(hi, 0, q, r0, r1);  // hi mod q, so (h:lo) < q 2^64
    return barrett128(lo, h, q, r0, r1);
}

// byte planes of D accumulated together: all of them when the accumulators fit
// 64 registers, else the largest divisor of NB that does
template <int NB, int NT>
constexpr int plane_group()
{
    for (int g = NB; g >= 1; g--)
        if (NB % g == 0 && g * NT * 4 <= 64) return g;
    return 1;
}

// Both operands are fp16 subnormals (bytes XX as XX 2^-24), so an mma sum is
// x = n 2^-48 with an integer n < 2^23.  x + 2^-25 lies in [2^-25, 2^-24), where
// the spacing of fp32 numbers is 2^-48: its bit pattern is MAC_BIAS_BITS + n.
// The fold adds these patterns unmasked and starts every 64-bit column at
// minus the sum of the MAC_BIAS_BITS terms that land on it (fold_bias), so the
// columns end at the exact sums of the n with one add per accumulator.
constexpr float MAC_BIAS = 2.98023223876953125e-08f;  // 2^-25
constexpr uint32_t MAC_BIAS_BITS = 0x33000000u;

__device__ __forceinline__ uint32_t f32_bits(float x)
{
    return __float_as_uint(x + MAC_BIAS);
}

// the (compile-time) sum of the bias patterns that the fold adds to column c
// of slot u: the same shifts as the fold's, over every plane of D and tile of X
template <int SP, int NB>
__host__ __device__ constexpr uint64_t fold_bias(int u, int c)
{
    uint64_t s = 0;
    for (int a = 0; a < NB; a++)
        for (int nt = 0; nt < (NB * SP + 7) / 8; nt++)
            for (int h = 0; h < 2; h++) {
                const int uu = SP >= 8 ? (nt % (SP / 8)) * 2 + h : h;
                const int b = SP >= 8 ? nt / (SP / 8) : nt * 8 / SP;
                const int sh = 8 * (a + b);
                if (uu == u && (sh >> 5) == c) s += (uint64_t)MAC_BIAS_BITS << (sh & 31);
            }
    return s;
}

__device__ __forceinline__ void add128(acc128& t, uint64_t lo, uint64_t hi)
{
    const uint64_t l = t.lo + lo;
    t.hi += hi + (l < lo);
    t.lo = l;
}

__device__ __forceinline__ acc128 shfl_xor128(acc128 v, int m)
{
    return {__shfl_xor_sync(0xffffffffu, v.lo, m), __shfl_xor_sync(0xffffffffu, v.hi, m)};
}

// 128-bit sum -> residue: below q 2^64 for byte planes of at most 6 (the sums
// of one item stay below 16 KT q^2 with KT < 2^20 / (256 NB)), any value else
template <int NB>
__device__ __forceinline__ uint64_t reduce_sum(acc128 t, uint64_t q, uint64_t r0, uint64_t r1)
{
    return NB <= 6 ? barrett128(t.lo, t.hi, q, r0, r1) : reduce128(t.lo, t.hi, q, r0, r1);
}

// B builder body: tile tau's baby-step coefficients as mma B fragments of the
// X byte planes in the buffer Bt (one warp; padding stays as it was)
template <int S, int NB>
__device__ __forceinline__ void build_b(const MacArgs& A, uint8_t* Bt, uint32_t tau, uint32_t lane)
{
    constexpr int SP = 2 * S;
    constexpr int NT = (NB * SP + 7) / 8;
    const uint32_t gi = tau / A.tiles_per_limb, i = A.limb[gi];
    const uint32_t j0 = (tau % A.tiles_per_limb) * A.CT;
    // lane -> coefficient jj = lane % CT and a stride of 32 / CT over the
    // rows f = (s, term pair, p) of all sequences, U of them per batch of
    // loads; baby-step row r = (s terms + t) 2 + p lives at r nN, and
    // terms 2 tp, 2 tp + 1 share one fp16 pair per byte plane
    const uint32_t jj = lane % A.CT, rstep = 32 / A.CT, TP2 = ((A.terms + 1) >> 1) * 2;
    const uint64_t* col0 = A.baby + (size_t)i * A.N + j0 + jj;
    uint8_t* Bjj = Bt + (size_t)jj * A.jstride;
    if constexpr (S == 1) {
        // one sequence: rows (term pair, p) in batches of U loads
#pragma unroll
        for (int s = 0; s < S; s++) {
            constexpr int U = 12;
            for (uint32_t v0 = lane / A.CT; v0 < TP2; v0 += U * rstep) {
                uint2 w0[U], w1[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const uint32_t v = v0 + u * rstep, p = v & 1, t = (v >> 1) * 2;
                    const size_t r = ((size_t)s * A.terms + t) * 2 + p;
                    w0[u] = w1[u] = make_uint2(0, 0);
                    if (v < TP2) {
                        w0[u] = *reinterpret_cast<const uint2*>(col0 + r * A.nN);
                        if (t + 1 < A.terms) w1[u] = *reinterpret_cast<const uint2*>(col0 + (r + 2) * A.nN);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const uint32_t v = v0 + u * rstep;
                    if (v >= TP2) break;
                    const uint32_t p = v & 1, t = (v >> 1) * 2, sp = 2 * s + p, kr = t & 15;
                    uint8_t* base = Bjj + (size_t)(t >> 4) * NT * 256 + ((kr & 7) >> 1) * 8 + (kr >> 3) * 4;
#pragma unroll
                    for (int b = 0; b < NB; b++) {
                        const uint32_t x0 = b < 4 ? w0[u].x : w0[u].y, x1 = b < 4 ? w1[u].x : w1[u].y;
                        const uint32_t two = __byte_perm(x0, x1, (b & 3) | ((4 + (b & 3)) << 4));
                        const uint32_t col = b * SP + sp;  // two bytes as fp16 subnormals
                        *reinterpret_cast<uint32_t*>(base + (col >> 3) * 256 + (col & 7) * 32) =
                            __byte_perm(two, 0, 0x4140);
                    }
                }
            }
        }
    } else {
        // batches: the rows f = (s, term pair, p) of all sequences in
        // one index, so that a tile's loads go out in few batches
        auto next = [&](uint32_t& s, uint32_t& v) {  // f += rstep as (s, v)
            v += rstep;
            while (v >= TP2) {
                v -= TP2;
                s++;
            }
        };
        constexpr int U = 12;
        for (uint32_t f0 = lane / A.CT; f0 < S * TP2; f0 += U * rstep) {
            const uint32_t s0 = f0 / TP2, v0 = f0 - s0 * TP2;
            uint2 w0[U], w1[U];
            {
                uint32_t s = s0, v = v0;
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const uint32_t p = v & 1, t = (v >> 1) * 2;
                    const size_t r = ((size_t)s * A.terms + t) * 2 + p;
                    w0[u] = w1[u] = make_uint2(0, 0);
                    if (s < S) {
                        w0[u] = *reinterpret_cast<const uint2*>(col0 + r * A.nN);
                        if (t + 1 < A.terms) w1[u] = *reinterpret_cast<const uint2*>(col0 + (r + 2) * A.nN);
                    }
                    next(s, v);
                }
            }
            uint32_t s = s0, v = v0;
#pragma unroll
            for (int u = 0; u < U; u++, next(s, v)) {
                if (s >= S) break;
                const uint32_t p = v & 1, t = (v >> 1) * 2, sp = 2 * s + p, kr = t & 15;
                uint8_t* base = Bjj + (size_t)(t >> 4) * NT * 256 + ((kr & 7) >> 1) * 8 + (kr >> 3) * 4;
#pragma unroll
                for (int b = 0; b < NB; b++) {
                    const uint32_t x0 = b < 4 ? w0[u].x : w0[u].y, x1 = b < 4 ? w1[u].x : w1[u].y;
                    const uint32_t two = __byte_perm(x0, x1, (b & 3) | ((4 + (b & 3)) << 4));
                    const uint32_t col = b * SP + sp;  // two bytes as fp16 subnormals
                    *reinterpret_cast<uint32_t*>(base + (col >> 3) * 256 + (col & 7) * 32) =
                        __byte_perm(two, 0, 0x4140);
                }
            }
        }
    }
}

template <int S, int NB>
__global__ void __launch_bounds__(mac_threads(S)) k_cp_mac_tc(const __grid_constant__ MacArgs A)
{
    constexpr int SP = 2 * S;                 // (sequence, polynomial) columns per byte plane of X
    constexpr int NT = (NB * SP + 7) / 8;     // n8 tiles
    constexpr int SLOTS = SP >= 8 ? SP / 4 : 2;
    constexpr int AG = plane_group<NB, NT>();
    constexpr int MAC_CONSUMERS = mac_consumers(S), MAC_THREADS = mac_threads(S);
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t item_bytes = A.KT * NB * 256;
    const uint32_t IPT = A.CT * A.NEB;  // items (coefficient, output block) per tile
    const uint32_t R = A.R;
    const size_t bbuf = ((size_t)A.CT * A.jstride + 127) & ~(size_t)127;
    const uint32_t NBB = S == 1 ? 2 : A.nbb;  // one sequence: always two (the launcher's choice)
    const bool selfb = S > 1 && A.selfb != 0;  // then NBB = consumers, one private buffer each
    uint8_t* Bs = smem;  // NBB buffers of B fragments
    uint8_t* ring = smem + NBB * bbuf;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + (size_t)R * item_bytes);
    volatile uint32_t* abort = reinterpret_cast<volatile uint32_t*>(bars + 2 * R + 2 * MAC_MAX_BBUFS);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + R), bfull0 = smem_u32(bars + 2 * R),
                   bempty0 = smem_u32(bars + 2 * R + MAC_MAX_BBUFS), ring0 = smem_u32(ring);

    // B padding (terms beyond the last term, columns beyond NB SP) stays zero
    for (uint32_t x = threadIdx.x; x < NBB * bbuf / 16; x += MAC_THREADS)
        reinterpret_cast<uint4*>(Bs)[x] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        for (uint32_t r = 0; r < R; r++) {
            mbar_init(full0 + 8 * r, 1);
            mbar_init(empty0 + 8 * r, 1);
        }
        for (uint32_t r = 0; r < NBB; r++) {
            mbar_init(bfull0 + 8 * r, 1);
            mbar_init(bempty0 + 8 * r, MAC_CONSUMERS);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == MAC_CONSUMERS + 1) {
        if (selfb) return;
        // ---- B builder: per tile, X's byte planes as mma B fragments, up to
        // NBB - 1 tiles ahead of the consumers
        for (uint32_t lt = 0, tau = blockIdx.x; tau < A.tiles; lt++, tau += gridDim.x) {
            const uint32_t buf = lt % NBB;
            // the lanes leave together (one lane's wait may expire as another's succeeds)
            if (lt >= NBB && !__all_sync(0xffffffffu, mbar_wait(bempty0 + 8 * buf, ((lt / NBB) - 1) & 1, abort, A.wait_ns)))
                break;
            build_b<S, NB>(A, Bs + buf * bbuf, tau, lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(bfull0 + 8 * buf);
        }
        if (lane == 0 && *abort) atomicExch(A.status, 1u);
        return;
    }
    if (warp == MAC_CONSUMERS) {
        // ---- streamer (lane 0): each tile's contiguous plaintext range into the ring
        if (lane == 0) {
            uint32_t issued = 0;
            for (uint32_t lt = 0, tau = blockIdx.x; !A.withhold && tau < A.tiles && !*abort; lt++, tau += gridDim.x) {
                const uint32_t gi = tau / A.tiles_per_limb, j0 = (tau % A.tiles_per_limb) * A.CT;
                const uint8_t* src = A.ptb + A.off[gi] + (size_t)j0 * A.NEB * item_bytes;
                for (uint32_t it = 0; it < IPT; it++) {
                    const uint32_t kg = lt * IPT + it, st = kg % R;
                    if (kg >= R && !mbar_wait(empty0 + 8 * st, ((kg / R) - 1) & 1, abort, A.wait_ns)) break;
                    mbar_expect_tx(full0 + 8 * st, item_bytes);
                    bulk_g2s(ring0 + st * item_bytes, src + (size_t)it * item_bytes, item_bytes, full0 + 8 * st);
                    issued = kg + 1;
                }
            }
            // shared memory must outlive every copy started here: wait for them
            // even after an abort (the copies land whatever the consumers do)
            for (uint32_t kg = issued > R ? issued - R : 0; kg < issued; kg++) {
                uint32_t dummy = 0;
                mbar_wait(full0 + 8 * (kg % R), (kg / R) & 1, &dummy, MAC_WAIT_NS);
            }
            if (*abort) atomicExch(A.status, 1u);
        }
        return;
    }

    // ---- consumer warps: item kg (global within the CTA) goes to warp kg % W
    const uint32_t g8 = lane >> 2, h4 = lane & 3;
    const uint32_t lane_b = SP >= 8 ? 0 : (2 * h4) / SP;  // byte plane offset of this lane's columns
    for (uint32_t lt = 0, tau = blockIdx.x; tau < A.tiles; lt++, tau += gridDim.x) {
        // building its own B, a consumer visits only the tiles whose single
        // item is its own
        if (selfb && lt % MAC_CONSUMERS != warp) continue;
        const uint32_t buf = lt % NBB, gi = tau / A.tiles_per_limb, i = A.limb[gi];
        const uint32_t j0 = (tau % A.tiles_per_limb) * A.CT;
        const uint64_t q = A.q[i], r0 = A.bar[2 * i], r1 = A.bar[2 * i + 1];
        if (selfb) {
            build_b<S, NB>(A, Bs + warp * bbuf, tau, lane);
            __syncwarp();
        } else if (!__all_sync(0xffffffffu, mbar_wait(bfull0 + 8 * buf, (lt / NBB) & 1, abort, A.wait_ns))) {
            break;
        }
        const uint8_t* Bt = Bs + (selfb ? warp : buf) * bbuf + lane * 8;
        uint32_t it = (warp + MAC_CONSUMERS - (lt * IPT) % MAC_CONSUMERS) % MAC_CONSUMERS;
        bool ok = true;
        for (; it < IPT; it += MAC_CONSUMERS) {
            const uint32_t kg = lt * IPT + it, st = kg % R;
            if (!__all_sync(0xffffffffu, mbar_wait(full0 + 8 * st, (kg / R) & 1, abort, A.wait_ns))) {
                ok = false;
                break;
            }
            const uint32_t jj = it / A.NEB, eblk = it % A.NEB;
            const uint8_t* As = ring + (size_t)st * item_bytes + lane * 8;
            const uint8_t* Bj = Bt + (size_t)jj * A.jstride;
            // 128-bit sums over the segments: raw for byte planes of at most
            // 6, segment residues above
            acc128 fin[2][SLOTS];
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int u = 0; u < SLOTS; u++) fin[r][u] = {0, 0};
            for (uint32_t ks = 0; ks < A.KT; ks += A.kseg) {
                const uint32_t ke = min(A.KT, ks + A.kseg);
                const bool last_seg = ke == A.KT;
                // 32-bit columns of the 128-bit sums: col c holds weight 2^{32 c}
                uint64_t col[2][SLOTS][4];
#pragma unroll
                for (int r = 0; r < 2; r++)
#pragma unroll
                    for (int u = 0; u < SLOTS; u++)
#pragma unroll
                        for (int c = 0; c < 4; c++) col[r][u][c] = 0 - fold_bias<SP, NB>(u, c);
#pragma unroll
                for (int a0 = 0; a0 < NB; a0 += AG) {
                    float acc[AG][NT][4];
#pragma unroll
                    for (int a = 0; a < AG; a++)
#pragma unroll
                        for (int nt = 0; nt < NT; nt++)
#pragma unroll
                            for (int e = 0; e < 4; e++) acc[a][nt][e] = 0.f;
                    for (uint32_t kt = ks; kt < ke; kt++) {
                        const uint8_t* Bk = Bj + (size_t)kt * NT * 256;
                        if (AG > 1) {  // B fragments reused by every plane of the group
                            uint2 bf[NT];
#pragma unroll
                            for (int nt = 0; nt < NT; nt++) bf[nt] = *reinterpret_cast<const uint2*>(Bk + nt * 256);
#pragma unroll
                            for (int a = 0; a < AG; a++) {
                                uint32_t af[4];
                                bytes_to_f16x2(*reinterpret_cast<const uint2*>(As + (size_t)(kt * NB + a0 + a) * 256),
                                               af);
#pragma unroll
                                for (int nt = 0; nt < NT; nt++) mma16816(acc[a][nt], af, bf[nt]);
                            }
                        } else {
                            uint32_t af[4];
                            bytes_to_f16x2(*reinterpret_cast<const uint2*>(As + (size_t)(kt * NB + a0) * 256), af);
#pragma unroll
                            for (int nt = 0; nt < NT; nt++)
                                mma16816(acc[0][nt], af, *reinterpret_cast<const uint2*>(Bk + nt * 256));
                        }
                    }
                    if (a0 + AG >= NB && last_seg) {  // last read of the stage: hand it back
                        __syncwarp();
                        if (lane == 0) mbar_arrive(empty0 + 8 * st);
                    }
                    // fold: column 8 nt + 2 h4 + (e & 1) of the n8 tile is byte plane
                    // b = b_ct(nt) + lane_b of (sequence, polynomial) slot; rows g8, g8 + 8
#pragma unroll
                    for (int a = 0; a < AG; a++)
#pragma unroll
                        for (int nt = 0; nt < NT; nt++)
#pragma unroll
                            for (int e = 0; e < 4; e++) {
                                const int r = e >> 1, h = e & 1;
                                const int u = SP >= 8 ? (nt % (SP / 8)) * 2 + h : h;
                                const int b = SP >= 8 ? nt / (SP / 8) : nt * 8 / SP;
                                const int sh = 8 * (a0 + a + b);
                                col[r][u][sh >> 5] += (uint64_t)f32_bits(acc[a][nt][e]) << (sh & 31);
                            }
                }
#pragma unroll
                for (int r = 0; r < 2; r++)
#pragma unroll
                    for (int u = 0; u < SLOTS; u++) {
                        uint64_t lo = col[r][u][0] + (col[r][u][1] << 32);
                        uint64_t hi = (col[r][u][1] >> 32) + col[r][u][2] + (col[r][u][3] << 32) + (lo < col[r][u][0]);
                        if (SP < 8 && lane_b) {  // this lane's planes start at b = lane_b
                            const uint32_t sh = 8 * lane_b;
                            hi = (hi << sh) | (lo >> (64 - sh));
                            lo <<= sh;
                        }
                        if (NB <= 6) add128(fin[r][u], lo, hi);
                        else add128(fin[r][u], reduce128(lo, hi, q, r0, r1), 0);
                    }
            }
            const size_t jcol = (size_t)i * A.N + j0 + jj;
            auto store = [&](uint32_t row, uint32_t sp, uint64_t v) {
                const uint32_t eg = eblk * 16 + row;
                if (eg < A.neg) A.T[((size_t)((sp >> 1) * A.neg + eg) * 2 + (sp & 1)) * A.nN + jcol] = v;
            };
            if (SP < 8) {
                // the other lanes of the quad hold other byte planes of the same
                // sums: a transposing reduction leaves each lane the sums it
                // stores, so each of them is reduced once.  Lanes h4, h4 ^ 2
                // exchange rows (keep row half r = h4 >> 1) ...
                const bool rhi = h4 & 2;
                acc128 k[2];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    k[u] = rhi ? fin[1][u] : fin[0][u];
                    const acc128 o = shfl_xor128(rhi ? fin[0][u] : fin[1][u], 2);
                    add128(k[u], o.lo, o.hi);
                }
                const uint32_t row = g8 + 8 * (h4 >> 1);
                if (SP == 2) {
                    // ... and for one sequence lanes h4, h4 ^ 1 hold the other
                    // planes too: exchange polynomials (keep p = h4 & 1)
                    const bool phi = h4 & 1;
                    acc128 w = phi ? k[1] : k[0];
                    const acc128 o = shfl_xor128(phi ? k[0] : k[1], 1);
                    add128(w, o.lo, o.hi);
                    store(row, h4 & 1, reduce_sum<NB>(w, q, r0, r1));
                } else {
#pragma unroll
                    for (int h = 0; h < 2; h++) store(row, 2 * (h4 & 1) + h, reduce_sum<NB>(k[h], q, r0, r1));
                }
            } else {
#pragma unroll
                for (int r = 0; r < 2; r++)
#pragma unroll
                    for (int u = 0; u < SLOTS; u++)
                        store(g8 + 8 * r, 8 * (u >> 1) + 2 * h4 + (u & 1), reduce_sum<NB>(fin[r][u], q, r0, r1));
            }
        }
        if (!ok) break;
        __syncwarp();  // (self-built B: every lane's reads end before the next build)
        if (!selfb && lane == 0) mbar_arrive(bempty0 + 8 * buf);
    }
    if (lane == 0 && *abort) atomicExch(A.status, 1u);
}

// one thread per 8-byte fragment word of one output block: ((j KT + kt) nb + a) 32 + lane
__global__ void k_cp_bytes(uint8_t* __restrict__ dst, const uint64_t* __restrict__ src, uint32_t i, uint32_t N,
                           uint64_t nN, uint32_t terms, uint32_t rows, uint32_t KT, uint32_t NEB, uint32_t nb,
                           uint32_t eblk)
{
    const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (uint64_t)N * KT * nb * 32) return;
    const uint32_t lane = idx & 31;
    uint64_t r = idx >> 5;
    const uint32_t a = r % nb;
    r /= nb;
    const uint32_t kt = r % KT, j = (uint32_t)(r / KT);
    const uint32_t g = lane >> 2, h = lane & 3;
    uint64_t out = 0;
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const uint32_t row = g + 8 * ((e >> 1) & 1), t = kt * 16 + 2 * h + (e & 1) + 8 * (e >> 2);
        if (row < rows && t < terms)
            out |= ((src[((size_t)row * terms + t) * nN + (size_t)i * N + j] >> (8 * a)) & 0xFFull) << (8 * e);
    }
    *reinterpret_cast<uint64_t*>(dst + ((((size_t)j * NEB + eblk) * KT + kt) * nb + a) * 256 + lane * 8) = out;
}

template <int S, int NB>
int launch_group(blb_ctx* c, MacArgs& a, uint32_t nlimbs)
{
    constexpr int SP = 2 * S, NT = (NB * SP + 7) / 8;
    const uint32_t item_bytes = a.KT * NB * 256;
    a.jstride = a.KT * NT * 256 + 16;
    a.CT = 16;
    while (a.CT > 1 && (size_t)a.CT * a.jstride > MAC_BBUF_BYTES) a.CT >>= 1;
    // batches: widen tiles towards four coefficients (one 32-byte sector of
    // every baby-step row per load) while two B buffers and the ring still fit
    // two CTAs per SM
    while (S > 1 && a.CT < 4 &&
           2 * (((size_t)2 * a.CT * a.jstride + 127) & ~(size_t)127) + (size_t)mac_consumers(S) * item_bytes +
                   16 * (mac_consumers(S) + MAC_MAX_BBUFS) + 16 <= (113u << 10))
        a.CT <<= 1;
    a.tiles_per_limb = c->N / a.CT;
    a.tiles = a.tiles_per_limb * nlimbs;
    // one ring stage per consumer: the fills of a stage all go to the same
    // warp, so a parity wait never sees the phase before the one it wants
    constexpr int W = mac_consumers(S);
    const size_t bbuf = ((size_t)a.CT * a.jstride + 127) & ~(size_t)127;
    a.R = W;
    // B buffers: two, and for batches whose tiles hold fewer items than there
    // are consumers, as many more (up to MAC_MAX_BBUFS) as keep two CTAs per SM
    // in shared memory, so that every consumer has a tile to work on
    const auto smem_for = [&](uint32_t nbb) {
        return nbb * bbuf + (size_t)a.R * item_bytes + 16 * (a.R + MAC_MAX_BBUFS) + 16;
    };
    // tiles of a single item (batches whose coefficient fills a B buffer):
    // each consumer builds its tile's B itself, in a buffer of its own, when
    // those fit two CTAs per SM; the builder warp alone could not keep four
    // consumers busy
    a.nbb = 2;
    a.selfb = S > 1 && a.CT * a.NEB == 1 && W <= (int)MAC_MAX_BBUFS && smem_for(W) <= (113u << 10);
    if (a.selfb) a.nbb = W;
    while (!a.selfb && S > 1 && a.nbb < MAC_MAX_BBUFS && (size_t)a.CT * a.NEB * a.nbb < (size_t)W &&
           smem_for(a.nbb + 1) <= (113u << 10))
        a.nbb++;
    const size_t smem = smem_for(a.nbb);
    if (smem > (227u << 10)) return blb_fail(BLB_ERR_ARG, "plaintext tile too large for shared memory");
    if (item_bytes >= (1u << 20)) return blb_fail(BLB_ERR_ARG, "too many plaintext terms per output");
    // the shared-memory opt-in is a property of each device
    static std::atomic<bool> attr[64];
    int per_sm = 0, dev = 0, sms = 0;
    BLB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return blb_fail(BLB_ERR_ARG, "device ordinal beyond 64");
    if (!attr[dev].load()) {
        BLB_CUDA(cudaFuncSetAttribute(k_cp_mac_tc<S, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 << 10));
        attr[dev].store(true);
    }
    BLB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cp_mac_tc<S, NB>, mac_threads(S), smem));
    BLB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint32_t grid = std::min<uint32_t>(a.tiles, (uint32_t)std::max(1, per_sm) * sms);
    k_cp_mac_tc<S, NB><<<grid, mac_threads(S), smem, c->stream>>>(a);
    BLB_LAUNCHED();
    return BLB_OK;
}

template <int S>
int launch_nb(blb_ctx* c, MacArgs& a, uint32_t nb, uint32_t nlimbs)
{
    switch (nb) {
    case 3: return launch_group<S, 3>(c, a, nlimbs);
    case 4: return launch_group<S, 4>(c, a, nlimbs);
    case 5: return launch_group<S, 5>(c, a, nlimbs);
    case 6: return launch_group<S, 6>(c, a, nlimbs);
    case 7: return launch_group<S, 7>(c, a, nlimbs);
    case 8: return launch_group<S, 8>(c, a, nlimbs);
    default: return blb_fail(BLB_ERR_PARAM, "prime size outside 17..64 bits for the tensor-core product");
    }
}

}  // namespace

uint32_t cp_word_bytes(uint64_t q)
{
    uint32_t bits = 64 - __builtin_clzll(q);
    return (bits + 7) / 8;
}

int cp_plan_layout(blb_ctx* c, blb_cp_plan* P)
{
    const uint32_t n = P->level + 1;
    P->KT = (P->nX * P->b1 + 15) / 16;
    P->NEB = (P->nY * P->G + 15) / 16;
    P->nb.assign(n, 0);
    P->off.assign(n, 0);
    uint64_t off = 0;
    for (uint32_t i = 0; i < n; i++) {
        P->nb[i] = (uint8_t)cp_word_bytes(c->q[i]);
        if (P->nb[i] < 3) return blb_fail(BLB_ERR_PARAM, "primes below 2^17 are not supported by matmul_cp");
        P->off[i] = off;
        off += (uint64_t)c->N * P->NEB * P->KT * P->nb[i] * 256;
    }
    P->bytes = off;
    return BLB_OK;
}

int cp_plan_store_block(blb_ctx* c, blb_cp_plan* P, const uint64_t* src, uint32_t eblk)
{
    const uint32_t n = P->level + 1, terms = P->nX * P->b1, neg = P->nY * P->G;
    const uint32_t rows = std::min<uint32_t>(16, neg - eblk * 16);
    for (uint32_t i = 0; i < n; i++) {
        const uint64_t total = (uint64_t)c->N * P->KT * P->nb[i] * 32;
        k_cp_bytes<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(P->d_ptb + P->off[i], src, i, c->N,
                                                                         (uint64_t)n * c->N, terms, rows, P->KT,
                                                                         P->NEB, P->nb[i], eblk);
        BLB_LAUNCHED();
    }
    return BLB_OK;
}

// baby: [S][nX][b1] ciphertexts; T: [S][nY][G] ciphertexts (level of the plan)
int launch_cp_mac(blb_ctx* c, const blb_cp_plan* P, const uint64_t* baby, uint64_t* T, uint32_t S)
{
    const uint32_t n = P->level + 1, N = c->N;
    const uint64_t terms = (uint64_t)P->nX * P->b1, neg = (uint64_t)P->nY * P->G;
    // algorithmic bytes: the byte-sliced plaintexts once, the baby-step
    // ciphertexts once, the (e, g) partial sums written once
    ProfScope prof(c, "cp_mac", P->bytes + (S * terms * 2 * n + S * neg * 2 * n) * N * 8);
    // batches: the tcgen05 kernel when chosen (blb_ctx_set_batch_mac) or, by
    // default, for 8 sequences and a single 16-output block, where it measured
    // faster on the B300 (wider plans and smaller batches: the mma.sync
    // kernel); its operands must fit shared memory
    if (S > 1 && (c->batch_mac == 2 || (c->batch_mac == 0 && S == 8 && P->NEB == 1))) {
        bool used = false;
        BLB_TRY(launch_cp_mac_umma(c, P, baby, T, S, &used));
        if (used) return BLB_OK;
    }
    MacArgs a{};
    a.T = T;
    a.baby = baby;
    a.ptb = P->d_ptb;
    a.q = c->d_q;
    a.bar = c->d_bar;
    a.status = c->d_status;
    a.wait_ns = c->wait_ns ? c->wait_ns : MAC_WAIT_NS;
    a.withhold = c->mac_withhold;
    a.nN = (uint64_t)n * N;
    a.seq_words = terms * 2 * a.nN;
    a.N = N;
    a.terms = (uint32_t)terms;
    a.KT = P->KT;
    a.neg = (uint32_t)neg;
    a.NEB = P->NEB;
    // limbs grouped by bytes per word, one launch per group
    for (uint32_t nb = 3; nb <= 8; nb++) {
        uint32_t cnt = 0;
        bool big = false;
        for (uint32_t i = 0; i < n; i++)
            if (P->nb[i] == nb) {
                if (cnt == MAC_MAX_GROUP) return blb_fail(BLB_ERR_PARAM, "too many limbs");
                a.limb[cnt] = i;
                a.off[cnt] = P->off[i];
                big |= c->q[i] >= (1ull << 60);
                cnt++;
            }
        if (!cnt) continue;
        // 8 tiles keep 8 x 16 x 255^2 < 2^23 (exact fp32 sums, read back by one
        // add); primes above 2^60 need 64 terms x q^2 < 2^128
        a.kseg = big ? 4 : 8;
        int rc;
        switch (S) {
        case 1: rc = launch_nb<1>(c, a, nb, cnt); break;
        case 2: rc = launch_nb<2>(c, a, nb, cnt); break;
        case 4: rc = launch_nb<4>(c, a, nb, cnt); break;
        case 8: rc = launch_nb<8>(c, a, nb, cnt); break;
        default: return blb_fail(BLB_ERR_ARG, "batch of sequences must be 1, 2, 4 or 8 per MAC launch");
        }
        if (rc) return rc;
    }
    return BLB_OK;
}
