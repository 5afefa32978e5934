// ntt.cu -- batched negacyclic NTT / inverse NTT over 64-bit primes.
//
// Forward: Cooley-Tukey butterflies with psi powers in bit-reversed order,
// natural-order input, output A[k] = a(psi^(2 bitrev(k) + 1)).  Inverse:
// Gentleman-Sande butterflies with psi^-1 powers, then N^-1.  For the element
// with global index j at the lower end of a butterfly:
//   forward stage s (2^s groups):        twiddle index 2^s + (j >> (logN - s))
//   inverse, butterfly distance 2^lt:    twiddle index (N + j) >> (lt + 1)
//
// N > 4096 is split N = N1 * N2 into two passes over 4096-word tiles held in
// shared memory: the "column" pass runs the log2(N1) stages whose butterflies
// pair elements N2 or more apart on sub-transforms {c + N2 r}, the "row" pass
// runs the remaining stages on contiguous blocks of N2.  Every pass reads and
// writes each word once.  Inside a pass each thread holds a group of up to 8
// elements in registers and runs up to 3 stages on it (radix 8); the first
// round loads its groups from global memory and the last stores them, so a
// pass of two or three rounds makes one or two shared-memory round trips
// instead of one per stage; radix 8 fits
// 64 registers, so four CTAs run per SM (measured on the B300 against radix 16
// at three CTAs and radix 8 at three or five).  Shared memory is padded by one
// word every 16 to keep strided group accesses conflict-free.
//
// Each (transform size, pass) is its own template instance, so every index,
// shift and loop bound of a pass is a compile-time constant; the twiddles are
// stored as (w, floor(w 2^64 / q)) pairs and read with one 16-byte load.
//
// Reduction: for primes q >= 2^(63 - logN) the butterflies reduce lazily
// (Harvey): forward values stay in [0, 4q), inverse values in [0, 2q).  For
// smaller primes no butterfly needs a conditional subtraction: forward values
// grow by at most 4q per stage (their products use a cheaper quotient
// estimate, within [0, 4q)), inverse sums at most double per stage, and both
// stay below 2^64 ((1 + 4 logN) q < 2^64); the last pass reduces once.
//
// Every pass is launched with programmatic stream serialization and starts
// with pdl_begin, so it can be scheduled while the previous kernel drains.
//
// Rows: either rows 0..rows-1 of `data` with prime map.p[row % map.n], or an
// explicit row list (entry = row index | prime index << 24) so that a batch can
// transform exactly the rows it needs in one launch.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr uint32_t kThreads = 256;
constexpr uint32_t kMaxGridY = 65535;

__device__ __forceinline__ uint32_t padi(uint32_t e) { return e + (e >> 4); }

__device__ __forceinline__ void row_of(const uint32_t* rowlist, const LimbMap& map, uint32_t y, uint32_t& row,
                                       uint32_t& pi)
{
    if (rowlist) {
        uint32_t e = rowlist[y];
        row = e & 0xFFFFFFu;
        pi = e >> 24;
    } else {
        row = y;
        pi = map.p[y % map.n];
    }
}

// Shoup product without the final correction: result in [0, 2q) for any x.
__device__ __forceinline__ uint64_t mul_shoup_lazy(uint64_t x, uint64_t w, uint64_t wp, uint64_t q)
{
    return x * w - __umul64hi(x, wp) * q;
}

// forward, lazy: X, Y in [0, 4q) -> X + WY, X - WY in [0, 4q)
__device__ __forceinline__ void bfly_fwd(uint64_t& X, uint64_t& Y, ulonglong2 w, uint64_t q, uint64_t q2)
{
    const uint64_t x = X >= q2 ? X - q2 : X;
    const uint64_t t = mul_shoup_lazy(Y, w.x, w.y, q);
    X = x + t;
    Y = x + q2 - t;
}

// Shoup product with the quotient estimate from the three high 32 x 32-bit
// partial products of Y wp (the low one and the low halves of the middle two
// dropped): the estimate is at most 2 below floor(Y wp / 2^64), so the result
// is in [0, 4q) for any 64-bit Y.
__device__ __forceinline__ uint64_t mul_shoup_lazy4(uint64_t x, uint64_t w, uint64_t wp, uint64_t q)
{
    const uint32_t xl = (uint32_t)x, xh = (uint32_t)(x >> 32), pl = (uint32_t)wp, ph = (uint32_t)(wp >> 32);
    const uint64_t qt = (uint64_t)xh * ph + __umulhi(xh, pl) + __umulhi(xl, ph);
    return x * w - qt * q;
}

// forward, small prime: X + t, X - t + 4q with t = W Y in [0, 4q), no reduction
// (values grow by at most 4q per stage)
__device__ __forceinline__ void bfly_fwd_s(uint64_t& X, uint64_t& Y, ulonglong2 w, uint64_t q, uint64_t q2)
{
    const uint64_t t = mul_shoup_lazy4(Y, w.x, w.y, q);
    const uint64_t x = X;
    X = x + t;
    Y = x + 2 * q2 - t;
}

// inverse, lazy: X, Y in [0, 2q) -> X + Y, W (X - Y) in [0, 2q)
__device__ __forceinline__ void bfly_inv(uint64_t& X, uint64_t& Y, ulonglong2 w, uint64_t q, uint64_t q2)
{
    uint64_t s = X + Y;
    s = s >= q2 ? s - q2 : s;
    const uint64_t d = X - Y + q2;
    X = s;
    Y = mul_shoup_lazy(d, w.x, w.y, q);
}

// inverse, small prime, stage inputs below C = 2^(lt+1) q: X + Y, W (X - Y + C)
// with the cheaper quotient estimate (in [0, 4q), still below 2^(lt+2) q, the
// next stage's bound, for every stage lt >= 0)
__device__ __forceinline__ void bfly_inv_s(uint64_t& X, uint64_t& Y, ulonglong2 w, uint64_t q, uint64_t C)
{
    const uint64_t x = X, y = Y;
    X = x + y;
    Y = mul_shoup_lazy4(x + C - y, w.x, w.y, q);
}

__device__ __forceinline__ bool small_prime(uint64_t q, uint32_t logN) { return q < (1ull << (63 - logN)); }

// Geometry of one pass: transform size 2^LOGN, sub-transform length 2^LP,
// column (COLS) or row pass.
template <int LOGN, int LP, bool COLS>
struct Geo {
    static constexpr uint32_t N = 1u << LOGN;
    static constexpr int LOGTILE = LOGN < 12 ? LOGN : 12;
    static constexpr uint32_t TILE = 1u << LOGTILE;
    static constexpr int LOGNSUB = LOGTILE - LP;  // sub-transforms per tile
    static constexpr uint32_t NSUB = 1u << LOGNSUB;
    static constexpr int GOFF = COLS ? LOGN - LP : 0;  // global bit of local bit 0
    static constexpr int LOGN2 = LOGN - LP;
};

// Finishing step of the transform's last pass (applied as the results are
// stored): the inverse multiplies by N^-1 (or the given factor), both reduce
// to [0, q)
struct Fin {
    uint64_t ni, nis, r1;
    bool small;
};

template <bool INV, bool LAST>
__device__ __forceinline__ uint64_t finish_value(uint64_t v, const Fin& f, uint64_t q, uint64_t q2)
{
    if (!LAST) return v;
    if (INV) v = mul_shoup_lazy(v, f.ni, f.nis, q);
    else if (f.small) v = v - __umul64hi(v, f.r1) * q;  // any 64-bit v -> [0, 2q)
    else v = v >= q2 ? v - q2 : v;
    return v >= q ? v - q : v;
}

// The row's part of a fused rescale (RescaleIO): where its lift comes from and
// where its result goes.
struct RsRow {
    const uint64_t* last;
    const uint64_t* in;
    uint64_t* out;
    uint64_t ql, rb, inv, inv_sh;
    // gather (GatherIO): the source's c1 row, its Galois element, the digit row
    const uint64_t* c1;
    uint64_t g;
    uint64_t* ext;
};

// the centered lift of v (a residue mod ql) reduced mod q, in [0, q)
__device__ __forceinline__ uint64_t lift_mod(uint64_t v, uint64_t ql, uint64_t q, uint64_t rb)
{
    if (v > ql / 2) {
        const uint64_t m = ql - v;
        const uint64_t r = m - __umul64hi(m, rb) * q;
        const uint64_t mr = r >= q ? r - q : r;
        return mr ? q - mr : 0;
    }
    const uint64_t r = v - __umul64hi(v, rb) * q;
    return r >= q ? r - q : r;
}

// global position (within the row) of tile element e
template <int LOGN, int LP, bool COLS>
__device__ __forceinline__ size_t tile_pos(uint32_t e, uint32_t c0)
{
    using G_ = Geo<LOGN, LP, COLS>;
    if (COLS) return ((size_t)(e >> G_::LOGNSUB) << G_::LOGN2) + c0 + (e & (G_::NSUB - 1));
    return ((size_t)c0 << LP) + e;
}

// One round: R stages on groups of 2^R elements whose local indices differ in
// bits [PLO, PLO + R).  The pass's first round reads its groups from the row
// in global memory (FROM_G) and its last round writes them back, finished
// (TO_G); the rounds between go through the tile in shared memory.
// RSL: the first round of a fused rescale's first pass (loads the lift of the
// last limb); RSS: the last round of its last pass (stores the rescaled limb);
// GL: the first round of a fused gather's first pass (loads the permuted source
// and writes it to the extended digit too).
template <int LOGN, int LP, bool COLS, bool INV, bool SMALL, int PLO, int R, bool FROM_G, bool TO_G, bool LAST,
          bool RSL = false, bool RSS = false, bool GL = false>
__device__ __forceinline__ void round(uint64_t* sm, uint64_t* __restrict__ a, uint32_t c0,
                                      const ulonglong2* __restrict__ W, uint64_t q, uint64_t q2, const Fin& fin,
                                      const RsRow& rr)
{
    using G_ = Geo<LOGN, LP, COLS>;
    constexpr uint32_t K = 1u << R;
    constexpr uint32_t GROUPS = G_::TILE >> R;
    constexpr int JSHIFT = G_::GOFF + PLO;
    constexpr uint32_t e_stride = COLS ? (G_::NSUB << PLO) : (1u << PLO);
#pragma unroll
    for (uint32_t G = threadIdx.x; G < GROUPS; G += kThreads) {
        uint32_t sub, g;
        if (COLS) {
            sub = G & (G_::NSUB - 1);
            g = G >> G_::LOGNSUB;
        } else {
            g = G & ((1u << (LP - R)) - 1);
            sub = G >> (LP - R);
        }
        const uint32_t base_r = ((g >> PLO) << (PLO + R)) | (g & ((1u << PLO) - 1));
        uint32_t e_base, j_base;
        if (COLS) {
            e_base = (base_r << G_::LOGNSUB) + sub;
            j_base = c0 + sub + (base_r << G_::GOFF);
        } else {
            e_base = (sub << LP) + base_r;
            j_base = ((c0 + sub) << LP) + base_r;
        }
        uint64_t x[K];
#pragma unroll
        for (uint32_t k = 0; k < K; k++) {
            const uint32_t e = e_base + k * e_stride;
            if (RSL) {
                x[k] = lift_mod(rr.last[tile_pos<LOGN, LP, COLS>(e, c0)], rr.ql, q, rr.rb);
            } else if (GL) {
                const uint32_t pos = (uint32_t)tile_pos<LOGN, LP, COLS>(e, c0);
                x[k] = rr.c1[perm_index(pos, LOGN, rr.g)];
                rr.ext[pos] = x[k];
            } else {
                x[k] = FROM_G ? a[tile_pos<LOGN, LP, COLS>(e, c0)] : sm[padi(e)];
            }
        }
        // The butterflied bits of base_r are zero, so for the pair (k, k | 2^u)
        // the lower element's twiddle index splits into a per-stage base plus
        // k >> (u + 1): stage u uses 2^(R-1-u) distinct twiddles.
        if (!INV) {
#pragma unroll
            for (int u = R - 1; u >= 0; u--) {
                const uint32_t s = LOGN - 1 - (JSHIFT + u);
                const uint32_t wbase = (1u << s) + (j_base >> (JSHIFT + u + 1));
#pragma unroll
                for (uint32_t h = 0; h < (K >> (u + 1)); h++) {
                    const ulonglong2 w = W[wbase + h];
#pragma unroll
                    for (uint32_t lo = 0; lo < (1u << u); lo++) {
                        const uint32_t k = (h << (u + 1)) | lo;
                        if (SMALL) bfly_fwd_s(x[k], x[k | (1u << u)], w, q, q2);
                        else bfly_fwd(x[k], x[k | (1u << u)], w, q, q2);
                    }
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < R; u++) {
                const uint32_t wbase = (G_::N + j_base) >> (JSHIFT + u + 1);
                const uint64_t C = q << (JSHIFT + u + 1);  // inputs of stage lt lie below 2^(lt+1) q
#pragma unroll
                for (uint32_t h = 0; h < (K >> (u + 1)); h++) {
                    const ulonglong2 w = W[wbase + h];
#pragma unroll
                    for (uint32_t lo = 0; lo < (1u << u); lo++) {
                        const uint32_t k = (h << (u + 1)) | lo;
                        if (SMALL) bfly_inv_s(x[k], x[k | (1u << u)], w, q, C);
                        else bfly_inv(x[k], x[k | (1u << u)], w, q, q2);
                    }
                }
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < K; k++) {
            const uint32_t e = e_base + k * e_stride;
            if (RSS) {
                const size_t pos = tile_pos<LOGN, LP, COLS>(e, c0);
                const uint64_t t = finish_value<INV, LAST>(x[k], fin, q, q2);
                rr.out[pos] = mul_shoup(sub_mod(rr.in[pos], t, q), rr.inv, rr.inv_sh, q);
            } else if (TO_G) {
                a[tile_pos<LOGN, LP, COLS>(e, c0)] = finish_value<INV, LAST>(x[k], fin, q, q2);
            } else {
                sm[padi(e)] = x[k];
            }
        }
    }
}

// forward rounds: local bits from the top down, up to RB stages per round
// (radix 2^RB); the first reads the row, the last writes it
template <int LOGN, int LP, bool COLS, bool SMALL, int PHI, int RB, bool LAST, bool RSL = false, bool RSS = false>
__device__ __forceinline__ void fwd_rounds(uint64_t* sm, uint64_t* a, uint32_t c0, const ulonglong2* W, uint64_t q,
                                           uint64_t q2, const Fin& fin, const RsRow& rr)
{
    if constexpr (PHI > 0) {
        constexpr int R = PHI >= RB ? RB : PHI;
        round<LOGN, LP, COLS, false, SMALL, PHI - R, R, PHI == LP, PHI - R == 0, LAST, RSL && PHI == LP,
              RSS && PHI - R == 0>(sm, a, c0, W, q, q2, fin, rr);
        if constexpr (PHI - R > 0) __syncthreads();
        fwd_rounds<LOGN, LP, COLS, SMALL, PHI - R, RB, LAST, RSL, RSS>(sm, a, c0, W, q, q2, fin, rr);
    }
}

// inverse rounds: local bits from the bottom up
template <int LOGN, int LP, bool COLS, bool SMALL, int PLO, int RB, bool LAST, bool GL = false>
__device__ __forceinline__ void inv_rounds(uint64_t* sm, uint64_t* a, uint32_t c0, const ulonglong2* W, uint64_t q,
                                           uint64_t q2, const Fin& fin, const RsRow& rr)
{
    if constexpr (PLO < LP) {
        constexpr int R = LP - PLO >= RB ? RB : LP - PLO;
        round<LOGN, LP, COLS, true, SMALL, PLO, R, PLO == 0, PLO + R == LP, LAST, false, false, GL && PLO == 0>(
            sm, a, c0, W, q, q2, fin, rr);
        if constexpr (PLO + R < LP) __syncthreads();
        inv_rounds<LOGN, LP, COLS, SMALL, PLO + R, RB, LAST, GL>(sm, a, c0, W, q, q2, fin, rr);
    }
}

// CTAs per SM for a radix: 16 needs the registers of three, 8 fits four
constexpr int ntt_ctas(int RB) { return RB >= 4 ? 3 : 4; }

// One pass over one tile of one row.  The last pass brings results to [0, q)
// (and, for the inverse, multiplies by N^-1).
// IO: 0 plain; 1 the forward transform of a fused rescale (RescaleIO); 2 the
// inverse transform of a fused key-switch gather (GatherIO).  IO > 0: rows by
// the map, no row list.
template <bool INV, int LOGN, int LP, bool COLS, int RB, int IO = 0>
__global__ void __launch_bounds__(kThreads, ntt_ctas(RB)) k_ntt(uint64_t* __restrict__ data, const __grid_constant__ LimbMap map,
                                                    const uint32_t* __restrict__ rowlist, uint32_t y0,
                                                    const uint64_t* __restrict__ qs,
                                                    const ulonglong2* __restrict__ tw,
                                                    const uint64_t* __restrict__ ninv,
                                                    const uint64_t* __restrict__ bar,
                                                    const __grid_constant__ RescaleIO rs,
                                                    const __grid_constant__ GatherIO ga)
{
    using G_ = Geo<LOGN, LP, COLS>;
    constexpr bool LAST = (LP == LOGN) || (INV ? COLS : !COLS);
    constexpr bool FIRST = (LP == LOGN) || (INV ? !COLS : COLS);
    constexpr bool RS = IO == 1, GA = IO == 2;
    static_assert(!(RS && INV) && !(GA && !INV), "rescale: forward only; gather: inverse only");
    __shared__ uint64_t sm[G_::TILE + G_::TILE / 16];
    pdl_begin();  // launched with programmatic stream serialization
    uint32_t row, pi;
    row_of(rowlist, map, y0 + blockIdx.y, row, pi);
    const uint32_t c0 = blockIdx.x << G_::LOGNSUB;
    const uint64_t q = qs[pi], q2 = 2 * q;
    const ulonglong2* W = tw + ((size_t)pi * 2 + (INV ? 1 : 0)) * G_::N;
    uint64_t* a = data + (size_t)row * G_::N;
    Fin fin{0, 0, 0, small_prime(q, LOGN)};
    if (INV && LAST) {
        fin.ni = ninv[2 * pi];
        fin.nis = ninv[2 * pi + 1];
    }
    if (!INV && LAST) fin.r1 = bar[2 * pi + 1];  // floor(2^64 / q)
    RsRow rr{};
    if (RS) {  // row = polynomial level + prime
        const uint32_t poly = row / rs.level, i = row % rs.level;
        rr.last = rs.last + (size_t)poly * G_::N;
        rr.in = rs.in + (size_t)(poly / rs.ppc) * rs.stride + ((size_t)(poly % rs.ppc) * (rs.level + 1) + i) * G_::N;
        rr.out = rs.out + (size_t)row * G_::N;
        rr.ql = qs[rs.level];
        rr.rb = bar[2 * pi + 1];
        rr.inv = rs.inv[2 * i];
        rr.inv_sh = rs.inv[2 * i + 1];
    }
    if (GA && FIRST) {  // row = source n + prime
        const uint32_t src = row / ga.n, i = row % ga.n;
        const GatherSrc d = ga.srcs[src];
        rr.c1 = d.c1 + (size_t)i * G_::N;
        rr.g = d.g;
        rr.ext = ga.ext + (((size_t)src * ga.beta + i / ga.alpha) * ga.E + i) * G_::N;
    }
    // the first round loads its groups from the row and the last stores them,
    // so the tile passes through shared memory only between rounds
    if (!INV) {
        if (fin.small) fwd_rounds<LOGN, LP, COLS, true, LP, RB, LAST, RS && FIRST, RS && LAST>(sm, a, c0, W, q, q2, fin, rr);
        else fwd_rounds<LOGN, LP, COLS, false, LP, RB, LAST, RS && FIRST, RS && LAST>(sm, a, c0, W, q, q2, fin, rr);
    } else {
        if (fin.small) inv_rounds<LOGN, LP, COLS, true, 0, RB, LAST, GA && FIRST>(sm, a, c0, W, q, q2, fin, rr);
        else inv_rounds<LOGN, LP, COLS, false, 0, RB, LAST, GA && FIRST>(sm, a, c0, W, q, q2, fin, rr);
    }
}

// One forward or inverse transform with the column pass over 2^L1-point
// sub-transforms and the row pass over 2^(LOGN - L1) points (L1 = 0: one pass).
// IO as k_ntt: 1 the forward transform of a fused rescale (rs), 2 the inverse
// transform of a fused gather (ga).
template <int LOGN, int L1, int RB, int IO>
int run_split(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map, const uint32_t* rowlist, bool inverse,
              const uint64_t* ninv, const RescaleIO& rs, const GatherIO& ga)
{
    constexpr uint32_t N = 1u << LOGN;
    constexpr uint32_t TILE = N < 4096 ? N : 4096;
    constexpr int L2 = LOGN - L1;
    static_assert(L2 <= 12 && (L1 == 0 || L1 <= 12), "pass longer than a tile");
    const ulonglong2* tw = reinterpret_cast<const ulonglong2*>(ctx->d_tw);
    const uint64_t* qs = (const uint64_t*)ctx->d_q;
    const uint64_t* bar = (const uint64_t*)ctx->d_bar;
    for (uint32_t y0 = 0; y0 < rows; y0 += kMaxGridY) {
        const dim3 grid(N / TILE, std::min(kMaxGridY, rows - y0));
        if (!inverse) {
            if constexpr (IO != 2) {
                if constexpr (L1 > 0) {
                    BLB_CUDA(launch_pdl(k_ntt<false, LOGN, L1, true, RB, IO>, grid, dim3(kThreads), 0, ctx->stream, data,
                                        map, rowlist, y0, qs, tw, ninv, bar, rs, ga));
                    BLB_LAUNCHED();
                }
                BLB_CUDA(launch_pdl(k_ntt<false, LOGN, L2, false, RB, IO>, grid, dim3(kThreads), 0, ctx->stream, data,
                                    map, rowlist, y0, qs, tw, ninv, bar, rs, ga));
                BLB_LAUNCHED();
            }
        } else if constexpr (IO != 1) {
            BLB_CUDA(launch_pdl(k_ntt<true, LOGN, L2, false, RB, IO>, grid, dim3(kThreads), 0, ctx->stream, data, map,
                                rowlist, y0, qs, tw, ninv, bar, rs, ga));
            BLB_LAUNCHED();
            if constexpr (L1 > 0) {
                BLB_CUDA(launch_pdl(k_ntt<true, LOGN, L1, true, RB, IO>, grid, dim3(kThreads), 0, ctx->stream, data, map,
                                    rowlist, y0, qs, tw, ninv, bar, rs, ga));
                BLB_LAUNCHED();
            }
        }
    }
    return BLB_OK;
}

// Transforms above one tile have three splits around the middle, chosen per
// context (ctx->ntt_split: 0 the middle, -1 / +1 a shorter / longer column
// pass), and two radices of the register rounds (ctx->ntt_radix: 8, four CTAs
// per SM, or 16, three); blb_ntt_autotune times all of them.
template <int LOGN, int RB, int IO>
int run_nr(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map, const uint32_t* rowlist, bool inverse,
           const uint64_t* ninv, const RescaleIO& rs, const GatherIO& ga)
{
    if constexpr (LOGN <= 12) {
        return run_split<LOGN, 0, RB, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
    } else {
        constexpr int M = LOGN / 2;
        switch (ctx->ntt_split) {
        case -1: return run_split<LOGN, M - 1, RB, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
        case 1:
            if constexpr (LOGN - (M + 1) >= 1)
                return run_split<LOGN, M + 1, RB, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
            else return run_split<LOGN, M, RB, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
        default: return run_split<LOGN, M, RB, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
        }
    }
}

template <int LOGN, int IO>
int run_n(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map, const uint32_t* rowlist, bool inverse,
          const uint64_t* ninv, const RescaleIO& rs, const GatherIO& ga)
{
    if (ctx->ntt_radix == 16) return run_nr<LOGN, 4, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
    return run_nr<LOGN, 3, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
}

template <int IO>
int run_io(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map, const uint32_t* rowlist, bool inverse,
           const uint64_t* ninv, const RescaleIO& rs, const GatherIO& ga)
{
    switch (ctx->logN) {
    case 10: return run_n<10, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
    case 11: return run_n<11, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
    case 12: return run_n<12, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
    case 13: return run_n<13, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
    case 14: return run_n<14, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
    case 15: return run_n<15, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
    case 16: return run_n<16, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
    case 17: return run_n<17, IO>(ctx, data, rows, map, rowlist, inverse, ninv, rs, ga);
    default: return blb_fail(BLB_ERR_ARG, "no NTT for this ring size");
    }
}

const RescaleIO kNoRescale{};
const GatherIO kNoGather{};

// ninv: [prime][2] the constant the last inverse pass multiplies by and its
// Shoup companion (N^-1 mod q, or N^-1 times a conversion factor, see
// ntt_inverse_scaled)
int run(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map, const uint32_t* rowlist, bool inverse,
        const uint64_t* ninv)
{
    return run_io<0>(ctx, data, rows, map, rowlist, inverse, ninv, kNoRescale, kNoGather);
}

}  // namespace

// us_per_row[6]: radix 8 at splits -1, 0, +1, then radix 16 at the same splits
extern "C" int blb_ntt_autotune(blb_ctx* ctx, uint32_t rows, int* split_out, int* radix_out, double* us_per_row)
{
    if (!ctx || rows == 0) return blb_fail(BLB_ERR_ARG, "null argument or no rows");
    BLB_TRY(refuse_capture(ctx, "NTT autotuning"));
    const size_t words = (size_t)rows * ctx->N;
    uint64_t* buf = (uint64_t*)dev_alloc(ctx, words * 8);
    if (!buf) return blb_fail(BLB_ERR_OOM, "autotune buffer");
    BLB_CUDA(cudaMemsetAsync(buf, 0, words * 8, ctx->stream));
    const LimbMap map = ctx->qmap(ctx->nQ);
    cudaEvent_t e0, e1;
    BLB_CUDA(cudaEventCreate(&e0));
    BLB_CUDA(cudaEventCreate(&e1));
    const int keep_split = ctx->ntt_split, keep_radix = ctx->ntt_radix;
    int best = 0, best_radix = 8, rc = BLB_OK;
    float best_ms = 1e30f;
    double per[6] = {0, 0, 0, 0, 0, 0};
    const int radices[2] = {8, 16};
    for (int ri = 0; ri < 2 && !rc; ri++) {
        for (int sp = -1; sp <= 1 && !rc; sp++) {
            if (ctx->logN <= 12 && sp) continue;
            ctx->ntt_split = sp;
            ctx->ntt_radix = radices[ri];
            float ms = 0;
            for (int rep = 0; rep < 3 && !rc; rep++) {  // the first run is a warm-up
                cudaEventRecord(e0, ctx->stream);
                rc = run(ctx, buf, rows, map, nullptr, false, ctx->d_ninv);
                if (!rc) rc = run(ctx, buf, rows, map, nullptr, true, ctx->d_ninv);
                cudaEventRecord(e1, ctx->stream);
                if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = blb_fail(BLB_ERR_CUDA, "autotune run failed");
                float t = 0;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep) ms += t;
            }
            per[3 * ri + sp + 1] = ms * 1e3 / (2.0 * 2.0 * rows);  // two timed runs, forward + inverse
            if (!rc && ms < best_ms) {
                best_ms = ms;
                best = sp;
                best_radix = radices[ri];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(ctx, buf, words * 8);
    ctx->ntt_split = rc ? keep_split : best;
    ctx->ntt_radix = rc ? keep_radix : best_radix;
    if (rc) return rc;
    if (split_out) *split_out = best;
    if (radix_out) *radix_out = best_radix;
    if (us_per_row)
        for (int k = 0; k < 6; k++) us_per_row[k] = per[k];
    return BLB_OK;
}

extern "C" int blb_ntt_set_radix(blb_ctx* ctx, int radix)
{
    if (!ctx) return blb_fail(BLB_ERR_ARG, "null context");
    if (radix != 8 && radix != 16) return blb_fail(BLB_ERR_ARG, "NTT radix must be 8 or 16");
    ctx->ntt_radix = radix;
    return BLB_OK;
}

extern "C" int blb_ntt_set_split(blb_ctx* ctx, int split)
{
    if (!ctx || split < -1 || split > 1) return blb_fail(BLB_ERR_ARG, "split must be -1, 0 or 1");
    ctx->ntt_split = split;
    return BLB_OK;
}

int ntt_forward(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "ntt", (uint64_t)rows * ctx->N * 16);  // one read + one write per word
    return run(ctx, data, rows, map, nullptr, false, ctx->d_ninv);
}

int ntt_inverse(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "intt", (uint64_t)rows * ctx->N * 16);
    return run(ctx, data, rows, map, nullptr, true, ctx->d_ninv);
}

int ntt_forward_rescale(blb_ctx* ctx, uint64_t* data, uint32_t rows, const RescaleIO& rs)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "ntt", (uint64_t)rows * ctx->N * 16);
    return run_io<1>(ctx, data, rows, ctx->qmap(rs.level), nullptr, false, ctx->d_ninv, rs, kNoGather);
}

int ntt_inverse_gather(blb_ctx* ctx, uint64_t* data, uint32_t rows, const GatherIO& ga, const uint64_t* ninv)
{
    if (rows == 0) return BLB_OK;
    // a site of its own (inside the key-switch site): besides the transform's
    // 16 bytes per word it reads the permuted source and writes the digit row
    ProfScope prof(ctx, "intt_gather", (uint64_t)rows * ctx->N * 32);
    return run_io<2>(ctx, data, rows, ctx->qmap(ga.n), nullptr, true, ninv, kNoRescale, ga);
}

int ntt_forward_list(blb_ctx* ctx, uint64_t* data, uint32_t rows, const uint32_t* d_rowlist)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "ntt", (uint64_t)rows * ctx->N * 16);
    LimbMap none{};
    none.n = 1;
    return run(ctx, data, rows, none, d_rowlist, false, ctx->d_ninv);
}

int ntt_inverse_list(blb_ctx* ctx, uint64_t* data, uint32_t rows, const uint32_t* d_rowlist)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "intt", (uint64_t)rows * ctx->N * 16);
    LimbMap none{};
    none.n = 1;
    return run(ctx, data, rows, none, d_rowlist, true, ctx->d_ninv);
}

int ntt_inverse_scaled(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map, const uint64_t* ninv)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "intt", (uint64_t)rows * ctx->N * 16);
    return run(ctx, data, rows, map, nullptr, true, ninv);
}

int ntt_inverse_list_scaled(blb_ctx* ctx, uint64_t* data, uint32_t rows, const uint32_t* d_rowlist, const uint64_t* ninv)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "intt", (uint64_t)rows * ctx->N * 16);
    LimbMap none{};
    none.n = 1;
    return run(ctx, data, rows, none, d_rowlist, true, ninv);
}
