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
// writes each word once.  Inside a pass each thread holds a group of up to 16
// elements in registers and runs up to 4 stages on it (radix 16), so a pass
// needs 2-3 shared-memory round trips instead of one per stage.  Shared memory
// is padded by one word every 16 to keep strided group accesses conflict-free.
// Butterflies reduce lazily (Harvey): forward values stay in [0, 4q), inverse
// values in [0, 2q); the last pass returns them to [0, q).
//
// Rows: either rows 0..rows-1 of `data` with prime map.p[row % map.n], or an
// explicit row list (entry = row index | prime index << 24) so that a batch can
// transform exactly the rows it needs in one launch.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr uint32_t kTile = 4096;  // words per CTA
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

// forward: X, Y in [0, 4q) -> X + WY, X - WY in [0, 4q)
__device__ __forceinline__ void bfly_fwd(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t wp, uint64_t q, uint64_t q2)
{
    uint64_t x = X >= q2 ? X - q2 : X;
    uint64_t t = mul_shoup_lazy(Y, w, wp, q);
    X = x + t;
    Y = x - t + q2;
}

// inverse: X, Y in [0, 2q) -> X + Y, W (X - Y) in [0, 2q)
__device__ __forceinline__ void bfly_inv(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t wp, uint64_t q, uint64_t q2)
{
    uint64_t s = X + Y;
    s = s >= q2 ? s - q2 : s;
    uint64_t d = X - Y + q2;
    X = s;
    Y = mul_shoup_lazy(d, w, wp, q);
}

struct Pass {
    uint32_t logN;  // transform size
    uint32_t l;     // log2 of the sub-transform length handled by this pass
    uint32_t goff;  // global index bit of local bit 0 (logN - l for the column pass, 0 for rows)
    uint32_t cols;  // 1: column pass (sub-transforms strided by N / L), 0: contiguous blocks
    uint32_t lognsub;
    uint32_t c0;    // first column (column pass) or first block (row pass) of this tile
};

// One round: R stages on groups of 2^R elements whose local indices differ in
// bits [p_lo, p_lo + R).
template <int R, bool INV>
__device__ __forceinline__ void round(uint64_t* sm, const Pass& P, uint32_t tile, uint32_t p_lo,
                                      const uint64_t* __restrict__ W, const uint64_t* __restrict__ Wp, uint64_t q,
                                      uint64_t q2)
{
    constexpr uint32_t K = 1u << R;
    const uint32_t L = 1u << P.l, nsub = 1u << P.lognsub;
    const uint32_t N = 1u << P.logN;
    const uint32_t groups = tile >> R;
    for (uint32_t G = threadIdx.x; G < groups; G += blockDim.x) {
        uint32_t sub, g;
        if (P.cols) {
            sub = G & (nsub - 1);
            g = G >> P.lognsub;
        } else {
            g = G & ((L >> R) - 1);
            sub = G >> (P.l - R);
        }
        const uint32_t base_r = ((g >> p_lo) << (p_lo + R)) | (g & ((1u << p_lo) - 1));
        uint32_t e_base, e_stride, j_base;
        if (P.cols) {
            e_base = (base_r << P.lognsub) + sub;
            e_stride = nsub << p_lo;
            j_base = P.c0 + sub + (base_r << P.goff);
        } else {
            e_base = (sub << P.l) + base_r;
            e_stride = 1u << p_lo;
            j_base = ((P.c0 + sub) << P.l) + base_r;
        }
        const uint32_t j_shift = P.goff + p_lo;
        uint64_t x[K];
#pragma unroll
        for (uint32_t k = 0; k < K; k++) x[k] = sm[padi(e_base + k * e_stride)];
        // The butterflied bits of base_r are zero, so for the pair (k, k | 2^u)
        // the lower element's twiddle index splits into a per-stage base plus
        // k >> (u + 1): stage u uses 2^(R-1-u) distinct twiddles.
        if (!INV) {
#pragma unroll
            for (int u = R - 1; u >= 0; u--) {
                const uint32_t s = P.logN - 1 - (j_shift + u);
                const uint32_t wbase = (1u << s) + (j_base >> (j_shift + u + 1));
#pragma unroll
                for (uint32_t h = 0; h < (K >> (u + 1)); h++) {
                    const uint64_t w = W[wbase + h], wp = Wp[wbase + h];
#pragma unroll
                    for (uint32_t lo = 0; lo < (1u << u); lo++) {
                        const uint32_t k = (h << (u + 1)) | lo;
                        bfly_fwd(x[k], x[k | (1u << u)], w, wp, q, q2);
                    }
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < R; u++) {
                const uint32_t lt = j_shift + u;
                const uint32_t wbase = (N + j_base) >> (lt + 1);
#pragma unroll
                for (uint32_t h = 0; h < (K >> (u + 1)); h++) {
                    const uint64_t w = W[wbase + h], wp = Wp[wbase + h];
#pragma unroll
                    for (uint32_t lo = 0; lo < (1u << u); lo++) {
                        const uint32_t k = (h << (u + 1)) | lo;
                        bfly_inv(x[k], x[k | (1u << u)], w, wp, q, q2);
                    }
                }
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < K; k++) sm[padi(e_base + k * e_stride)] = x[k];
    }
}

template <bool INV>
__device__ __forceinline__ void round_r(uint32_t R, uint64_t* sm, const Pass& P, uint32_t tile, uint32_t p_lo,
                                        const uint64_t* W, const uint64_t* Wp, uint64_t q, uint64_t q2)
{
    switch (R) {
        case 4: round<4, INV>(sm, P, tile, p_lo, W, Wp, q, q2); break;
        case 3: round<3, INV>(sm, P, tile, p_lo, W, Wp, q, q2); break;
        case 2: round<2, INV>(sm, P, tile, p_lo, W, Wp, q, q2); break;
        default: round<1, INV>(sm, P, tile, p_lo, W, Wp, q, q2); break;
    }
}

// One pass over one tile of one row.  last: bring results to [0, q) (and, for
// the inverse, multiply by N^-1).
template <bool INV>
__global__ void __launch_bounds__(kThreads, 3) k_ntt_pass(uint64_t* __restrict__ data, LimbMap map,
                                                       const uint32_t* __restrict__ rowlist, uint32_t y0,
                                                       const uint64_t* __restrict__ qs,
                                                       const uint64_t* __restrict__ tw,
                                                       const uint64_t* __restrict__ ninv, uint32_t logN, uint32_t l,
                                                       uint32_t cols, int last)
{
    __shared__ uint64_t sm[kTile + kTile / 16];
    uint32_t row, pi;
    row_of(rowlist, map, y0 + blockIdx.y, row, pi);
    const uint32_t N = 1u << logN;
    const uint32_t tile = N < kTile ? N : kTile;
    Pass P;
    P.logN = logN;
    P.l = l;
    P.goff = cols ? logN - l : 0;
    P.cols = cols;
    P.lognsub = __ffs(tile >> l) - 1;  // tile / L sub-transforms per tile
    P.c0 = blockIdx.x << P.lognsub;
    const uint64_t q = qs[pi], q2 = 2 * q;
    const uint64_t* W = tw + (size_t)pi * 4 * N + (INV ? 2 * N : 0);
    const uint64_t* Wp = W + N;
    uint64_t* a = data + (size_t)row * N;
    // load the tile: element e = r * nsub + sub (columns) or sub * L + r (rows)
    if (cols) {
        const uint32_t logN2 = logN - l, nsub = 1u << P.lognsub;
        for (uint32_t e = threadIdx.x; e < tile; e += blockDim.x)
            sm[padi(e)] = a[((size_t)(e >> P.lognsub) << logN2) + P.c0 + (e & (nsub - 1))];
    } else {
        const uint64_t* src = a + ((size_t)P.c0 << l);
        for (uint32_t e = threadIdx.x; e < tile; e += blockDim.x) sm[padi(e)] = src[e];
    }
    __syncthreads();
    if (!INV) {
        for (int p_hi = (int)l; p_hi > 0;) {
            const uint32_t R = p_hi >= 4 ? 4 : (uint32_t)p_hi;
            round_r<false>(R, sm, P, tile, (uint32_t)p_hi - R, W, Wp, q, q2);
            p_hi -= (int)R;
            __syncthreads();
        }
    } else {
        for (uint32_t p_lo = 0; p_lo < l;) {
            const uint32_t R = l - p_lo >= 4 ? 4 : l - p_lo;
            round_r<true>(R, sm, P, tile, p_lo, W, Wp, q, q2);
            p_lo += R;
            __syncthreads();
        }
    }
    uint64_t ni = 0, nis = 0;
    if (INV && last) {
        ni = ninv[2 * pi];
        nis = ninv[2 * pi + 1];
    }
    auto finish = [&](uint64_t v) -> uint64_t {
        if (!last) return v;
        if (INV) v = mul_shoup_lazy(v, ni, nis, q);
        else v = v >= q2 ? v - q2 : v;
        return v >= q ? v - q : v;
    };
    if (cols) {
        const uint32_t logN2 = logN - l, nsub = 1u << P.lognsub;
        for (uint32_t e = threadIdx.x; e < tile; e += blockDim.x)
            a[((size_t)(e >> P.lognsub) << logN2) + P.c0 + (e & (nsub - 1))] = finish(sm[padi(e)]);
    } else {
        uint64_t* dst = a + ((size_t)P.c0 << l);
        for (uint32_t e = threadIdx.x; e < tile; e += blockDim.x) dst[e] = finish(sm[padi(e)]);
    }
}

struct Split {
    uint32_t l1, l2;  // column pass length (0: single pass), row pass length
};

Split split(uint32_t logN)
{
    if (logN <= 12) return {0, logN};
    return {logN / 2, logN - logN / 2};
}

int run(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map, const uint32_t* rowlist, bool inverse)
{
    const uint32_t logN = ctx->logN, N = 1u << logN;
    const uint32_t tile = N < kTile ? N : kTile;
    const Split sp = split(logN);
    const uint32_t gx = N / tile;
    for (uint32_t y0 = 0; y0 < rows; y0 += kMaxGridY) {
        const uint32_t ny = std::min(kMaxGridY, rows - y0);
        const dim3 grid(gx, ny);
        if (!inverse) {
            if (sp.l1) {
                k_ntt_pass<false><<<grid, kThreads, 0, ctx->stream>>>(data, map, rowlist, y0, ctx->d_q, ctx->d_tw,
                                                                     ctx->d_ninv, logN, sp.l1, 1, 0);
                BLB_LAUNCHED();
            }
            k_ntt_pass<false><<<grid, kThreads, 0, ctx->stream>>>(data, map, rowlist, y0, ctx->d_q, ctx->d_tw,
                                                                 ctx->d_ninv, logN, sp.l2, 0, 1);
            BLB_LAUNCHED();
        } else {
            k_ntt_pass<true><<<grid, kThreads, 0, ctx->stream>>>(data, map, rowlist, y0, ctx->d_q, ctx->d_tw,
                                                                ctx->d_ninv, logN, sp.l2, 0, sp.l1 == 0);
            BLB_LAUNCHED();
            if (sp.l1) {
                k_ntt_pass<true><<<grid, kThreads, 0, ctx->stream>>>(data, map, rowlist, y0, ctx->d_q, ctx->d_tw,
                                                                    ctx->d_ninv, logN, sp.l1, 1, 1);
                BLB_LAUNCHED();
            }
        }
    }
    return BLB_OK;
}

}  // namespace

int ntt_forward(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "ntt", (uint64_t)rows * ctx->N * 16);  // one read + one write per word
    return run(ctx, data, rows, map, nullptr, false);
}

int ntt_inverse(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "intt", (uint64_t)rows * ctx->N * 16);
    return run(ctx, data, rows, map, nullptr, true);
}

int ntt_forward_list(blb_ctx* ctx, uint64_t* data, uint32_t rows, const uint32_t* d_rowlist)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "ntt", (uint64_t)rows * ctx->N * 16);
    LimbMap none{};
    none.n = 1;
    return run(ctx, data, rows, none, d_rowlist, false);
}

int ntt_inverse_list(blb_ctx* ctx, uint64_t* data, uint32_t rows, const uint32_t* d_rowlist)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "intt", (uint64_t)rows * ctx->N * 16);
    LimbMap none{};
    none.n = 1;
    return run(ctx, data, rows, none, d_rowlist, true);
}
