// ntt.cu -- batched negacyclic NTT / inverse NTT over 64-bit primes.
//
// Forward: Cooley-Tukey butterflies with psi powers in bit-reversed order,
// natural-order input, output A[k] = a(psi^(2 bitrev(k) + 1)).  Inverse:
// Gentleman-Sande butterflies with psi^-1 powers, then N^-1.
//
// Large N is split N = N1 * N2.  The first log2(N1) forward stages pair elements
// whose distance is a multiple of N2; they act on "columns" {c + N2 r}, and a
// CTA processes a tile of kCols adjacent columns in shared memory (each row of
// the tile is a contiguous 8*kCols-byte segment of HBM).  The remaining
// log2(N2) stages act on contiguous blocks of N2 words.  Each pass reads and
// writes the limb once.  The inverse runs the two passes in the opposite order
// and folds N^-1 into the last one.
#include "common.cuh"

namespace {

constexpr int kCols = 16;         // columns per CTA in the strided pass
constexpr int kSmemWords = 4096;  // 32 KB of shared memory per CTA
constexpr int kThreads = 256;

struct NttGeom {
    uint32_t logN, logN1, N, N1, N2;
};

NttGeom geom(uint32_t logN)
{
    NttGeom g;
    g.logN = logN;
    g.N = 1u << logN;
    g.logN1 = logN <= 12 ? 0 : logN / 2;  // N <= 4096 fits one CTA: single pass
    g.N1 = 1u << g.logN1;
    g.N2 = g.N >> g.logN1;
    return g;
}

// forward, stages m = 1 .. N1/2 on column tiles
__global__ void __launch_bounds__(kThreads) k_ntt_fwd_cols(uint64_t* __restrict__ data, LimbMap map,
                                                           const uint64_t* __restrict__ qs,
                                                           const uint64_t* __restrict__ tw, uint32_t logN,
                                                           uint32_t logN1)
{
    __shared__ uint64_t sm[kSmemWords];
    const uint32_t N = 1u << logN, N1 = 1u << logN1, N2 = N >> logN1;
    const uint32_t row = blockIdx.y;
    const uint32_t pi = map.p[row % map.n];
    const uint64_t q = qs[pi];
    const uint64_t* W = tw + (size_t)pi * 4 * N;
    const uint64_t* Wp = W + N;
    uint64_t* a = data + (size_t)row * N;
    const uint32_t c0 = blockIdx.x * kCols;
    for (uint32_t idx = threadIdx.x; idx < N1 * kCols; idx += blockDim.x) {
        uint32_t r = idx / kCols, c = idx % kCols;
        sm[idx] = a[(size_t)r * N2 + c0 + c];
    }
    __syncthreads();
    for (uint32_t m = 1, tr = N1 / 2; m < N1; m <<= 1, tr >>= 1) {
        for (uint32_t idx = threadIdx.x; idx < (N1 / 2) * kCols; idx += blockDim.x) {
            uint32_t c = idx % kCols, bf = idx / kCols;
            uint32_t i = bf / tr, jr = bf % tr;
            uint32_t r = 2 * i * tr + jr;
            uint64_t U = sm[r * kCols + c];
            uint64_t V = mul_shoup(sm[(r + tr) * kCols + c], W[m + i], Wp[m + i], q);
            sm[r * kCols + c] = add_mod(U, V, q);
            sm[(r + tr) * kCols + c] = sub_mod(U, V, q);
        }
        __syncthreads();
    }
    for (uint32_t idx = threadIdx.x; idx < N1 * kCols; idx += blockDim.x) {
        uint32_t r = idx / kCols, c = idx % kCols;
        a[(size_t)r * N2 + c0 + c] = sm[idx];
    }
}

// forward, stages m = N1 .. N/2 on contiguous blocks of N2 (bpc blocks per CTA)
__global__ void __launch_bounds__(kThreads) k_ntt_fwd_rows(uint64_t* __restrict__ data, LimbMap map,
                                                           const uint64_t* __restrict__ qs,
                                                           const uint64_t* __restrict__ tw, uint32_t logN,
                                                           uint32_t logN1, uint32_t bpc)
{
    __shared__ uint64_t sm[kSmemWords];
    const uint32_t N = 1u << logN, N1 = 1u << logN1, N2 = N >> logN1;
    const uint32_t row = blockIdx.y;
    const uint32_t pi = map.p[row % map.n];
    const uint64_t q = qs[pi];
    const uint64_t* W = tw + (size_t)pi * 4 * N;
    const uint64_t* Wp = W + N;
    const uint32_t b0 = blockIdx.x * bpc;
    uint64_t* a = data + (size_t)row * N + (size_t)b0 * N2;
    const uint32_t words = bpc * N2;
    for (uint32_t idx = threadIdx.x; idx < words; idx += blockDim.x) sm[idx] = a[idx];
    __syncthreads();
    for (uint32_t ml = 1, t = N2 / 2; ml < N2; ml <<= 1, t >>= 1) {
        for (uint32_t idx = threadIdx.x; idx < words / 2; idx += blockDim.x) {
            uint32_t blk = idx / (N2 / 2), bf = idx % (N2 / 2);
            uint32_t il = bf / t, jl = bf % t;
            uint32_t r = blk * N2 + 2 * il * t + jl;
            uint32_t wi = N1 * ml + (b0 + blk) * ml + il;
            uint64_t U = sm[r];
            uint64_t V = mul_shoup(sm[r + t], W[wi], Wp[wi], q);
            sm[r] = add_mod(U, V, q);
            sm[r + t] = sub_mod(U, V, q);
        }
        __syncthreads();
    }
    for (uint32_t idx = threadIdx.x; idx < words; idx += blockDim.x) a[idx] = sm[idx];
}

// inverse, stages t = 1 .. N2/2 on contiguous blocks; optionally times N^-1
__global__ void __launch_bounds__(kThreads) k_ntt_inv_rows(uint64_t* __restrict__ data, LimbMap map,
                                                           const uint64_t* __restrict__ qs,
                                                           const uint64_t* __restrict__ tw,
                                                           const uint64_t* __restrict__ ninv, uint32_t logN,
                                                           uint32_t logN1, uint32_t bpc, int scale)
{
    __shared__ uint64_t sm[kSmemWords];
    const uint32_t N = 1u << logN, N2 = N >> logN1;
    const uint32_t row = blockIdx.y;
    const uint32_t pi = map.p[row % map.n];
    const uint64_t q = qs[pi];
    const uint64_t* W = tw + (size_t)pi * 4 * N + 2 * N;
    const uint64_t* Wp = W + N;
    const uint32_t b0 = blockIdx.x * bpc;
    uint64_t* a = data + (size_t)row * N + (size_t)b0 * N2;
    const uint32_t words = bpc * N2;
    for (uint32_t idx = threadIdx.x; idx < words; idx += blockDim.x) sm[idx] = a[idx];
    __syncthreads();
    for (uint32_t t = 1; t < N2; t <<= 1) {
        const uint32_t h = N / (2 * t);
        for (uint32_t idx = threadIdx.x; idx < words / 2; idx += blockDim.x) {
            uint32_t blk = idx / (N2 / 2), bf = idx % (N2 / 2);
            uint32_t il = bf / t, jl = bf % t;
            uint32_t r = blk * N2 + 2 * il * t + jl;
            uint32_t wi = h + (b0 + blk) * (N2 / (2 * t)) + il;
            uint64_t U = sm[r], V = sm[r + t];
            sm[r] = add_mod(U, V, q);
            sm[r + t] = mul_shoup(sub_mod(U, V, q), W[wi], Wp[wi], q);
        }
        __syncthreads();
    }
    if (scale) {
        const uint64_t ni = ninv[2 * pi], nis = ninv[2 * pi + 1];
        for (uint32_t idx = threadIdx.x; idx < words; idx += blockDim.x) a[idx] = mul_shoup(sm[idx], ni, nis, q);
    } else {
        for (uint32_t idx = threadIdx.x; idx < words; idx += blockDim.x) a[idx] = sm[idx];
    }
}

// inverse, stages t = N2 .. N/2 on column tiles, then times N^-1
__global__ void __launch_bounds__(kThreads) k_ntt_inv_cols(uint64_t* __restrict__ data, LimbMap map,
                                                           const uint64_t* __restrict__ qs,
                                                           const uint64_t* __restrict__ tw,
                                                           const uint64_t* __restrict__ ninv, uint32_t logN,
                                                           uint32_t logN1)
{
    __shared__ uint64_t sm[kSmemWords];
    const uint32_t N = 1u << logN, N1 = 1u << logN1, N2 = N >> logN1;
    const uint32_t row = blockIdx.y;
    const uint32_t pi = map.p[row % map.n];
    const uint64_t q = qs[pi];
    const uint64_t* W = tw + (size_t)pi * 4 * N + 2 * N;
    const uint64_t* Wp = W + N;
    uint64_t* a = data + (size_t)row * N;
    const uint32_t c0 = blockIdx.x * kCols;
    for (uint32_t idx = threadIdx.x; idx < N1 * kCols; idx += blockDim.x) {
        uint32_t r = idx / kCols, c = idx % kCols;
        sm[idx] = a[(size_t)r * N2 + c0 + c];
    }
    __syncthreads();
    for (uint32_t tr = 1; tr < N1; tr <<= 1) {
        const uint32_t h = N1 / (2 * tr);  // = N / (2 t) with t = tr * N2
        for (uint32_t idx = threadIdx.x; idx < (N1 / 2) * kCols; idx += blockDim.x) {
            uint32_t c = idx % kCols, bf = idx / kCols;
            uint32_t i = bf / tr, jr = bf % tr;
            uint32_t r = 2 * i * tr + jr;
            uint64_t U = sm[r * kCols + c], V = sm[(r + tr) * kCols + c];
            sm[r * kCols + c] = add_mod(U, V, q);
            sm[(r + tr) * kCols + c] = mul_shoup(sub_mod(U, V, q), W[h + i], Wp[h + i], q);
        }
        __syncthreads();
    }
    const uint64_t ni = ninv[2 * pi], nis = ninv[2 * pi + 1];
    for (uint32_t idx = threadIdx.x; idx < N1 * kCols; idx += blockDim.x) {
        uint32_t r = idx / kCols, c = idx % kCols;
        a[(size_t)r * N2 + c0 + c] = mul_shoup(sm[idx], ni, nis, q);
    }
}

}  // namespace

int ntt_forward(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "ntt", (uint64_t)rows * ctx->N * 16);  // one read + one write per word
    NttGeom g = geom(ctx->logN);
    if (g.N1 > 1) {
        dim3 grid(g.N2 / kCols, rows);
        k_ntt_fwd_cols<<<grid, kThreads, 0, ctx->stream>>>(data, map, ctx->d_q, ctx->d_tw, g.logN, g.logN1);
        BLB_LAUNCHED();
    }
    uint32_t bpc = g.N2 >= (uint32_t)kSmemWords ? 1 : kSmemWords / g.N2;
    if (bpc > g.N1) bpc = g.N1;
    dim3 grid(g.N1 / bpc, rows);
    k_ntt_fwd_rows<<<grid, kThreads, 0, ctx->stream>>>(data, map, ctx->d_q, ctx->d_tw, g.logN, g.logN1, bpc);
    BLB_LAUNCHED();
    return BLB_OK;
}

int ntt_inverse(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map)
{
    if (rows == 0) return BLB_OK;
    ProfScope prof(ctx, "intt", (uint64_t)rows * ctx->N * 16);
    NttGeom g = geom(ctx->logN);
    uint32_t bpc = g.N2 >= (uint32_t)kSmemWords ? 1 : kSmemWords / g.N2;
    if (bpc > g.N1) bpc = g.N1;
    dim3 grid(g.N1 / bpc, rows);
    k_ntt_inv_rows<<<grid, kThreads, 0, ctx->stream>>>(data, map, ctx->d_q, ctx->d_tw, ctx->d_ninv, g.logN, g.logN1,
                                                       bpc, g.N1 == 1);
    BLB_LAUNCHED();
    if (g.N1 > 1) {
        dim3 grid2(g.N2 / kCols, rows);
        k_ntt_inv_cols<<<grid2, kThreads, 0, ctx->stream>>>(data, map, ctx->d_q, ctx->d_tw, ctx->d_ninv, g.logN,
                                                            g.logN1);
        BLB_LAUNCHED();
    }
    return BLB_OK;
}
