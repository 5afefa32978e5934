// kernels.cu -- element-wise RNS kernels: products and sums per limb, the
// Galois automorphism in the evaluation domain, Philox samplers, rescale and
// the ciphertext tensor product.
#include "common.cuh"

namespace {
constexpr int kT = 256;

inline dim3 grid_rows(uint32_t N, uint32_t rows) { return dim3((N + kT - 1) / kT, rows); }

__global__ void k_mul_rows(uint64_t* __restrict__ out, const uint64_t* __restrict__ a,
                           const uint64_t* __restrict__ b, const __grid_constant__ LimbMap map, const uint64_t* __restrict__ qs,
                           const uint64_t* __restrict__ bar, uint32_t N, uint32_t b_rows, int accumulate)
{
    const uint32_t row = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const uint32_t pi = map.p[row % map.n];
    const uint64_t q = qs[pi];
    const size_t o = (size_t)row * N + c;
    uint64_t v = mul_mod(a[o], b[(size_t)(row % b_rows) * N + c], q, bar[2 * pi], bar[2 * pi + 1]);
    out[o] = accumulate ? add_mod(out[o], v, q) : v;
}

// op: 0 add, 1 sub, 2 neg (b unused)
__global__ void k_addsub_rows(uint64_t* __restrict__ out, const uint64_t* __restrict__ a,
                              const uint64_t* __restrict__ b, const __grid_constant__ LimbMap map, const uint64_t* __restrict__ qs,
                              uint32_t N, int op)
{
    const uint32_t row = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const uint64_t q = qs[map.p[row % map.n]];
    const size_t o = (size_t)row * N + c;
    uint64_t x = a[o];
    out[o] = op == 0 ? add_mod(x, b[o], q) : op == 1 ? sub_mod(x, b[o], q) : neg_mod(x, q);
}

struct RowConst {
    uint64_t w[BLB_MAXP * 4], wp[BLB_MAXP * 4];
};
__global__ void k_mul_const_rows(uint64_t* __restrict__ out, const uint64_t* __restrict__ a, const __grid_constant__ LimbMap map,
                                 const uint64_t* __restrict__ qs, uint32_t N, RowConst rc)
{
    const uint32_t row = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const uint64_t q = qs[map.p[row % map.n]];
    const size_t o = (size_t)row * N + c;
    out[o] = mul_shoup(a[o], rc.w[row], rc.wp[row], q);
}

// Evaluation-domain automorphism.  With A[k] = a(psi^(2 brv(k) + 1)),
// sigma_g(a)(psi^e) = a(psi^(g e)); output slot k reads input slot
// brv(((g (2 brv(k) + 1)) mod 2N - 1) / 2).  A pure permutation.
__global__ void k_automorph_ntt(uint64_t* __restrict__ out, const uint64_t* __restrict__ in, uint32_t logN,
                                uint64_t g)
{
    const uint32_t N = 1u << logN;
    const uint32_t row = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const uint64_t e = 2 * (uint64_t)(__brev(k) >> (32 - logN)) + 1;
    const uint32_t ge = (uint32_t)((g * e) & (2ull * N - 1));
    const uint32_t src = __brev((ge - 1) >> 1) >> (32 - logN);
    out[(size_t)row * N + k] = in[(size_t)row * N + src];
}

__global__ void k_signed_to_rows(uint64_t* __restrict__ out, const int64_t* __restrict__ in, const __grid_constant__ LimbMap map,
                                 const uint64_t* __restrict__ qs, const uint64_t* __restrict__ bar, uint32_t N)
{
    const uint32_t row = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const uint32_t pi = map.p[row % map.n];
    out[(size_t)row * N + c] = signed_mod(in[c], qs[pi], bar[2 * pi + 1]);
}

// --- Philox draws: counter (coefficient i, sub-index j, object, purpose) ---
__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t i, uint32_t j, uint32_t obj, uint32_t purpose)
{
    return philox_draw(seed, i, j, obj, purpose);
}

__global__ void k_sample_ternary(int64_t* out, uint32_t N, uint64_t seed, uint32_t obj, uint32_t purpose, uint32_t j)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint4 r = draw(seed, i, j, obj, purpose);
    out[i] = (int64_t)(r.x % 3u) - 1;
}

// discrete Gaussian by inversion of the cumulative table of |e|; sign from
// bit 0 of the third word
__global__ void k_sample_gauss(int64_t* out, uint32_t N, const uint64_t* __restrict__ cdt, uint64_t seed,
                               uint32_t obj, uint32_t purpose, uint32_t j)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint4 r = draw(seed, i, j, obj, purpose);
    uint64_t u = (uint64_t)r.x | ((uint64_t)r.y << 32);
    int64_t k = 0;
#pragma unroll
    for (int t = 0; t < 19; t++) k += (u >= cdt[t]);
    out[i] = (r.z & 1u) ? -k : k;
}

struct RowJ {
    uint32_t j[BLB_MAXP * 4];
};

// uniform residue: the 128-bit draw (word 3 most significant) mod q
__global__ void k_sample_uniform(uint64_t* out, uint32_t N, const __grid_constant__ LimbMap map, const uint64_t* __restrict__ qs,
                                 const uint64_t* __restrict__ bar, uint64_t seed, uint32_t obj, uint32_t purpose,
                                 RowJ rj)
{
    const uint32_t row = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t pi = map.p[row % map.n];
    uint4 r = draw(seed, i, rj.j[row], obj, purpose);
    uint64_t lo = (uint64_t)r.x | ((uint64_t)r.y << 32), hi = (uint64_t)r.z | ((uint64_t)r.w << 32);
    out[(size_t)row * N + i] = barrett128(lo, hi, qs[pi], bar[2 * pi], bar[2 * pi + 1]);
}

// Rescale (Sec. 2.4), evaluation domain: out_i = (in_i - T_i) * q_l^-1 where T_i
// is the NTT mod q_i of the centered lift of the last limb (the lift, the
// transform and the division run as one forward transform, ntt_forward_rescale).
// input polynomial pp of a stack of ciphertexts with ppc polynomials each,
// `stride` words apart
__device__ __forceinline__ const uint64_t* stack_poly(const uint64_t* in, uint32_t pp, uint32_t ppc, size_t stride,
                                                      uint32_t level, uint32_t N)
{
    return in + (size_t)(pp / ppc) * stride + (size_t)(pp % ppc) * (level + 1) * N;
}

__global__ void k_copy_last(uint64_t* __restrict__ dst, const uint64_t* __restrict__ in, uint32_t N, uint32_t level,
                            uint32_t ppc, size_t stride)
{
    const uint32_t poly = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    dst[(size_t)poly * N + c] = stack_poly(in, poly, ppc, stride, level, N)[(size_t)level * N + c];
}

__global__ void k_tensor(uint64_t* __restrict__ out, const uint64_t* __restrict__ a, const uint64_t* __restrict__ b,
                         const uint64_t* __restrict__ qs, const uint64_t* __restrict__ bar, uint32_t N, uint32_t n)
{
    const uint32_t i = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const uint64_t q = qs[i], r0 = bar[2 * i], r1 = bar[2 * i + 1];
    const size_t o0 = (size_t)i * N + c, o1 = ((size_t)n + i) * N + c;
    uint64_t a0 = a[o0], a1 = a[o1], b0 = b[o0], b1 = b[o1];
    acc128 x{0, 0};
    mad128(x, a0, b1);
    mad128(x, a1, b0);
    out[o0] = mul_mod(a0, b0, q, r0, r1);
    out[o1] = barrett128(x.lo, x.hi, q, r0, r1);
    out[((size_t)2 * n + i) * N + c] = mul_mod(a1, b1, q, r0, r1);
}

}  // namespace

int launch_mul_rows(blb_ctx* ctx, uint64_t* out, const uint64_t* a, const uint64_t* b, uint32_t rows,
                    const LimbMap& map, uint32_t b_rows)
{
    if (!rows) return BLB_OK;
    k_mul_rows<<<grid_rows(ctx->N, rows), kT, 0, ctx->stream>>>(out, a, b, map, ctx->d_q, ctx->d_bar, ctx->N,
                                                               b_rows ? b_rows : rows, 0);
    BLB_LAUNCHED();
    return BLB_OK;
}

int launch_mac_rows(blb_ctx* ctx, uint64_t* acc, const uint64_t* a, const uint64_t* b, uint32_t rows,
                    const LimbMap& map, uint32_t b_rows)
{
    if (!rows) return BLB_OK;
    k_mul_rows<<<grid_rows(ctx->N, rows), kT, 0, ctx->stream>>>(acc, a, b, map, ctx->d_q, ctx->d_bar, ctx->N,
                                                               b_rows ? b_rows : rows, 1);
    BLB_LAUNCHED();
    return BLB_OK;
}

int launch_add_rows(blb_ctx* ctx, uint64_t* out, const uint64_t* a, const uint64_t* b, uint32_t rows,
                    const LimbMap& map)
{
    if (!rows) return BLB_OK;
    k_addsub_rows<<<grid_rows(ctx->N, rows), kT, 0, ctx->stream>>>(out, a, b, map, ctx->d_q, ctx->N, 0);
    BLB_LAUNCHED();
    return BLB_OK;
}

int launch_sub_rows(blb_ctx* ctx, uint64_t* out, const uint64_t* a, const uint64_t* b, uint32_t rows,
                    const LimbMap& map)
{
    if (!rows) return BLB_OK;
    k_addsub_rows<<<grid_rows(ctx->N, rows), kT, 0, ctx->stream>>>(out, a, b, map, ctx->d_q, ctx->N, 1);
    BLB_LAUNCHED();
    return BLB_OK;
}

int launch_neg_rows(blb_ctx* ctx, uint64_t* out, const uint64_t* a, uint32_t rows, const LimbMap& map)
{
    if (!rows) return BLB_OK;
    k_addsub_rows<<<grid_rows(ctx->N, rows), kT, 0, ctx->stream>>>(out, a, a, map, ctx->d_q, ctx->N, 2);
    BLB_LAUNCHED();
    return BLB_OK;
}

int launch_mul_const_rows(blb_ctx* ctx, uint64_t* out, const uint64_t* a, uint32_t rows, const LimbMap& map,
                          const uint64_t* consts)
{
    if (!rows) return BLB_OK;
    if (rows > BLB_MAXP * 4) return blb_fail(BLB_ERR_ARG, "too many rows for one constant-product launch");
    RowConst rc{};
    for (uint32_t r = 0; r < rows; r++) {
        uint64_t q = ctx->q[map.p[r % map.n]];
        rc.w[r] = consts[r] % q;
        rc.wp[r] = shoup_companion(rc.w[r], q);
    }
    k_mul_const_rows<<<grid_rows(ctx->N, rows), kT, 0, ctx->stream>>>(out, a, map, ctx->d_q, ctx->N, rc);
    BLB_LAUNCHED();
    return BLB_OK;
}

int launch_automorph_ntt(blb_ctx* ctx, uint64_t* out, const uint64_t* in, uint32_t rows, uint64_t g)
{
    if (!rows) return BLB_OK;
    k_automorph_ntt<<<grid_rows(ctx->N, rows), kT, 0, ctx->stream>>>(out, in, ctx->logN, g);
    BLB_LAUNCHED();
    return BLB_OK;
}

int launch_signed_to_rows(blb_ctx* ctx, uint64_t* out, const int64_t* in, uint32_t rows, const LimbMap& map)
{
    if (!rows) return BLB_OK;
    k_signed_to_rows<<<grid_rows(ctx->N, rows), kT, 0, ctx->stream>>>(out, in, map, ctx->d_q, ctx->d_bar, ctx->N);
    BLB_LAUNCHED();
    return BLB_OK;
}

int launch_sample_ternary(blb_ctx* ctx, int64_t* out, uint64_t seed, uint32_t obj, uint32_t purpose, uint32_t j)
{
    k_sample_ternary<<<(ctx->N + kT - 1) / kT, kT, 0, ctx->stream>>>(out, ctx->N, seed, obj, purpose, j);
    BLB_LAUNCHED();
    return BLB_OK;
}

int launch_sample_gauss(blb_ctx* ctx, int64_t* out, uint64_t seed, uint32_t obj, uint32_t purpose, uint32_t j)
{
    k_sample_gauss<<<(ctx->N + kT - 1) / kT, kT, 0, ctx->stream>>>(out, ctx->N, ctx->d_cdt, seed, obj, purpose, j);
    BLB_LAUNCHED();
    return BLB_OK;
}

int launch_sample_uniform(blb_ctx* ctx, uint64_t* out, uint32_t rows, const LimbMap& map, uint64_t seed,
                          uint32_t obj, uint32_t purpose, const uint32_t* j_of_row)
{
    if (!rows) return BLB_OK;
    if (rows > BLB_MAXP * 4) return blb_fail(BLB_ERR_ARG, "too many rows for one sampling launch");
    RowJ rj{};
    for (uint32_t r = 0; r < rows; r++) rj.j[r] = j_of_row[r];
    k_sample_uniform<<<grid_rows(ctx->N, rows), kT, 0, ctx->stream>>>(out, ctx->N, map, ctx->d_q, ctx->d_bar, seed,
                                                                      obj, purpose, rj);
    BLB_LAUNCHED();
    return BLB_OK;
}

// in: npolys x (level+1) rows; out: npolys x level rows (may not alias in).
// Temporaries: npolys rows (last limb) + npolys*level rows, in the operation
// scratch when they fit, else in a temporary allocation.
int launch_rescale_stack(blb_ctx* ctx, uint64_t* out, const uint64_t* in, uint32_t level, uint32_t npolys)
{
    return launch_rescale_strided(ctx, out, in, level, npolys, npolys, 0);
}

// npolys polynomials taken from ciphertexts of ppc polynomials that lie
// `stride` words apart in `in` (0: back to back); out is one contiguous stack
int launch_rescale_strided(blb_ctx* ctx, uint64_t* out, const uint64_t* in, uint32_t level, uint32_t npolys,
                           uint32_t ppc, size_t stride)
{
    if (stride == 0) stride = (size_t)ppc * (level + 1) * ctx->N;
    if (level == 0) return blb_fail(BLB_ERR_LEVEL, "rescale at level 0");
    const uint32_t N = ctx->N;
    const size_t need = (size_t)npolys * (level + 1) * N;
    const size_t have = ctx->scratch_words - ctx->ks_words();
    uint64_t* tmp = nullptr;
    uint64_t* last = ctx->op_scratch();
    if (need > have) {
        tmp = (uint64_t*)dev_alloc(ctx, need * 8);
        if (!tmp) return blb_fail(BLB_ERR_OOM, "rescale temporary");
        last = tmp;
    }
    uint64_t* T = last + (size_t)npolys * N;
    int rc = BLB_OK;
    do {
        k_copy_last<<<grid_rows(N, npolys), kT, 0, ctx->stream>>>(last, in, N, level, ppc, stride);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "rescale launch failed"); break; }
        blb_count_launch();
        if ((rc = ntt_inverse(ctx, last, npolys, ctx->qmap(1, level)))) break;
        // the lift of the last limb, its forward transforms and the division
        // by q_level in one transform (T holds the rows between its passes)
        RescaleIO rs{};
        rs.last = last;
        rs.in = in;
        rs.out = out;
        rs.stride = stride;
        rs.level = level;
        rs.ppc = ppc;
        rs.inv = ctx->d_ql_inv + (size_t)level * ctx->nQ * 2;
        if ((rc = ntt_forward_rescale(ctx, T, npolys * level, rs))) break;
    } while (0);
    if (tmp) dev_free(ctx, tmp, need * 8);
    return rc;
}

int launch_rescale(blb_ctx* ctx, uint64_t* out, const uint64_t* in, uint32_t level, uint32_t npolys)
{
    return launch_rescale_stack(ctx, out, in, level, npolys);
}

int launch_tensor(blb_ctx* ctx, uint64_t* out, const uint64_t* a, const uint64_t* b, uint32_t level)
{
    k_tensor<<<grid_rows(ctx->N, level + 1), kT, 0, ctx->stream>>>(out, a, b, ctx->d_q, ctx->d_bar, ctx->N,
                                                                   level + 1);
    BLB_LAUNCHED();
    return BLB_OK;
}
