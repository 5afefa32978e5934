// encode.cu -- CKKS encoding / decoding (Sec. 6.1, Eq. 2) and the plaintext
// diagonals of matmul_cp.
//
// Slot j of a real polynomial m is m(zeta^(5^j)), zeta = exp(i pi / N), j < s = N/2
// (real slots, footnote to Eq. 2).  With v_t = m_t + i m_{t+s}, slot j equals
// sum_t v_t zeta^(t 5^j): an s-point DFT (root omega = zeta^4) of v_t zeta^t
// read at k_j = (5^j - 1)/4.  Encoding inverts it: V[k_j] = z_j, inverse DFT,
// c_t = a_t zeta^-t, m_t = round(Re c_t * scale/s), m_{t+s} = round(Im c_t * scale/s),
// rounding half to even, then residues mod each prime and the NTT.
//
// The DFT is the radix-2 decimation-in-time network on bit-reversed input:
// stage len = 2, 4, ..., s pairs (i + j, i + j + len/2) with twiddle
// zeta^(4 j s/len) (conjugated for the inverse), product (ac - bd, ad + bc).
// Every product and sum is an IEEE round-to-nearest operation (__dmul_rn,
// __dadd_rn, __dsub_rn: nothing is contracted into fused multiply-adds), so the
// result is a fixed function of the inputs, the same for any thread schedule.
// The first stages (len <= kChunk) run in shared memory on contiguous chunks,
// the later ones on column tiles {c + kChunk r}.
#include "common.cuh"

namespace {
constexpr int kT = 256;
constexpr uint32_t kChunk = 2048;  // complex values per CTA (32 KB)

__device__ __forceinline__ double2 cmul(double2 x, double2 w)
{
    double t1 = __dmul_rn(x.x, w.x), t2 = __dmul_rn(x.y, w.y);
    double t3 = __dmul_rn(x.x, w.y), t4 = __dmul_rn(x.y, w.x);
    return make_double2(__dsub_rn(t1, t2), __dadd_rn(t3, t4));
}

__device__ __forceinline__ void butterfly(double2& lo, double2& hi, double2 w)
{
    double2 u = lo, v = cmul(hi, w);
    lo = make_double2(__dadd_rn(u.x, v.x), __dadd_rn(u.y, v.y));
    hi = make_double2(__dsub_rn(u.x, v.x), __dsub_rn(u.y, v.y));
}

// A[pt][brv(k_j)] = (z[pt][j], 0) for j < n, zero elsewhere
__global__ void k_scatter_slots(double2* __restrict__ A, const double* __restrict__ z, uint32_t n, uint32_t logs,
                                const uint32_t* __restrict__ kperm)
{
    const uint32_t s = 1u << logs;
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x, pt = blockIdx.y;
    if (j >= s) return;
    const uint32_t k = kperm[j];
    const uint32_t pos = __brev(k) >> (32 - logs);
    A[(size_t)pt * s + pos] = make_double2(j < n ? z[(size_t)pt * n + j] : 0.0, 0.0);
}

// stages len = 2 .. min(s, kChunk) on contiguous chunks
__global__ void __launch_bounds__(kT) k_dit_chunks(double2* __restrict__ A, uint32_t logs,
                                                   const double2* __restrict__ zeta, int inverse)
{
    __shared__ double2 sm[kChunk];
    const uint32_t s = 1u << logs, C = s < kChunk ? s : kChunk;
    double2* a = A + (size_t)blockIdx.y * s + (size_t)blockIdx.x * C;
    for (uint32_t i = threadIdx.x; i < C; i += blockDim.x) sm[i] = a[i];
    __syncthreads();
    for (uint32_t len = 2; len <= C; len <<= 1) {
        const uint32_t half = len / 2, step = s / len;
        for (uint32_t idx = threadIdx.x; idx < C / 2; idx += blockDim.x) {
            uint32_t grp = idx / half, j = idx % half;
            uint32_t lo = grp * len + j;
            double2 w = zeta[4 * j * step];
            if (inverse) w.y = -w.y;
            butterfly(sm[lo], sm[lo + half], w);
        }
        __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < C; i += blockDim.x) a[i] = sm[i];
}

// stages len = 2 kChunk .. s on column tiles: element (r, c) = A[c + kChunk r]
__global__ void __launch_bounds__(kT) k_dit_cols(double2* __restrict__ A, uint32_t logs,
                                                 const double2* __restrict__ zeta, int inverse)
{
    __shared__ double2 sm[kChunk];
    const uint32_t s = 1u << logs, R = s / kChunk, cols = kChunk / R;
    double2* a = A + (size_t)blockIdx.y * s;
    const uint32_t c0 = blockIdx.x * cols;
    for (uint32_t idx = threadIdx.x; idx < R * cols; idx += blockDim.x) {
        uint32_t r = idx / cols, c = idx % cols;
        sm[idx] = a[(size_t)r * kChunk + c0 + c];
    }
    __syncthreads();
    for (uint32_t len = 2 * kChunk; len <= s; len <<= 1) {
        const uint32_t half_r = len / (2 * kChunk), step = s / len;
        for (uint32_t idx = threadIdx.x; idx < (R / 2) * cols; idx += blockDim.x) {
            uint32_t c = idx % cols, bf = idx / cols;
            uint32_t grp = bf / half_r, jr = bf % half_r;
            uint32_t r = grp * 2 * half_r + jr;
            uint32_t j = c0 + c + kChunk * jr;  // lower element's index mod len
            double2 w = zeta[4 * j * step];
            if (inverse) w.y = -w.y;
            butterfly(sm[r * cols + c], sm[(r + half_r) * cols + c], w);
        }
        __syncthreads();
    }
    for (uint32_t idx = threadIdx.x; idx < R * cols; idx += blockDim.x) {
        uint32_t r = idx / cols, c = idx % cols;
        a[(size_t)r * kChunk + c0 + c] = sm[idx];
    }
}

// twist by zeta^-t, scale, round half to even, residues: out[pt][i][t], [t+s]
__global__ void k_twist_round(uint64_t* __restrict__ out, const double2* __restrict__ A, uint32_t logs,
                              const double2* __restrict__ zeta, double f, uint32_t nlimbs,
                              const uint64_t* __restrict__ qs, const uint64_t* __restrict__ bar,
                              int* __restrict__ overflow)
{
    const uint32_t s = 1u << logs, N = 2 * s;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, pt = blockIdx.y;
    if (t >= s) return;
    double2 w = zeta[t];
    w.y = -w.y;
    double2 c = cmul(A[(size_t)pt * s + t], w);
    double re = __dmul_rn(c.x, f), im = __dmul_rn(c.y, f);
    if (fabs(re) >= 9.2e18 || fabs(im) >= 9.2e18) *overflow = 1;
    long long mr = __double2ll_rn(re), mi = __double2ll_rn(im);
    for (uint32_t i = 0; i < nlimbs; i++) {
        const uint64_t q = qs[i], rb = bar[2 * i + 1];
        const uint64_t r0 = signed_mod(mr, q, rb), r1 = signed_mod(mi, q, rb);
        uint64_t* o = out + ((size_t)pt * nlimbs + i) * N;
        o[t] = r0;
        o[t + s] = r1;
    }
}

// decode: A[brv(t)] = (m_t, m_{t+s}) zeta^t from the centered q_0 limb
__global__ void k_decode_gather(double2* __restrict__ A, const uint64_t* __restrict__ coef, uint64_t q0,
                                uint32_t logs, const double2* __restrict__ zeta)
{
    const uint32_t s = 1u << logs;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= s) return;
    uint64_t a = coef[t], b = coef[t + s];
    double re = a > q0 / 2 ? -(double)(q0 - a) : (double)a;
    double im = b > q0 / 2 ? -(double)(q0 - b) : (double)b;
    A[__brev(t) >> (32 - logs)] = cmul(make_double2(re, im), zeta[t]);
}

__global__ void k_decode_finish(double* __restrict__ z, const double2* __restrict__ A, uint32_t logs,
                                const uint32_t* __restrict__ kperm, double scale)
{
    const uint32_t s = 1u << logs;
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= s) return;
    z[j] = __ddiv_rn(A[kperm[j]].x, scale);
}

// matmul_cp plaintext diagonal for plan index p = ((e G + g) nX + c) b1 + b:
// slot i + m beta holds W[c k + (beta + b) mod k][e k + (beta - g b1) mod k]
__global__ void k_cp_diag(double* __restrict__ z, const double* __restrict__ W, uint32_t m, uint32_t d,
                          uint32_t d_out, uint32_t k, uint32_t b1, uint32_t G, uint32_t nX, uint32_t first)
{
    const uint32_t s = m * k;
    const uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x, pl = blockIdx.y;
    if (slot >= s) return;
    const uint32_t p = first + pl;
    const uint32_t b = p % b1, c = (p / b1) % nX, g = (p / (b1 * nX)) % G, e = p / (b1 * nX * G);
    const uint32_t beta = slot / m;
    const uint32_t row = c * k + (beta + b) % k;
    const uint32_t col = e * k + (beta + k - (g * b1) % k) % k;
    z[(size_t)pl * s + slot] = (row < d && col < d_out) ? W[(size_t)row * d_out + col] : 0.0;
}

// Diagonal-input weights (App. C.2): input column r holds head head[r] and
// dense diagonal delta[r] of Att in diagonal packing; the weight at row i is
// W[head Dh + (i + delta) mod Dh][col].
__global__ void k_cp_diag_rows(double* __restrict__ z, const double* __restrict__ W, uint32_t m, uint32_t d_out,
                               uint32_t k, uint32_t b1, uint32_t G, uint32_t nX, uint32_t first,
                               const int32_t* __restrict__ head, const int32_t* __restrict__ delta, uint32_t Dh)
{
    const uint32_t s = m * k;
    const uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x, pl = blockIdx.y;
    if (slot >= s) return;
    const uint32_t p = first + pl;
    const uint32_t b = p % b1, c = (p / b1) % nX, g = (p / (b1 * nX)) % G, e = p / (b1 * nX * G);
    const uint32_t beta = slot / m, i = slot % m;
    const uint32_t r = c * k + (beta + b) % k;
    const uint32_t col = e * k + (beta + k - (g * b1) % k) % k;
    double w = 0.0;
    if (col < d_out && head[r] >= 0)
        w = W[((size_t)head[r] * Dh + (i + (uint32_t)delta[r]) % Dh) * d_out + col];
    z[(size_t)pl * s + slot] = w;
}

int run_dit(blb_ctx* ctx, double2* A, uint32_t npts, int inverse, const double2* zeta)
{
    const uint32_t logs = ctx->logN - 1, s = 1u << logs;
    const uint32_t C = s < kChunk ? s : kChunk;
    k_dit_chunks<<<dim3(s / C, npts), kT, 0, ctx->stream>>>(A, logs, zeta, inverse);
    BLB_LAUNCHED();
    if (s > kChunk) {
        const uint32_t R = s / kChunk, cols = kChunk / R;
        k_dit_cols<<<dim3(kChunk / cols, npts), kT, 0, ctx->stream>>>(A, logs, zeta, inverse);
        BLB_LAUNCHED();
    }
    return BLB_OK;
}

}  // namespace

int encode_slots(blb_ctx* ctx, const double* d_z, uint32_t npts, uint32_t n, uint32_t level, double scale,
                 uint64_t* d_out)
{
    if (npts == 0) return BLB_OK;
    if (capturing(ctx))  // the overflow flag is read back on the host
        return blb_fail(BLB_ERR_ARG, "encoding cannot run inside a graph capture");
    const uint32_t logs = ctx->logN - 1, s = 1u << logs, nl = level + 1;
    if (n > s) return blb_fail(BLB_ERR_ARG, "more values than slots");
    const size_t words = (size_t)npts * s * 2;  // double2 per slot
    const size_t op_words = ctx->scratch_words - ctx->ks_words();
    double2* A;
    bool own = words > op_words;
    if (own) {
        A = (double2*)dev_alloc(ctx, words * 8);
        if (!A) return blb_fail(BLB_ERR_OOM, "encoding buffer allocation failed");
    } else {
        A = (double2*)ctx->op_scratch();
    }
    int rc = BLB_OK;
    do {
        k_scatter_slots<<<dim3((s + kT - 1) / kT, npts), kT, 0, ctx->stream>>>(A, d_z, n, logs, ctx->d_kperm);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "scatter launch failed"); break; }
        if ((rc = run_dit(ctx, A, npts, 1, ctx->d_zeta))) break;
        // deferred checks: the flag accumulates until blb_ctx_sync reads it
        int* flag_dev = ctx->encode_deferred ? ctx->d_flag_deferred : ctx->d_flag;
        if (!ctx->encode_deferred && cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream) != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "memset failed"); break; }
        const double f = scale / (double)s;
        k_twist_round<<<dim3((s + kT - 1) / kT, npts), kT, 0, ctx->stream>>>(d_out, A, logs, ctx->d_zeta, f, nl,
                                                                            ctx->d_q, ctx->d_bar, flag_dev);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "twist launch failed"); break; }
        if ((rc = ntt_forward(ctx, d_out, npts * nl, ctx->qmap(nl)))) break;
        if (ctx->encode_deferred) break;
        int flag = 0;
        if (cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "encode sync failed"); break; }
        if (flag) rc = blb_fail(BLB_ERR_ARG, "encoded coefficient exceeds 2^63: value * scale too large");
    } while (0);
    if (own) {
        dev_free(ctx, A, words * 8);
    }
    return rc;
}

int decode_limb0(blb_ctx* ctx, const uint64_t* d_coef0, double scale, double* d_slots)
{
    const uint32_t logs = ctx->logN - 1, s = 1u << logs;
    double2* A = (double2*)(ctx->op_scratch() + (size_t)3 * ctx->nQ * ctx->N);  // decoding row of the operation scratch
    k_decode_gather<<<(s + kT - 1) / kT, kT, 0, ctx->stream>>>(A, d_coef0, ctx->q[0], logs, ctx->d_zeta);
    BLB_LAUNCHED();
    BLB_TRY(run_dit(ctx, A, 1, 0, ctx->d_zeta));
    k_decode_finish<<<(s + kT - 1) / kT, kT, 0, ctx->stream>>>(d_slots, A, logs, ctx->d_kperm, scale);
    BLB_LAUNCHED();
    return BLB_OK;
}

int cp_build_diagonals(blb_ctx* ctx, const blb_cp_plan* plan, const double* d_W, uint32_t first, uint32_t count,
                       double* d_z, const int32_t* d_head, const int32_t* d_delta, uint32_t Dh)
{
    const uint32_t s = ctx->N / 2;
    if (d_head)
        k_cp_diag_rows<<<dim3((s + kT - 1) / kT, count), kT, 0, ctx->stream>>>(
            d_z, d_W, plan->m, plan->d_out, plan->k, plan->b1, plan->G, plan->nX, first, d_head, d_delta, Dh);
    else
        k_cp_diag<<<dim3((s + kT - 1) / kT, count), kT, 0, ctx->stream>>>(d_z, d_W, plan->m, plan->d, plan->d_out,
                                                                        plan->k, plan->b1, plan->G, plan->nX, first);
    BLB_LAUNCHED();
    return BLB_OK;
}
