// keyswitch.cu -- hybrid key switching (decompose into dnum digits, ModUp by
// fast base conversion, inner product with the key, ModDown by P).
//
// The paper's rotations and ct-ct products (Sec. 2.4) need key switching but do
// not restate it; this is the standard hybrid method.  For a polynomial d at
// level l (n = l+1 primes) and a key {(b_j, a_j)} from s' to s:
//   digits D_j = {j alpha, ..., min((j+1) alpha, n) - 1}, j < beta = ceil(n/alpha)
//   d~_j = Conv_{D_j -> Q_l u P}([d]_{D_j})   (the digit's own primes keep d)
//   acc  = sum_j d~_j (b_j, a_j)              (over Q_l u P)
//   out_i = (acc_i - X_i) * P^-1 mod q_i = round(acc / P) mod q_i, X the centered
//           representative of acc mod P (k_moddown_conv)
// Conv(x)_t = sum_i [x_i (S/s_i)^-1]_{s_i} (S/s_i mod t) mod t, the ModUp
// conversion, without overflow correction (the overflow is a multiple of the
// digit modulus, which the key's gadget factor cancels).  Every step is an exact integer function of d's
// coefficients, so any correct schedule of it yields the same limbs.
#include <algorithm>
#include <cstring>
#include <string>

#include "common.cuh"

namespace {
constexpr int kT = 256;

// Base conversion of `npolys` polynomials: sources are tab.ns consecutive rows
// at src (poly stride src_ps words), targets 0..nt-1 of the table written to
// dst rows tab.dst_row[k] (poly stride dst_ps words).  Coefficient form.
__global__ void k_conv(const uint64_t* __restrict__ src, size_t src_ps, const ConvTable* __restrict__ tab,
                       uint32_t nt, uint64_t* __restrict__ dst, size_t dst_ps, const uint64_t* __restrict__ qs,
                       const uint64_t* __restrict__ bar, uint32_t N)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x, poly = blockIdx.y;
    if (c >= N) return;
    const uint32_t ns = tab->ns;
    uint64_t y[BLB_MAXP];
    for (uint32_t i = 0; i < ns; i++) {
        uint64_t si = qs[tab->src[i]];
        y[i] = mul_shoup(src[poly * src_ps + (size_t)i * N + c], tab->hat_inv[i], tab->hat_inv_sh[i], si);
    }
    for (uint32_t k = 0; k < nt; k++) {
        const uint32_t pt = tab->dst[k];
        acc128 a{0, 0};
        for (uint32_t i = 0; i < ns; i++) mad128(a, y[i], tab->hat[i][k]);
        dst[poly * dst_ps + (size_t)tab->dst_row[k] * N + c] = barrett128(a.lo, a.hi, qs[pt], bar[2 * pt], bar[2 * pt + 1]);
    }
}

// ModDown conversion with rounding (Halevi, Polyakov, Shoup 2019): for the P
// limbs x_k, y_k = [x_k (P/p_k)^-1]_{p_k}, v = round(sum_k y_k / p_k), and
// X = sum_k y_k (P/p_k) - v P is the representative of x mod P in (-P/2, P/2];
// dst row t gets X mod q_t.  The sum is taken in 128-bit fixed point, y_k / p_k
// as y_k floor(2^128 / p_k) (the Barrett constant of p_k, below 2^128 since
// y_k < p_k) with the carries counted: the exact rounding unless the fraction
// is within 2^-65 of 1/2, and no FP64 (a small fraction of B300's integer rate).
// NS > 0: at most NS source primes, the y_k in registers (NS = 0: any count,
// the y_k in a local array).  PRE: the source rows already hold y_k (the
// inverse NTT that produced them multiplied by (P/p_k)^-1 with N^-1).
template <int NS, bool PRE>
__global__ void k_moddown_conv(const uint64_t* __restrict__ src, size_t src_ps, const ConvTable* __restrict__ tab,
                               uint32_t nt, uint64_t* __restrict__ dst, size_t dst_ps,
                               const uint64_t* __restrict__ qs, const uint64_t* __restrict__ bar, uint32_t N)
{
    constexpr int YN = NS > 0 ? NS : BLB_MAXP;
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x, poly = blockIdx.y;
    if (c >= N) return;
    const uint32_t ns = tab->ns;
    uint64_t y[YN];
    uint64_t f_lo = 0, f_hi = 0, whole = 0;
#pragma unroll
    for (uint32_t k = 0; k < (NS > 0 ? (uint32_t)NS : ns); k++) {
        if (k >= ns) break;
        const uint32_t pk_i = tab->src[k];
        const uint64_t x = src[poly * src_ps + (size_t)k * N + c];
        y[k] = PRE ? x : mul_shoup(x, tab->hat_inv[k], tab->hat_inv_sh[k], qs[pk_i]);
        const uint64_t b0 = bar[2 * pk_i], b1 = bar[2 * pk_i + 1];
        const uint64_t lo = y[k] * b0, hi = __umul64hi(y[k], b0) + y[k] * b1;  // y_k floor(2^128/p_k)
        const uint64_t s_lo = f_lo + lo;
        const uint64_t c0 = s_lo < f_lo;
        const uint64_t s_hi = f_hi + hi;
        const uint64_t c1 = s_hi < f_hi;
        const uint64_t s_hi2 = s_hi + c0;
        whole += c1 + (s_hi2 < s_hi);
        f_lo = s_lo;
        f_hi = s_hi2;
    }
    const uint64_t v = whole + (f_hi >> 63);
    for (uint32_t t = 0; t < nt; t++) {
        const uint32_t pt = tab->dst[t];
        const uint64_t q = qs[pt], r0 = bar[2 * pt], r1 = bar[2 * pt + 1];
        // sum_k y_k (P/p_k) - v P, the subtraction folded into the lazy sum as
        // v (q_t - P mod q_t): one reduction per target
        acc128 a{0, 0};
#pragma unroll
        for (uint32_t k = 0; k < (NS > 0 ? (uint32_t)NS : ns); k++) {
            if (k >= ns) break;
            mad128(a, y[k], tab->hat[k][t]);
        }
        mad128(a, v, tab->neg_prod_mod_t[t]);
        dst[poly * dst_ps + (size_t)tab->dst_row[t] * N + c] = barrett128(a.lo, a.hi, q, r0, r1);
    }
}

// launches with the register form when the source count allows it (ModDown: nP
// sources; ModUp below: alpha)
template <bool PRE, typename... Args>
void launch_moddown_conv(uint32_t ns, dim3 grid, cudaStream_t st, Args... args)
{
    switch (ns) {
    case 1: k_moddown_conv<1, PRE><<<grid, kT, 0, st>>>(args...); break;
    case 2: k_moddown_conv<2, PRE><<<grid, kT, 0, st>>>(args...); break;
    case 3: k_moddown_conv<3, PRE><<<grid, kT, 0, st>>>(args...); break;
    case 4: k_moddown_conv<4, PRE><<<grid, kT, 0, st>>>(args...); break;
    default: k_moddown_conv<0, PRE><<<grid, kT, 0, st>>>(args...); break;
    }
}

// acc_p[t] = sum_{j < beta} ext[j][t] * key[j][p][kt],  p in {0, 1}
__global__ void k_ks_inner(uint64_t* __restrict__ acc, const uint64_t* __restrict__ ext,
                           const uint64_t* __restrict__ key, const __grid_constant__ LimbMap emap, uint32_t n, uint32_t E, uint32_t beta,
                           uint32_t nQ, uint32_t np, const uint64_t* __restrict__ qs,
                           const uint64_t* __restrict__ bar, uint32_t N)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x, t = blockIdx.y;
    if (c >= N) return;
    const uint32_t pi = emap.p[t];
    const uint32_t kt = t < n ? t : nQ + (t - n);
    acc128 a0{0, 0}, a1{0, 0};
    for (uint32_t j = 0; j < beta; j++) {
        uint64_t x = ext[((size_t)j * E + t) * N + c];
        mad128(a0, x, key[(((size_t)j * 2 + 0) * np + kt) * N + c]);
        mad128(a1, x, key[(((size_t)j * 2 + 1) * np + kt) * N + c]);
    }
    const uint64_t q = qs[pi], r0 = bar[2 * pi], r1 = bar[2 * pi + 1];
    acc[(size_t)t * N + c] = barrett128(a0.lo, a0.hi, q, r0, r1);
    acc[((size_t)E + t) * N + c] = barrett128(a1.lo, a1.hi, q, r0, r1);
}

struct PInv {
    uint64_t w[BLB_MAXP], wp[BLB_MAXP];
};
// out_p[i] = (acc_p[i] - cv_p[i]) * P^-1 mod q_i
__global__ void k_moddown_finish(uint64_t* __restrict__ out0, uint64_t* __restrict__ out1,
                                 const uint64_t* __restrict__ acc, const uint64_t* __restrict__ cv, uint32_t n,
                                 uint32_t E, PInv pinv, const uint64_t* __restrict__ qs, uint32_t N)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y;  // row = p * n + i
    if (c >= N) return;
    const uint32_t p = row / n, i = row % n;
    const uint64_t q = qs[i];
    uint64_t x = acc[((size_t)p * E + i) * N + c];
    uint64_t v = cv[(size_t)row * N + c];
    uint64_t r = mul_shoup(sub_mod(x, v, q), pinv.w[i], pinv.wp[i], q);
    (p ? out1 : out0)[(size_t)i * N + c] = r;
}

}  // namespace

// Key-switch body on an explicit scratch area of ks_scratch_words(level) words.
static int keyswitch_impl(blb_ctx* ctx, const uint64_t* d_ntt, uint32_t level, const uint64_t* key, uint64_t* out0,
                          uint64_t* out1, uint64_t* scratch, bool profile)
{
    const uint32_t N = ctx->N, n = level + 1, nP = ctx->nP, E = n + nP;
    const uint32_t alpha = ctx->alpha, beta = (n + alpha - 1) / alpha;
    // algorithmic bytes: read d and the used key digits, write (k0, k1)
    ProfScope prof(profile ? ctx : nullptr, "keyswitch", ((uint64_t)n + 2ull * beta * E + 2ull * n) * N * 8);
    uint64_t* coef = scratch;
    uint64_t* ext = coef + (size_t)n * N;
    uint64_t* acc = ext + (size_t)beta * E * N;
    uint64_t* cv = acc + (size_t)2 * E * N;
    const LimbMap emap = ctx->extmap(level);
    const dim3 g1((N + kT - 1) / kT, 1);

    // 1. coefficient form of d
    BLB_CUDA(cudaMemcpyAsync(coef, d_ntt, (size_t)n * N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    BLB_TRY(ntt_inverse(ctx, coef, n, ctx->qmap(n)));
    // 2. ModUp of every digit, then back to the evaluation domain
    for (uint32_t j = 0; j < beta; j++) {
        const uint32_t lo = j * alpha, hi = std::min((j + 1) * alpha, n);
        const ConvTable& h = ctx->h_modup[(size_t)level * ctx->dnum + j];
        uint64_t* ej = ext + (size_t)j * E * N;
        k_conv<<<g1, kT, 0, ctx->stream>>>(coef + (size_t)lo * N, 0, ctx->d_modup[(size_t)level * ctx->dnum + j], h.nt,
                                           ej, 0, ctx->d_q, ctx->d_bar, N);
        BLB_LAUNCHED();
        if (lo > 0) BLB_TRY(ntt_forward(ctx, ej, lo, ctx->qmap(lo)));
        LimbMap tail{};
        for (uint32_t r = hi; r < E; r++) tail.p[r - hi] = emap.p[r];
        tail.n = E - hi;
        BLB_TRY(ntt_forward(ctx, ej + (size_t)hi * N, E - hi, tail));
        BLB_CUDA(cudaMemcpyAsync(ej + (size_t)lo * N, d_ntt + (size_t)lo * N, (size_t)(hi - lo) * N * 8,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
    }
    // 3. inner product with the key
    k_ks_inner<<<dim3((N + kT - 1) / kT, E), kT, 0, ctx->stream>>>(acc, ext, key, emap, n, E, beta, ctx->nQ, ctx->np,
                                                                   ctx->d_q, ctx->d_bar, N);
    BLB_LAUNCHED();
    // 4. ModDown: P limbs to coefficient form, convert to Q_l, back to evaluation
    BLB_TRY(ntt_inverse(ctx, acc + (size_t)n * N, nP, ctx->pmap()));
    BLB_TRY(ntt_inverse(ctx, acc + ((size_t)E + n) * N, nP, ctx->pmap()));
    launch_moddown_conv<false>(nP, dim3((N + kT - 1) / kT, 2), ctx->stream, (const uint64_t*)(acc + (size_t)n * N),
                        (size_t)E * N, (const ConvTable*)ctx->d_moddown, n, cv, (size_t)n * N,
                        (const uint64_t*)ctx->d_q, (const uint64_t*)ctx->d_bar, N);
    BLB_LAUNCHED();
    BLB_TRY(ntt_forward(ctx, cv, 2 * n, ctx->qmap(n)));
    PInv pinv{};
    for (uint32_t i = 0; i < n; i++) {
        pinv.w[i] = ctx->P_inv_mod_q[i];
        pinv.wp[i] = shoup_companion(pinv.w[i], ctx->q[i]);
    }
    k_moddown_finish<<<dim3((N + kT - 1) / kT, 2 * n), kT, 0, ctx->stream>>>(out0, out1, acc, cv, n, E, pinv,
                                                                             ctx->d_q, N);
    BLB_LAUNCHED();
    return BLB_OK;
}

int keyswitch(blb_ctx* ctx, const uint64_t* d_ntt, uint32_t level, const uint64_t* key, uint64_t* out0,
              uint64_t* out1)
{
    return keyswitch_impl(ctx, d_ntt, level, key, out0, out1, ctx->scratch, true);
}

// ===========================================================================
// Allocation-free key switching
// ===========================================================================
// Some callers cannot allocate device memory while they run: a serving process
// whose memory manager reserved the whole device budget at start-up and
// rejects any other allocation, a latency-critical loop that must not pay
// cudaMalloc's implicit device-wide synchronization, or code that runs inside
// the allocator callbacks installed with blb_set_allocator.  For them
// blb_keyswitch_noalloc keeps every temporary in the fixed array below.  The
// array is a property of the loaded library: each GPU that loads it holds these
// 32 MiB until the process exits, and all calls on one GPU share it.
static constexpr size_t kNoAllocScratchWords = (size_t)4 << 20;  // 32 MiB of uint64 words
static __device__ __align__(256) uint64_t blb_noalloc_scratch[kNoAllocScratchWords];

// The array's host-side name is not a device address.  Context creation asks
// the runtime for the real one, with the context's device current, and keeps
// it in the context; that lookup is also what loads this file's module (and
// with it the array) under lazy module loading, so the load happens there and
// not inside an allocation-free call.  The kernels of the entry point are
// loaded at the same time, for the same reason.
int keyswitch_noalloc_prepare(blb_ctx* c)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, blb_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return blb_fail(BLB_ERR_CUDA, std::string("cudaGetSymbolAddress of the key-switch scratch failed: ") +
                                          cudaGetErrorString(e));
    }
    cudaFuncAttributes fa;
    const void* kernels[] = {(const void*)k_conv,
                             (const void*)k_ks_inner,
                             (const void*)k_moddown_finish,
                             (const void*)k_moddown_conv<0, false>,
                             (const void*)k_moddown_conv<1, false>,
                             (const void*)k_moddown_conv<2, false>,
                             (const void*)k_moddown_conv<3, false>,
                             (const void*)k_moddown_conv<4, false>};
    for (const void* k : kernels) BLB_CUDA(cudaFuncGetAttributes(&fa, k));
    c->noalloc_scratch = (uint64_t*)p;
    return BLB_OK;
}

extern "C" int blb_keyswitch_noalloc(blb_ctx* c, const blb_keys* K, int32_t rot, const uint64_t* d, uint32_t level,
                                     uint64_t* out)
{
    if (c && ((d && !is_device_ptr(d)) || (out && !is_device_ptr(out))))
        BLB_TRY(refuse_capture(c, "blb_keyswitch_noalloc on host buffers"));
    if (!c || !K || !d || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (level >= c->nQ) return blb_fail(BLB_ERR_LEVEL, "level out of range");
    const KeyEntry* k = K->find(galois_element(c->N, rot));
    if (!k) return blb_fail(BLB_ERR_NO_KEY, "no Galois key for that rotation");
    const uint32_t N = c->N, n = level + 1, E = n + c->nP, beta = (n + c->alpha - 1) / c->alpha;
    // input copy (n rows) + outputs (2n rows) + key-switch body (n + beta E + 2E + 2n rows)
    const size_t need = ((size_t)3 * n + n + (size_t)beta * E + 2 * (size_t)E + 2 * (size_t)n) * N;
    if (need > kNoAllocScratchWords)
        return blb_fail(BLB_ERR_ARG, "blb_keyswitch_noalloc: this level and ring size need " +
                                         std::to_string(need * 8 >> 20) + " MiB of scratch; the fixed area holds " +
                                         std::to_string(kNoAllocScratchWords * 8 >> 20) + " MiB");
    uint64_t* S = c->noalloc_scratch;
    if (!S) return blb_fail(BLB_ERR_CUDA, "the context holds no address of the key-switch scratch array");
    uint64_t* dd = S;
    uint64_t* o = S + (size_t)n * N;
    uint64_t* body = S + (size_t)3 * n * N;
    BLB_CUDA(cudaMemcpyAsync(dd, d, (size_t)n * N * 8, cudaMemcpyDefault, c->stream));
    BLB_TRY(ntt_forward(c, dd, n, c->qmap(n)));
    BLB_TRY(keyswitch_impl(c, dd, level, k->d, o, o + (size_t)n * N, body, false));
    BLB_TRY(ntt_inverse(c, o, 2 * n, c->qmap(n)));
    BLB_CUDA(cudaMemcpyAsync(out, o, (size_t)2 * n * N * 8, cudaMemcpyDefault, c->stream));
    if (!is_device_ptr(out)) BLB_CUDA(cudaStreamSynchronize(c->stream));
    return BLB_OK;
}

// ===========================================================================
// Key-switching passes over many polynomials (one set of launches per chunk).
//
// A pass has sources, products and groups:
//   source s : a polynomial c1_s (NTT domain) and an automorphism g applied
//              before the decomposition; its extended digits are built once;
//   product x: source s, an automorphism g' applied to the extended digits
//              (hoisting: x~_j -> sigma_g'(x~_j), an index permutation in the
//              NTT domain) and a key; it contributes sum_j sigma_g'(x~_j) key_j;
//   group  G : the sum of its products over Q_l u P, one ModDown, then
//              out_p = [out_p +] sum of its addends of polynomial p (each read
//              through its own automorphism) + ModDown_p.
// One rotation is a source, a product and a group; hoisted rotations of one
// ciphertext share the source; a giant-step sum puts several products (each
// its own source) into one group.
// ===========================================================================
namespace {

using DevSource = GatherSrc;
struct DevProduct {
    uint32_t src;
    uint64_t g;
    const uint64_t* key;
    uint64_t ginv;  // g^-1 mod 2N: the output position whose digits are read at k' is perm(k', ginv)
};
struct DevGroup {
    uint64_t* out0;
    uint64_t* out1;
    uint32_t prod0, prod1, add0, add1;
};


// ModUp of every digit of every source: grid.y = source * beta + j.  The
// coefficient rows arrive as y_i = [x_i (D_j/q_i)^-1]_{q_i}: the inverse NTT
// that produced them multiplied by that factor together with N^-1.
template <int NS>  // as for k_moddown_conv: at most NS primes per digit, 0 = any
__global__ void k_ksb_modup(const uint64_t* __restrict__ coef, uint64_t* __restrict__ ext,
                            const ConvTable* __restrict__ tabs, uint32_t n, uint32_t E, uint32_t beta,
                            uint32_t alpha, const uint64_t* __restrict__ qs, const uint64_t* __restrict__ bar,
                            uint32_t N)
{
    constexpr int YN = NS > 0 ? NS : BLB_MAXP;
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const uint32_t src = blockIdx.y / beta, j = blockIdx.y % beta;
    const ConvTable* tab = tabs + j;
    const uint32_t ns = tab->ns, nt = tab->nt;
    const uint64_t* in = coef + ((size_t)src * n + j * alpha) * N + c;
    uint64_t* dst = ext + ((size_t)src * beta + j) * E * N + c;
    uint64_t y[YN];
#pragma unroll
    for (uint32_t i = 0; i < (NS > 0 ? (uint32_t)NS : ns); i++) {
        if (i >= ns) break;
        y[i] = in[(size_t)i * N];
    }
    for (uint32_t t = 0; t < nt; t++) {
        const uint32_t pt = tab->dst[t];
        acc128 a{0, 0};
#pragma unroll
        for (uint32_t i = 0; i < (NS > 0 ? (uint32_t)NS : ns); i++) {
            if (i >= ns) break;
            mad128(a, y[i], tab->hat[i][t]);
        }
        dst[(size_t)tab->dst_row[t] * N] = barrett128(a.lo, a.hi, qs[pt], bar[2 * pt], bar[2 * pt + 1]);
    }
}

template <typename... Args>
void launch_modup(uint32_t alpha, dim3 grid, cudaStream_t st, Args... args)
{
    switch (alpha) {
    case 1: k_ksb_modup<1><<<grid, kT, 0, st>>>(args...); break;
    case 2: k_ksb_modup<2><<<grid, kT, 0, st>>>(args...); break;
    case 3: k_ksb_modup<3><<<grid, kT, 0, st>>>(args...); break;
    case 4: k_ksb_modup<4><<<grid, kT, 0, st>>>(args...); break;
    default: k_ksb_modup<0><<<grid, kT, 0, st>>>(args...); break;
    }
}

// acc[group][p][t] = sum over the group's products x of sum_j sigma_x(ext[src_x][j][t]) key_x[j][p][kt]
// for the special-prime rows t = n + blockIdx.z only: they are the input of
// the ModDown conversion.  The ciphertext-prime rows are summed where they are
// used, in k_ksb_finish, so they are never written out.
// NB: the digit count beta as a compile-time loop bound (0 = any), so that
// every digit's loads are in flight together.
// Grid order of the inner-product and finish kernels: the group (or source)
// index is blockIdx.x, so the CTAs of all groups for one coefficient tile and
// prime are scheduled together and a key tile that several groups use (the
// giant-step keys of every output, the baby-step keys of every source, the
// relinearization key) is read from HBM once and then from L2.
template <int NB>
__global__ void __launch_bounds__(256, 6) k_ksb_inner(uint64_t* __restrict__ acc, const uint64_t* __restrict__ ext,
                            const DevGroup* __restrict__ groups, const DevProduct* __restrict__ prods, const __grid_constant__ LimbMap emap,
                            uint32_t n, uint32_t E, uint32_t beta, uint32_t nQ, uint32_t np,
                            const uint64_t* __restrict__ qs, const uint64_t* __restrict__ bar, uint32_t logN)
{
    const uint32_t N = 1u << logN;
    const uint32_t gr = blockIdx.x, c = blockIdx.y * blockDim.x + threadIdx.x, t = n + blockIdx.z;
    if (c >= N) return;
    const uint32_t pi = emap.p[t];
    const uint32_t kt = nQ + (t - n);
    const uint64_t q = qs[pi], r0 = bar[2 * pi], r1 = bar[2 * pi + 1];
    const DevGroup G = groups[gr];
    uint64_t s0 = 0, s1 = 0;
    for (uint32_t x = G.prod0; x < G.prod1; x++) {
        const DevProduct P = prods[x];
        const uint64_t* xs = ext + (size_t)P.src * beta * E * N + (size_t)t * N + perm_index(c, logN, P.g);
        acc128 a0{0, 0}, a1{0, 0};
#pragma unroll
        for (uint32_t j = 0; j < (NB > 0 ? (uint32_t)NB : beta); j++) {
            const uint64_t v = xs[(size_t)j * E * N];
            mad128(a0, v, P.key[(((size_t)j * 2 + 0) * np + kt) * N + c]);
            mad128(a1, v, P.key[(((size_t)j * 2 + 1) * np + kt) * N + c]);
        }
        s0 = add_mod(s0, barrett128(a0.lo, a0.hi, q, r0, r1), q);
        s1 = add_mod(s1, barrett128(a1.lo, a1.hi, q, r0, r1), q);
    }
    uint64_t* o = acc + (size_t)gr * 2 * E * N + (size_t)t * N + c;
    o[0] = s0;
    o[(size_t)E * N] = s1;
}

// Ciphertext prime i of group gr, both polynomials: the inner product
// acc_p = sum over the group's products of sum_j sigma_x(ext[src_x][j][i]) key_x[j][p][i]
// (the same sums k_ksb_inner forms for the special primes), then
// out_p = [out_p +] sum_{addends of p} add[perm(k)] + (acc_p - cv_p) P^-1
template <int NB>  // as for k_ksb_inner
__global__ void __launch_bounds__(256, 6) k_ksb_finish(const DevGroup* __restrict__ groups, const DevProduct* __restrict__ prods,
                             const uint64_t* __restrict__ ext, const KsAdd* __restrict__ adds,
                             const uint64_t* __restrict__ cv, uint32_t n, uint32_t E, uint32_t beta, uint32_t np,
                             PInv pinv, const uint64_t* __restrict__ qs, const uint64_t* __restrict__ bar,
                             uint32_t logN, int accumulate)
{
    const uint32_t N = 1u << logN;
    const uint32_t gr = blockIdx.x, k = blockIdx.y * blockDim.x + threadIdx.x, i = blockIdx.z;
    if (k >= N) return;
    const DevGroup G = groups[gr];
    const uint64_t q = qs[i], r0 = bar[2 * i], r1 = bar[2 * i + 1];
    // lazy 128-bit sums: reduced after every product for q >= 2^50 (beta terms
    // below 2^120 each), once at the end below that (terms below 2^100)
    const bool per_product = q >= (1ull << 50);
    uint64_t s[2] = {0, 0};
    acc128 a0{0, 0}, a1{0, 0};
    for (uint32_t x = G.prod0; x < G.prod1; x++) {
        const DevProduct P = prods[x];
        const uint64_t* xs = ext + (size_t)P.src * beta * E * N + (size_t)i * N + perm_index(k, logN, P.g);
#pragma unroll
        for (uint32_t j = 0; j < (NB > 0 ? (uint32_t)NB : beta); j++) {
            const uint64_t v = xs[(size_t)j * E * N];
            mad128(a0, v, P.key[(((size_t)j * 2 + 0) * np + i) * N + k]);
            mad128(a1, v, P.key[(((size_t)j * 2 + 1) * np + i) * N + k]);
        }
        if (per_product) {
            s[0] = add_mod(s[0], barrett128(a0.lo, a0.hi, q, r0, r1), q);
            s[1] = add_mod(s[1], barrett128(a1.lo, a1.hi, q, r0, r1), q);
            a0 = a1 = acc128{0, 0};
        }
    }
    if (!per_product) {
        s[0] = barrett128(a0.lo, a0.hi, q, r0, r1);
        s[1] = barrett128(a1.lo, a1.hi, q, r0, r1);
    }
#pragma unroll
    for (uint32_t p = 0; p < 2; p++) {
        const uint64_t v = cv[(((size_t)gr * 2 + p) * n + i) * N + k];
        uint64_t r = mul_shoup(sub_mod(s[p], v, q), pinv.w[i], pinv.wp[i], q);
        for (uint32_t x = G.add0; x < G.add1; x++) {
            const KsAdd A = adds[x];
            if (A.poly == p) r = add_mod(r, A.ptr[(size_t)i * N + perm_index(k, logN, A.g)], q);
        }
        uint64_t* o = (p ? G.out1 : G.out0) + (size_t)i * N + k;
        *o = accumulate ? add_mod(*o, r, q) : r;
    }
}

// The finish of a pass whose groups are single rotations of shared sources
// (hoisted rotations): one thread per (digit position k', prime i, source)
// reads the source's extended digits at k' once and serves every rotation of
// that source, whose output position is the k with perm(k, g) = k', i.e.
// k = perm(k', g^-1); per rotation as k_ksb_finish: the ciphertext-prime inner
// product with its key, the ModDown finish and the addends.  (k_ksb_finish reads
// the digits again for every rotation.)
template <int NB>
__global__ void __launch_bounds__(256, 6) k_ksb_finish_src(const DevGroup* __restrict__ groups,
                                 const DevProduct* __restrict__ prods, const uint64_t* __restrict__ ext,
                                 const KsAdd* __restrict__ adds, const uint64_t* __restrict__ cv,
                                 const uint32_t* __restrict__ so, const uint32_t* __restrict__ sg, uint32_t n,
                                 uint32_t E, uint32_t beta, uint32_t np, PInv pinv, const uint64_t* __restrict__ qs,
                                 const uint64_t* __restrict__ bar, uint32_t logN)
{
    constexpr int VN = NB > 0 ? NB : BLB_MAXP;
    const uint32_t N = 1u << logN;
    const uint32_t s = blockIdx.x, kp = blockIdx.y * blockDim.x + threadIdx.x, i = blockIdx.z;
    if (kp >= N) return;
    const uint64_t q = qs[i], r0 = bar[2 * i], r1 = bar[2 * i + 1];
    const uint64_t* xs = ext + (size_t)s * beta * E * N + (size_t)i * N + kp;
    uint64_t v[VN];
#pragma unroll
    for (uint32_t j = 0; j < (NB > 0 ? (uint32_t)NB : beta); j++) v[j] = xs[(size_t)j * E * N];
    for (uint32_t x = so[s]; x < so[s + 1]; x++) {
        const uint32_t gr = sg[x];
        const DevGroup G = groups[gr];
        const DevProduct P = prods[G.prod0];
        const uint32_t k = perm_index(kp, logN, P.ginv);
        acc128 a0{0, 0}, a1{0, 0};
#pragma unroll
        for (uint32_t j = 0; j < (NB > 0 ? (uint32_t)NB : beta); j++) {
            mad128(a0, v[j], P.key[(((size_t)j * 2 + 0) * np + i) * N + k]);
            mad128(a1, v[j], P.key[(((size_t)j * 2 + 1) * np + i) * N + k]);
        }
        const uint64_t sm[2] = {barrett128(a0.lo, a0.hi, q, r0, r1), barrett128(a1.lo, a1.hi, q, r0, r1)};
#pragma unroll
        for (uint32_t p = 0; p < 2; p++) {
            const uint64_t c = cv[(((size_t)gr * 2 + p) * n + i) * N + k];
            uint64_t r = mul_shoup(sub_mod(sm[p], c, q), pinv.w[i], pinv.wp[i], q);
            for (uint32_t y = G.add0; y < G.add1; y++) {
                const KsAdd A = adds[y];
                if (A.poly == p) r = add_mod(r, A.ptr[(size_t)i * N + perm_index(k, logN, A.g)], q);
            }
            (p ? G.out1 : G.out0)[(size_t)i * N + k] = r;
        }
    }
}

// g^-1 mod m for odd g and m a power of two (Newton's iteration doubles the
// correct low bits: 3 -> 6 -> ... -> 96)
uint64_t inv_mod_pow2(uint64_t g, uint64_t m)
{
    uint64_t x = g;
    for (int it = 0; it < 5; it++) x *= 2 - g * x;
    return x & (m - 1);
}

template <typename... Args>
void launch_finish_src(uint32_t beta, dim3 grid, cudaStream_t st, Args... args)
{
    switch (beta) {
    case 1: k_ksb_finish_src<1><<<grid, kT, 0, st>>>(args...); break;
    case 2: k_ksb_finish_src<2><<<grid, kT, 0, st>>>(args...); break;
    case 3: k_ksb_finish_src<3><<<grid, kT, 0, st>>>(args...); break;
    case 4: k_ksb_finish_src<4><<<grid, kT, 0, st>>>(args...); break;
    default: k_ksb_finish_src<0><<<grid, kT, 0, st>>>(args...); break;
    }
}

// launches with the digit count as a compile-time bound where it is small
template <typename... Args>
void launch_inner(uint32_t beta, dim3 grid, cudaStream_t st, Args... args)
{
    switch (beta) {
    case 1: k_ksb_inner<1><<<grid, kT, 0, st>>>(args...); break;
    case 2: k_ksb_inner<2><<<grid, kT, 0, st>>>(args...); break;
    case 3: k_ksb_inner<3><<<grid, kT, 0, st>>>(args...); break;
    case 4: k_ksb_inner<4><<<grid, kT, 0, st>>>(args...); break;
    default: k_ksb_inner<0><<<grid, kT, 0, st>>>(args...); break;
    }
}

template <typename... Args>
void launch_finish(uint32_t beta, dim3 grid, cudaStream_t st, Args... args)
{
    switch (beta) {
    case 1: k_ksb_finish<1><<<grid, kT, 0, st>>>(args...); break;
    case 2: k_ksb_finish<2><<<grid, kT, 0, st>>>(args...); break;
    case 3: k_ksb_finish<3><<<grid, kT, 0, st>>>(args...); break;
    case 4: k_ksb_finish<4><<<grid, kT, 0, st>>>(args...); break;
    default: k_ksb_finish<0><<<grid, kT, 0, st>>>(args...); break;
    }
}

}  // namespace

int ks_run(blb_ctx* ctx, uint32_t level, const KsSource* sources, uint32_t n_src, const KsProduct* prods,
           const KsGroup* groups, uint32_t n_groups, const KsAdd* adds, int accumulate)
{
    if (n_groups == 0) return BLB_OK;
    const uint32_t N = ctx->N, n = level + 1, nP = ctx->nP, E = n + nP;
    const uint32_t alpha = ctx->alpha, beta = (n + alpha - 1) / alpha;
    const size_t per_src = ((size_t)n + (size_t)beta * E) * N;      // coef, ext
    const size_t per_grp = ((size_t)2 * E + (size_t)2 * n) * N;     // acc, cv
    const size_t budget = (size_t)1 << 29;                           // 4 GiB per chunk
    // extension rows of one source and P rows of one group (row | prime << 24)
    std::vector<uint32_t> src_rows, grp_rows;
    for (uint32_t j = 0; j < beta; j++) {
        const uint32_t lo = j * alpha, hi = std::min((j + 1) * alpha, n);
        for (uint32_t t = 0; t < E; t++)
            if (t < lo || t >= hi) src_rows.push_back(j * E + t);
    }
    for (uint32_t pp = 0; pp < 2; pp++)
        for (uint32_t k = 0; k < nP; k++) grp_rows.push_back(pp * E + n + k);
    const auto prime_of = [&](uint32_t t) { return t < n ? t : ctx->nQ + (t - n); };
    PInv pinv{};
    for (uint32_t i = 0; i < n; i++) {
        pinv.w[i] = ctx->P_inv_mod_q[i];
        pinv.wp[i] = shoup_companion(pinv.w[i], ctx->q[i]);
    }
    const LimbMap emap = ctx->extmap(level);
    const uint32_t gx = (N + kT - 1) / kT;
    const uint64_t* ninv_conv = ctx->d_ninv_conv + (size_t)level * ctx->np * 2;
    std::vector<int32_t> local(n_src, -1);
    for (uint32_t g0 = 0; g0 < n_groups;) {
        // chunk: groups g0..g1 and the sources their products need
        std::vector<uint32_t> used;
        uint32_t g1 = g0;
        while (g1 < n_groups) {
            uint32_t extra = 0;
            for (uint32_t x = groups[g1].prod0; x < groups[g1].prod1; x++)
                if (local[prods[x].src] == -1) {
                    local[prods[x].src] = -2;  // counted for this group, not yet placed
                    extra++;
                }
            const size_t need = (used.size() + extra) * per_src + (size_t)(g1 - g0 + 1) * per_grp;
            if (g1 > g0 && need > budget) {
                for (uint32_t x = groups[g1].prod0; x < groups[g1].prod1; x++)
                    if (local[prods[x].src] <= -2) local[prods[x].src] = -1;
                break;
            }
            for (uint32_t x = groups[g1].prod0; x < groups[g1].prod1; x++)
                if (local[prods[x].src] <= -2) {
                    local[prods[x].src] = (int32_t)used.size();
                    used.push_back(prods[x].src);
                }
            g1++;
        }
        const uint32_t ns = (uint32_t)used.size(), ng = g1 - g0;
        // groups of the chunk ordered by their first key, so that the groups
        // sharing a key run back to back and the key is read from HBM about once
        std::vector<uint32_t> order(ng);
        for (uint32_t g = 0; g < ng; g++) order[g] = g0 + g;
        auto key_of = [&](uint32_t g) {
            return groups[g].prod1 > groups[g].prod0 ? (uintptr_t)prods[groups[g].prod0].key : (uintptr_t)0;
        };
        std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return key_of(a) < key_of(b); });
        // device tables for the chunk
        std::vector<DevSource> hs(ns);
        for (uint32_t s = 0; s < ns; s++) hs[s] = DevSource{sources[used[s]].c1, sources[used[s]].g};
        std::vector<DevProduct> hp;
        std::vector<DevGroup> hg(ng);
        std::vector<KsAdd> ha;
        for (uint32_t g = 0; g < ng; g++) {
            const KsGroup& G = groups[order[g]];
            hg[g].out0 = G.out0;
            hg[g].out1 = G.out1;
            hg[g].prod0 = (uint32_t)hp.size();
            for (uint32_t x = G.prod0; x < G.prod1; x++)
                hp.push_back(DevProduct{(uint32_t)local[prods[x].src], prods[x].g, prods[x].key,
                                        inv_mod_pow2(prods[x].g, 2ull * N)});
            hg[g].prod1 = (uint32_t)hp.size();
            hg[g].add0 = (uint32_t)ha.size();
            for (uint32_t x = G.add0; x < G.add1; x++) ha.push_back(adds[x]);
            hg[g].add1 = (uint32_t)ha.size();
        }
        // the finish by source when every group is one rotation of a shared
        // source (hoisted passes): the rotations of each source in one list
        bool by_src = !accumulate && ns > 0 && ng >= 2 * ns;
        for (uint32_t g = 0; g < ng && by_src; g++) by_src = hg[g].prod1 == hg[g].prod0 + 1;
        std::vector<uint32_t> so, sg;
        if (by_src) {
            so.assign(ns + 1, 0);
            for (uint32_t g = 0; g < ng; g++) so[hp[hg[g].prod0].src + 1]++;
            for (uint32_t s = 0; s < ns; s++) so[s + 1] += so[s];
            sg.assign(ng, 0);
            std::vector<uint32_t> fill(so.begin(), so.end() - 1);
            for (uint32_t g = 0; g < ng; g++) sg[fill[hp[hg[g].prod0].src]++] = g;
        }
        std::vector<uint32_t> ext_rows, p_rows;
        for (uint32_t s = 0; s < ns; s++)
            for (uint32_t r : src_rows) ext_rows.push_back((uint32_t)((size_t)s * beta * E + r) | (prime_of(r % E) << 24));
        for (uint32_t g = 0; g < ng; g++)
            for (uint32_t r : grp_rows) p_rows.push_back((uint32_t)((size_t)g * 2 * E + r) | (prime_of(r % E) << 24));
        if ((size_t)ns * beta * E >= (1u << 24) || (size_t)ng * 2 * E >= (1u << 24))
            return blb_fail(BLB_ERR_ARG, "key-switch batch too large");
        auto words = [](size_t bytes) { return (bytes + 7) / 8; };
        const size_t table_words = words(hs.size() * sizeof(DevSource)) + words(hp.size() * sizeof(DevProduct)) +
                                   words(hg.size() * sizeof(DevGroup)) + words(ha.size() * sizeof(KsAdd)) +
                                   words((ext_rows.size() + p_rows.size()) * 4) + words((so.size() + sg.size()) * 4) + 8;
        const bool cap = capturing(ctx);
        if (cap) ctx->captured = true;
        // under capture the tables go to a buffer of their own, so the arena
        // holds only the data every replay rewrites
        const size_t need = (size_t)ns * per_src + (size_t)ng * per_grp + (cap ? 0 : table_words);
        if (need > ctx->batch_words) {
            if (cap)
                return blb_fail(BLB_ERR_ARG, "key-switch arena too small during graph capture: run the call once "
                                             "before capturing it");
            BLB_CUDA(cudaStreamSynchronize(ctx->stream));  // the arena may still be read by earlier launches
            if (ctx->captured) ctx->graph_keep.push_back({ctx->batch, ctx->batch_words * 8});  // graphs read it
            else dev_free(ctx, ctx->batch, ctx->batch_words * 8);
            ctx->batch = (uint64_t*)dev_alloc(ctx, need * 8);
            ctx->batch_words = ctx->batch ? need : 0;
            if (!ctx->batch) return blb_fail(BLB_ERR_OOM, "key-switch batch arena");
        }
        uint64_t* coef = ctx->batch;
        uint64_t* ext = coef + (size_t)ns * n * N;
        uint64_t* acc = ext + (size_t)ns * beta * E * N;
        uint64_t* cv = acc + (size_t)ng * 2 * E * N;
        std::vector<uint64_t> host_tables;
        uint64_t* tw = cv + (size_t)ng * 2 * n * N;
        uint64_t* tw0 = tw;
        if (cap) {
            host_tables.assign(table_words, 0);
            tw = tw0 = host_tables.data();
        }
        DevSource* d_src = (DevSource*)tw;
        tw += words(hs.size() * sizeof(DevSource));
        DevProduct* d_prod = (DevProduct*)tw;
        tw += words(hp.size() * sizeof(DevProduct));
        DevGroup* d_grp = (DevGroup*)tw;
        tw += words(hg.size() * sizeof(DevGroup));
        KsAdd* d_add = (KsAdd*)tw;
        tw += words(ha.size() * sizeof(KsAdd));
        uint32_t* d_ext_rows = (uint32_t*)tw;
        uint32_t* d_p_rows = d_ext_rows + ext_rows.size();
        uint32_t* d_so = d_p_rows + p_rows.size();
        uint32_t* d_sg = d_so + so.size();
        if (cap) {
            // fill the host image, copy it once, and point every table into the copy
            memcpy(d_src, hs.data(), hs.size() * sizeof(DevSource));
            memcpy(d_prod, hp.data(), hp.size() * sizeof(DevProduct));
            memcpy(d_grp, hg.data(), hg.size() * sizeof(DevGroup));
            memcpy(d_add, ha.data(), ha.size() * sizeof(KsAdd));
            memcpy(d_ext_rows, ext_rows.data(), ext_rows.size() * 4);
            memcpy(d_p_rows, p_rows.data(), p_rows.size() * 4);
            memcpy(d_so, so.data(), so.size() * 4);
            memcpy(d_sg, sg.data(), sg.size() * 4);
            void* dev = nullptr;
            BLB_TRY(persist_upload(ctx, host_tables.data(), table_words * 8, &dev));
            auto rebase = [&](auto* p) { return (decltype(p))((uint8_t*)dev + ((uint8_t*)p - (uint8_t*)tw0)); };
            d_src = rebase(d_src);
            d_prod = rebase(d_prod);
            d_grp = rebase(d_grp);
            d_add = rebase(d_add);
            d_ext_rows = rebase(d_ext_rows);
            d_p_rows = rebase(d_p_rows);
            d_so = rebase(d_so);
            d_sg = rebase(d_sg);
        } else {
            auto up = [&](void* dst, const void* src, size_t bytes) {
                return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream) : cudaSuccess;
            };
            BLB_CUDA(up(d_src, hs.data(), hs.size() * sizeof(DevSource)));
            BLB_CUDA(up(d_prod, hp.data(), hp.size() * sizeof(DevProduct)));
            BLB_CUDA(up(d_grp, hg.data(), hg.size() * sizeof(DevGroup)));
            BLB_CUDA(up(d_add, ha.data(), ha.size() * sizeof(KsAdd)));
            BLB_CUDA(up(d_ext_rows, ext_rows.data(), ext_rows.size() * 4));
            BLB_CUDA(up(d_p_rows, p_rows.data(), p_rows.size() * 4));
            BLB_CUDA(up(d_so, so.data(), so.size() * 4));
            BLB_CUDA(up(d_sg, sg.data(), sg.size() * 4));
        }
        // algorithmic bytes: each source read and its digits written once; each
        // product reads its digits and key; each group writes its output
        ProfScope prof(ctx, "keyswitch",
                       ((uint64_t)ns * (n + (uint64_t)beta * E) + (uint64_t)hp.size() * 3 * beta * E +
                        (uint64_t)ng * 2 * n) * N * 8);
        {
            // arithmetic per coefficient, summed over the launches below
            const uint64_t nprod = hp.size();
            uint64_t mad = 0, red = 0, bfly = 0;
            for (uint32_t j = 0; j < beta; j++) {  // ModUp: |D_j| sources to E - |D_j| targets
                const uint64_t dj = std::min((j + 1) * alpha, n) - j * alpha;
                mad += ns * dj * (E - dj);
                red += ns * (E - dj);
            }
            mad += nprod * 2 * beta * nP;                      // inner products, special primes
            red += nprod * 2 * nP;
            mad += (uint64_t)ng * 2 * (nP + (uint64_t)n * (nP + 1));  // ModDown: rounding sum, n targets
            red += (uint64_t)ng * 2 * n;
            mad += nprod * 2 * beta * n;                       // inner products, ciphertext primes
            for (uint32_t i = 0; i < n; i++) red += 2 * (ctx->q[i] >= (1ull << 50) || by_src ? nprod : ng);
            bfly += (uint64_t)ng * 2 * n;                      // the P^-1 Shoup products
            const uint64_t ntt_rows = (uint64_t)ns * n + ext_rows.size() + p_rows.size() + (uint64_t)ng * 2 * n;
            prof.ops(mad * N, red * N, bfly * N + ntt_rows * (N / 2) * ctx->logN);
        }
        if (ns) {
            // the gather of the sources' c1 rows (permuted) runs in the first
            // pass of their inverse transform
            BLB_TRY(ntt_inverse_gather(ctx, coef, ns * n, GatherIO{d_src, ext, n, E, beta, alpha}, ninv_conv));
            launch_modup(alpha, dim3(gx, ns * beta), ctx->stream, (const uint64_t*)coef, ext,
                         (const ConvTable*)ctx->d_modup[(size_t)level * ctx->dnum], n, E, beta, alpha,
                         (const uint64_t*)ctx->d_q, (const uint64_t*)ctx->d_bar, N);
            BLB_LAUNCHED();
            BLB_TRY(ntt_forward_list(ctx, ext, (uint32_t)ext_rows.size(), d_ext_rows));
        }
        launch_inner(beta, dim3(ng, gx, nP), ctx->stream, acc, (const uint64_t*)ext, (const DevGroup*)d_grp,
                     (const DevProduct*)d_prod, emap, n, E, beta, ctx->nQ, ctx->np, (const uint64_t*)ctx->d_q,
                     (const uint64_t*)ctx->d_bar, ctx->logN);
        BLB_LAUNCHED();
        BLB_TRY(ntt_inverse_list_scaled(ctx, acc, (uint32_t)p_rows.size(), d_p_rows, ninv_conv));
        launch_moddown_conv<true>(nP, dim3(gx, 2 * ng), ctx->stream, (const uint64_t*)(acc + (size_t)n * N),
                            (size_t)E * N, (const ConvTable*)ctx->d_moddown, n, cv, (size_t)n * N,
                            (const uint64_t*)ctx->d_q, (const uint64_t*)ctx->d_bar, N);
        BLB_LAUNCHED();
        BLB_TRY(ntt_forward(ctx, cv, ng * 2 * n, ctx->qmap(n)));
        if (by_src)
            launch_finish_src(beta, dim3(ns, gx, n), ctx->stream, (const DevGroup*)d_grp, (const DevProduct*)d_prod,
                              (const uint64_t*)ext, (const KsAdd*)d_add, (const uint64_t*)cv, (const uint32_t*)d_so,
                              (const uint32_t*)d_sg, n, E, beta, ctx->np, pinv, (const uint64_t*)ctx->d_q,
                              (const uint64_t*)ctx->d_bar, ctx->logN);
        else
            launch_finish(beta, dim3(ng, gx, n), ctx->stream, (const DevGroup*)d_grp, (const DevProduct*)d_prod,
                          (const uint64_t*)ext, (const KsAdd*)d_add, (const uint64_t*)cv, n, E, beta, ctx->np, pinv,
                          (const uint64_t*)ctx->d_q, (const uint64_t*)ctx->d_bar, ctx->logN, accumulate);
        BLB_LAUNCHED();
        for (uint32_t s : used) local[s] = -1;
        g0 = g1;
    }
    return BLB_OK;
}

int keyswitch_batch(blb_ctx* ctx, uint32_t level, const KsItem* items, uint32_t count, int accumulate)
{
    std::vector<KsSource> src(count);
    std::vector<KsProduct> prod(count);
    std::vector<KsGroup> grp(count);
    std::vector<KsAdd> adds;
    for (uint32_t i = 0; i < count; i++) {
        const KsItem& it = items[i];
        src[i] = KsSource{it.c1, it.g};
        prod[i] = KsProduct{i, 1, it.key};
        grp[i].out0 = it.out0;
        grp[i].out1 = it.out1;
        grp[i].prod0 = i;
        grp[i].prod1 = i + 1;
        grp[i].add0 = (uint32_t)adds.size();
        if (it.c0) adds.push_back(KsAdd{it.c0, it.g, 0});
        if (it.add1) adds.push_back(KsAdd{it.add1, it.g, 1});
        grp[i].add1 = (uint32_t)adds.size();
    }
    return ks_run(ctx, level, src.data(), count, prod.data(), grp.data(), count, adds.data(), accumulate);
}
