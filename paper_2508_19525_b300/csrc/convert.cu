// convert.cu -- the parties' local steps of the conversions between CKKS
// ciphertexts and additive shares (Alg. 1 steps 3-4, Alg. 2, Sec. 6.3,
// App. C.3), batched over many ciphertexts.
//
// CKKS -> MPC: each party turns its share of the coefficients of Encode(x) mod
// q_0 into a share over the extended ring Z_{2^128} (field to ring), then
// decodes it locally with a fixed-point FFT whose products are truncated by
// SecureML's local rule, and keeps the real slots at the MPC scale 2^-sf mod
// 2^l.  MPC -> CKKS: each party extends its slot shares from Z_{2^l} to
// Z_{2^128}, encodes them locally with the inverse FFT (each butterfly halved
// by a truncation), and reduces the coefficient shares mod every prime of the
// target level (ring to field).  The comparisons inside the ring/field
// extensions are MPC protocols; their ideal functionality is simulated by
// blb_f2r_wrap_sim / blb_ext_wrap_sim.
//
// Fixed point: roots round(2^30 c zeta^k) (c = 1, or the scale's mantissa
// folded in), FFT data at resolution 2^-26 slot units, so every truncated
// product stays near or below 2^87 and a truncation fails with probability
// |m| / 2^128 < 2^-40.
//
// GPU layout: one FFT of s = N/2 complex 128-bit shares (32 B each) is
// radix-2 decimation in time on bit-reversed input, the same butterflies as
// the definition, in two passes over 1024-element shared-memory tiles (32 KB):
// pass 1 runs stages 1..H1 on contiguous blocks of 2^H1 elements, pass 2
// stages H1+1..log2 s on the 2^H1 interleaved sub-problems.  Integer results
// do not depend on the schedule, so both passes reproduce the definition bit
// for bit.
#include "common.cuh"

namespace {

constexpr int FX_F = 30;    // fraction bits of the roots
constexpr int FX_P = 26;    // resolution 2^-26 of the FFT data
constexpr int FX_T = 512;   // threads per CTA: one butterfly each per stage
constexpr int FX_E = 1024;  // complex elements per CTA tile

struct u128 {
    uint64_t lo, hi;
};
struct __align__(16) c128 {
    u128 re, im;
};

__device__ __forceinline__ u128 add(u128 a, u128 b)
{
    u128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo);
    return r;
}
__device__ __forceinline__ u128 sub(u128 a, u128 b)
{
    u128 r;
    r.lo = a.lo - b.lo;
    r.hi = a.hi - b.hi - (a.lo < b.lo);
    return r;
}
__device__ __forceinline__ u128 neg(u128 a) { return sub(u128{0, 0}, a); }
// shifts by 0 <= k < 64
__device__ __forceinline__ u128 shl(u128 a, int k)
{
    if (k == 0) return a;
    return u128{a.lo << k, (a.hi << k) | (a.lo >> (64 - k))};
}
__device__ __forceinline__ u128 sar(u128 a, int k)
{
    if (k == 0) return a;
    return u128{(a.lo >> k) | (a.hi << (64 - k)), (uint64_t)((int64_t)a.hi >> k)};
}
// probabilistic truncation (SecureML): party 0 floor(x / 2^k), party 1
// ceil(x / 2^k), the share read as a signed 128-bit integer
template <bool P1>
__device__ __forceinline__ u128 trunc(u128 a, int k)
{
    if (P1) return neg(sar(neg(a), k));
    return sar(a, k);
}

// a * w mod 2^128 for |w| < 2^31, from 32 x 32 -> 64-bit products
__device__ __forceinline__ u128 mul_s(u128 a, int32_t w)
{
    const uint32_t m = w < 0 ? (uint32_t)(-w) : (uint32_t)w;
    const uint64_t p0 = (uint64_t)(uint32_t)a.lo * m;
    const uint64_t p1 = (uint64_t)(uint32_t)(a.lo >> 32) * m;
    u128 r;
    r.lo = p0 + (p1 << 32);
    r.hi = (p1 >> 32) + (r.lo < p0) + a.hi * m;
    return w < 0 ? neg(r) : r;
}
// (v.re + i v.im)(w.x + i w.y), untruncated
__device__ __forceinline__ c128 cmul(const c128& v, int2 w)
{
    return c128{sub(mul_s(v.re, w.x), mul_s(v.im, w.y)), add(mul_s(v.re, w.y), mul_s(v.im, w.x))};
}
__device__ __forceinline__ u128 ld2(const uint64_t* p, size_t i)
{
    const ulonglong2 v = reinterpret_cast<const ulonglong2*>(p)[i];
    return u128{v.x, v.y};
}
__device__ __forceinline__ uint32_t brev(uint32_t x, int bits) { return __brev(x) >> (32 - bits); }

// field to ring, party's local step: U = t' - <w> q - [P0] h, t' = t + h mod q for P0
template <bool P1>
__device__ __forceinline__ u128 f2r(uint64_t t, u128 ws, uint64_t q, uint64_t h)
{
    const uint64_t tp = P1 ? t : add_mod(t, h, q);
    const u128 wq{ws.lo * q, __umul64hi(ws.lo, q) + ws.hi * q};
    const u128 u = sub(u128{tp, 0}, wq);
    return P1 ? u : sub(u, u128{h, 0});
}
// signed extension, party's local step: X = x' - <w> 2^l - [P0] 2^(l-1)
template <bool P1>
__device__ __forceinline__ u128 ext(uint64_t x, u128 ws, int l)
{
    const uint64_t M = 1ull << l, mask = M - 1, half = M >> 1;
    const uint64_t xp = P1 ? (x & mask) : ((x + half) & mask);
    const u128 v = sub(u128{xp, 0}, shl(ws, l));
    return P1 ? v : sub(v, u128{half, 0});
}

// decoding butterfly: v' = trunc(v w, F); (u, v) <- (u + v', u - v')
// encoding butterfly: p = v conj(w); (u, v) <- trunc(u 2^F +- p, F + 1)
template <bool INV, bool P1>
__device__ __forceinline__ void bfly(c128& u, c128& v, int2 w)
{
    if (!INV) {
        const c128 pr = cmul(v, w);
        const u128 vr = trunc<P1>(pr.re, FX_F), vi = trunc<P1>(pr.im, FX_F);
        const c128 a = u;
        u = c128{add(a.re, vr), add(a.im, vi)};
        v = c128{sub(a.re, vr), sub(a.im, vi)};
    } else {
        const c128 pr = cmul(v, make_int2(w.x, -w.y));
        const u128 ur = shl(u.re, FX_F), ui = shl(u.im, FX_F);
        u = c128{trunc<P1>(add(ur, pr.re), FX_F + 1), trunc<P1>(add(ui, pr.im), FX_F + 1)};
        v = c128{trunc<P1>(sub(ur, pr.re), FX_F + 1), trunc<P1>(sub(ui, pr.im), FX_F + 1)};
    }
}

// stages 1..H1 on the CTA's 1024 >> H1 contiguous blocks of 2^H1 elements,
// thread b owning butterfly b of every stage; the next stage's root is
// fetched before the current stage's butterfly so its latency overlaps it
template <int LOGS, bool INV, bool P1>
__device__ __forceinline__ void stages_pass1(c128* sm, const int2* __restrict__ root)
{
    constexpr int H1 = (LOGS + 1) / 2;
    const int b = threadIdx.x;
    const int col = b >> (H1 - 1), bb = b & ((1 << (H1 - 1)) - 1);
    c128* base = sm + (col << H1);
    int2 w = root[0];
#pragma unroll
    for (int sg = 1; sg <= H1; sg++) {
        const int half = 1 << (sg - 1);
        const int j = bb & (half - 1), i0 = ((bb >> (sg - 1)) << sg) + j;
        int2 wn = w;
        if (sg < H1) wn = root[(bb & (2 * half - 1)) << (LOGS - sg + 1)];
        bfly<INV, P1>(base[i0], base[i0 + half], w);
        w = wn;
        __syncthreads();
    }
}

// stages H1+1..LOGS on the CTA's 1024 >> H2 interleaved sub-problems r0.. (element
// i = r + 2^H1 b', stored at sm[(r - r0) 2^H2 + b'])
template <int LOGS, bool INV, bool P1>
__device__ __forceinline__ void stages_pass2(c128* sm, const int2* __restrict__ root, uint32_t r0)
{
    constexpr int H1 = (LOGS + 1) / 2, H2 = LOGS - H1;
    const int b = threadIdx.x;
    const int row = b >> (H2 - 1), bb = b & ((1 << (H2 - 1)) - 1);
    c128* base = sm + (row << H2);
    const uint32_t r = r0 + row;
    int2 w = root[r << (LOGS - H1 + 1)];
#pragma unroll
    for (int sg = H1 + 1; sg <= LOGS; sg++) {
        const int sl = sg - H1, half = 1 << (sl - 1);
        const int jj = bb & (half - 1), i0 = ((bb >> (sl - 1)) << sl) + jj;
        int2 wn = w;
        if (sg < LOGS) wn = root[(r + ((uint32_t)(bb & (2 * half - 1)) << H1)) << (LOGS - sg + 1)];
        bfly<INV, P1>(base[i0], base[i0 + half], w);
        w = wn;
        __syncthreads();
    }
}

// CKKS -> MPC pass 1: field to ring, scaling to 2^-P, twist, bit reversal and
// the first H1 stages.  T: count x N residues mod q_0; W: count x N wrap-bit
// shares (2 words each); A: count x s complex shares in bit-reversed order.
template <int LOGS, bool P1>
__global__ void __launch_bounds__(FX_T) k_c2m_pass1(const uint64_t* __restrict__ T, const uint64_t* __restrict__ W,
                                                    c128* __restrict__ A, const int2* __restrict__ root,
                                                    const int2* __restrict__ twist, uint64_t q, int sh_in)
{
    constexpr int H1 = (LOGS + 1) / 2, H2 = LOGS - H1, C = FX_E >> H1;
    constexpr uint32_t S = 1u << LOGS;
    __shared__ c128 sm[FX_E];
    const uint32_t c0 = blockIdx.x * C;
    const size_t mem = blockIdx.y;
    const uint64_t* Tm = T + mem * 2 * S;
    const uint64_t* Wm = W + mem * 4 * S;
    const uint64_t h = (q - 1) / 2;
    for (int e = threadIdx.x; e < FX_E; e += FX_T) {
        const uint32_t co = e % C, rp = e / C;
        const uint32_t t = (rp << H2) + c0 + co;
        u128 y0 = f2r<P1>(Tm[t], ld2(Wm, t), q, h), y1 = f2r<P1>(Tm[t + S], ld2(Wm, t + S), q, h);
        if (sh_in >= 0) {
            y0 = trunc<P1>(y0, sh_in);
            y1 = trunc<P1>(y1, sh_in);
        } else {
            y0 = shl(y0, -sh_in);
            y1 = shl(y1, -sh_in);
        }
        const c128 v = cmul(c128{y0, y1}, twist[t]);
        sm[(co << H1) + brev(rp, H1)] = c128{trunc<P1>(v.re, FX_F), trunc<P1>(v.im, FX_F)};
    }
    __syncthreads();
    stages_pass1<LOGS, false, P1>(sm, root);
    c128* Am = A + mem * S;
    for (int e = threadIdx.x; e < FX_E; e += FX_T) {
        const uint32_t col = e >> H1, r = e & ((1 << H1) - 1);
        Am[(brev(c0 + col, H2) << H1) + r] = sm[e];
    }
}

// CKKS -> MPC pass 2: the remaining stages, then slot j = Re A[k_j] truncated
// to 2^-sf and reduced mod 2^l.  out: count x s words.
template <int LOGS, bool P1>
__global__ void __launch_bounds__(FX_T) k_c2m_pass2(const c128* __restrict__ A, uint64_t* __restrict__ out,
                                                    const int2* __restrict__ root, const uint32_t* __restrict__ kinv,
                                                    int sh_out, uint64_t mask)
{
    constexpr int H1 = (LOGS + 1) / 2, H2 = LOGS - H1, C2 = FX_E >> H2;
    constexpr uint32_t S = 1u << LOGS;
    __shared__ c128 sm[FX_E];
    const uint32_t r0 = blockIdx.x * C2;
    const size_t mem = blockIdx.y;
    const c128* Am = A + mem * S;
    for (int e = threadIdx.x; e < FX_E; e += FX_T) {
        const uint32_t ro = e % C2, bp = e / C2;
        sm[(ro << H2) + bp] = Am[r0 + ro + (bp << H1)];
    }
    __syncthreads();
    stages_pass2<LOGS, false, P1>(sm, root, r0);
    uint64_t* om = out + mem * S;
    for (int e = threadIdx.x; e < FX_E; e += FX_T) {
        const uint32_t ro = e % C2, bp = e / C2;
        const uint32_t i = r0 + ro + (bp << H1);
        om[kinv[i]] = trunc<P1>(sm[(ro << H2) + bp].re, sh_out).lo & mask;
    }
}

// MPC -> CKKS pass 1: extension, shift to 2^-P, placement V[k_j] = x_j in
// bit-reversed order, the first H1 halved inverse stages.  X: count x n words;
// W: count x n wrap-bit shares.
template <int LOGS, bool P1>
__global__ void __launch_bounds__(FX_T) k_m2c_pass1(const uint64_t* __restrict__ X, const uint64_t* __restrict__ W,
                                                    c128* __restrict__ A, const int2* __restrict__ root,
                                                    const uint32_t* __restrict__ kinv, uint32_t n, int l, int sh_up)
{
    constexpr int H1 = (LOGS + 1) / 2, H2 = LOGS - H1, C = FX_E >> H1;
    constexpr uint32_t S = 1u << LOGS;
    __shared__ c128 sm[FX_E];
    const uint32_t c0 = blockIdx.x * C;
    const size_t mem = blockIdx.y;
    const uint64_t* Xm = X + mem * n;
    const uint64_t* Wm = W + mem * 2 * n;
    for (int e = threadIdx.x; e < FX_E; e += FX_T) {
        const uint32_t co = e % C, rp = e / C;
        const uint32_t k = (rp << H2) + c0 + co;
        const uint32_t j = kinv[k];
        u128 v{0, 0};
        if (j < n) v = shl(ext<P1>(Xm[j], ld2(Wm, j), l), sh_up);
        sm[(co << H1) + brev(rp, H1)] = c128{v, u128{0, 0}};
    }
    __syncthreads();
    stages_pass1<LOGS, true, P1>(sm, root);
    c128* Am = A + mem * S;
    for (int e = threadIdx.x; e < FX_E; e += FX_T) {
        const uint32_t col = e >> H1, r = e & ((1 << H1) - 1);
        Am[(brev(c0 + col, H2) << H1) + r] = sm[e];
    }
}

struct R2FConsts {
    uint64_t q[BLB_MAXP], r0[BLB_MAXP], r1[BLB_MAXP], two128[BLB_MAXP];
};

// ring to field of one share read as a signed 128-bit integer
__device__ __forceinline__ uint64_t r2f(u128 v, uint64_t q, uint64_t b0, uint64_t b1, uint64_t two128)
{
    const uint64_t r = barrett128(v.lo, v.hi, q, b0, b1);
    return (v.hi >> 63) ? sub_mod(r, two128, q) : r;
}

// MPC -> CKKS pass 2: the remaining stages, the twist and scaling to Delta,
// then ring to field for every prime of the level.  out: count x nl x N words.
template <int LOGS, bool P1>
__global__ void __launch_bounds__(FX_T) k_m2c_pass2(const c128* __restrict__ A, uint64_t* __restrict__ out,
                                                    const int2* __restrict__ root, const int2* __restrict__ twist,
                                                    const __grid_constant__ R2FConsts K, uint32_t nl, int sh)
{
    constexpr int H1 = (LOGS + 1) / 2, H2 = LOGS - H1, C2 = FX_E >> H2;
    constexpr uint32_t S = 1u << LOGS;
    __shared__ c128 sm[FX_E];
    const uint32_t r0 = blockIdx.x * C2;
    const size_t mem = blockIdx.y;
    const c128* Am = A + mem * S;
    for (int e = threadIdx.x; e < FX_E; e += FX_T) {
        const uint32_t ro = e % C2, bp = e / C2;
        sm[(ro << H2) + bp] = Am[r0 + ro + (bp << H1)];
    }
    __syncthreads();
    stages_pass2<LOGS, true, P1>(sm, root, r0);
    uint64_t* om = out + mem * nl * 2 * S;
    for (int e = threadIdx.x; e < FX_E; e += FX_T) {
        const uint32_t ro = e % C2, bp = e / C2;
        const uint32_t t = r0 + ro + (bp << H1);
        const int2 w = twist[t];
        c128 c = cmul(sm[(ro << H2) + bp], make_int2(w.x, -w.y));
        if (sh >= 0) {
            c.re = trunc<P1>(c.re, sh);
            c.im = trunc<P1>(c.im, sh);
        } else {
            c.re = shl(c.re, -sh);
            c.im = shl(c.im, -sh);
        }
        for (uint32_t li = 0; li < nl; li++) {
            uint64_t* row = om + (size_t)li * 2 * S;
            row[t] = r2f(c.re, K.q[li], K.r0[li], K.r1[li], K.two128[li]);
            row[t + S] = r2f(c.im, K.q[li], K.r0[li], K.r1[li], K.two128[li]);
        }
    }
}

// ideal functionality of the comparisons inside Pi_Ext: arithmetic shares of
// the wrap bit, P0 rho (128-bit Philox draw (i, 0, nonce, WRAP)), P1 w - rho
__device__ __forceinline__ void share_bit(uint32_t w, uint64_t seed, uint32_t i, uint32_t nonce, ulonglong2* w0,
                                          ulonglong2* w1)
{
    const uint4 d = philox_draw(seed, i, 0, nonce, PURPOSE_WRAP);
    const u128 rho{(uint64_t)d.x | ((uint64_t)d.y << 32), (uint64_t)d.z | ((uint64_t)d.w << 32)};
    const u128 r1 = sub(u128{w, 0}, rho);
    w0[i] = make_ulonglong2(rho.lo, rho.hi);
    w1[i] = make_ulonglong2(r1.lo, r1.hi);
}

__global__ void k_f2r_wrap_sim(const uint64_t* __restrict__ t0, const uint64_t* __restrict__ t1,
                               uint64_t* __restrict__ w0, uint64_t* __restrict__ w1, uint32_t n, uint64_t q,
                               uint64_t seed, const uint32_t* __restrict__ nonces)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t m = blockIdx.y;
    const uint64_t a = add_mod(t0[m * n + i], (q - 1) / 2, q);
    share_bit(a + t1[m * n + i] >= q, seed, i, nonces[m], reinterpret_cast<ulonglong2*>(w0) + m * n,
              reinterpret_cast<ulonglong2*>(w1) + m * n);
}

__global__ void k_ext_wrap_sim(const uint64_t* __restrict__ x0, const uint64_t* __restrict__ x1,
                               uint64_t* __restrict__ w0, uint64_t* __restrict__ w1, uint32_t n, int l, uint64_t seed,
                               const uint32_t* __restrict__ nonces)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t m = blockIdx.y;
    const uint64_t M = 1ull << l, mask = M - 1;
    const uint64_t a = (x0[m * n + i] + (M >> 1)) & mask;
    share_bit(a + (x1[m * n + i] & mask) >= M, seed, i, nonces[m], reinterpret_cast<ulonglong2*>(w0) + m * n,
              reinterpret_cast<ulonglong2*>(w1) + m * n);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// (round(2^F c cos(pi k/N)), round(2^F c sin(pi k/N))), C library cos / sin,
// round half to even
int2 fx_root(uint32_t N, uint32_t k, double c)
{
    const double ang = M_PI * (double)k / (double)N;
    return make_int2((int)rint(ldexp(cos(ang) * c, FX_F)), (int)rint(ldexp(sin(ang) * c, FX_F)));
}

// roots zeta^k for k < N, and the inverse of the slot permutation k_j
int fx_tables(blb_ctx* c)
{
    if (c->d_fx_root) return BLB_OK;
    BLB_TRY(refuse_capture(c, "the first conversion of a context"));  // the tables it caches
    const uint32_t N = c->N, s = N / 2;
    std::vector<int2> root(N);
    for (uint32_t k = 0; k < N; k++) root[k] = fx_root(N, k, 1.0);
    std::vector<uint32_t> kinv(s);
    uint64_t g = 1;
    for (uint32_t j = 0; j < s; j++) {
        kinv[(g - 1) / 4] = j;
        g = (g * 5) % (2ull * N);
    }
    int2* dr = (int2*)dev_alloc(c, (size_t)N * sizeof(int2));
    uint32_t* dk = (uint32_t*)dev_alloc(c, (size_t)s * 4);
    if (!dr || !dk) {
        dev_free(c, dr, (size_t)N * sizeof(int2));
        dev_free(c, dk, (size_t)s * 4);
        return blb_fail(BLB_ERR_OOM, "conversion tables");
    }
    BLB_CUDA(cudaMemcpyAsync(dr, root.data(), (size_t)N * sizeof(int2), cudaMemcpyHostToDevice, c->stream));
    BLB_CUDA(cudaMemcpyAsync(dk, kinv.data(), (size_t)s * 4, cudaMemcpyHostToDevice, c->stream));
    BLB_CUDA(cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
    c->d_fx_root = dr;
    c->d_kinv = dk;
    return BLB_OK;
}

// twist table round(2^F c zeta^t), t < N/2, cached per multiplier c
int fx_twist(blb_ctx* c, double mul, const int2** out)
{
    for (auto& t : c->fx_twist)
        if (t.mul == mul) {
            *out = t.d;
            return BLB_OK;
        }
    BLB_TRY(refuse_capture(c, "the first conversion with this scale"));  // the table it caches
    const uint32_t N = c->N, s = N / 2;
    std::vector<int2> tw(s);
    for (uint32_t k = 0; k < s; k++) tw[k] = fx_root(N, k, mul);
    if (c->fx_twist.size() >= 8) {
        dev_free(c, c->fx_twist.front().d, (size_t)s * sizeof(int2));
        c->fx_twist.erase(c->fx_twist.begin());
    }
    int2* d = (int2*)dev_alloc(c, (size_t)s * sizeof(int2));
    if (!d) return blb_fail(BLB_ERR_OOM, "conversion twist table");
    BLB_CUDA(cudaMemcpyAsync(d, tw.data(), (size_t)s * sizeof(int2), cudaMemcpyHostToDevice, c->stream));
    BLB_CUDA(cudaStreamSynchronize(c->stream));
    c->fx_twist.push_back({mul, d});
    *out = d;
    return BLB_OK;
}

// device view of a caller buffer: the buffer itself if it is device memory,
// else a scratch copy (inputs) or a scratch buffer copied back later (outputs)
const void* dev_in(blb_ctx* c, Scratch& S, const void* p, size_t bytes, int* rc)
{
    if (is_device_ptr(p)) return p;
    void* d = S.get(bytes);
    if (!d) {
        *rc = blb_fail(BLB_ERR_OOM, "conversion input staging");
        return nullptr;
    }
    *rc = copy_in(c, d, p, bytes);
    return d;
}
void* dev_out(Scratch& S, void* p, size_t bytes, int* rc)
{
    if (is_device_ptr(p)) return p;
    void* d = S.get(bytes);
    if (!d) *rc = blb_fail(BLB_ERR_OOM, "conversion output staging");
    return d;
}

int check_fixed(blb_ctx* c, uint32_t l, uint32_t sf)
{
    if (c->logN < 12 || c->logN > 17) return blb_fail(BLB_ERR_ARG, "conversions need 2^12 <= N <= 2^17");
    if (l > 62 || sf > (uint32_t)FX_P || l < sf + 2)
        return blb_fail(BLB_ERR_ARG, "need sf <= 26 and sf + 2 <= l <= 62");
    return BLB_OK;
}

// run the statement with L_ = log2(N/2) as a compile-time constant
#define FX_DISPATCH(LOGS, ...)                                           \
    do {                                                                 \
    switch (LOGS) {                                                      \
    case 11: { constexpr int L_ = 11; __VA_ARGS__; } break;              \
    case 12: { constexpr int L_ = 12; __VA_ARGS__; } break;              \
    case 13: { constexpr int L_ = 13; __VA_ARGS__; } break;              \
    case 14: { constexpr int L_ = 14; __VA_ARGS__; } break;              \
    case 15: { constexpr int L_ = 15; __VA_ARGS__; } break;              \
    case 16: { constexpr int L_ = 16; __VA_ARGS__; } break;              \
    default: return blb_fail(BLB_ERR_ARG, "unsupported ring degree");    \
    }                                                                    \
    } while (0)

// 128-bit share arrays in device memory are read and written as 16-byte
// vectors (host arrays are staged through aligned scratch)
bool aligned16(const void* p) { return !is_device_ptr(p) || ((uintptr_t)p & 15) == 0; }

std::vector<uint32_t> nonce_words(const uint64_t* nonces, uint32_t count)
{
    std::vector<uint32_t> v(count);
    for (uint32_t k = 0; k < count; k++) v[k] = (uint32_t)nonces[k];
    return v;
}

}  // namespace

extern "C" int blb_f2r_wrap_sim(blb_ctx* c, const uint64_t* t0, const uint64_t* t1, uint32_t count, uint64_t seed,
                                const uint64_t* nonces, uint64_t* w0, uint64_t* w1)
{
    if (!c || !t0 || !t1 || !nonces || !w0 || !w1) return blb_fail(BLB_ERR_ARG, "null argument");
    if (!aligned16(w0) || !aligned16(w1)) return blb_fail(BLB_ERR_ARG, "share arrays must be 16-byte aligned");
    if (count == 0) return BLB_OK;
    const uint32_t N = c->N;
    Scratch S(c);
    int rc = BLB_OK;
    const size_t nin = (size_t)count * N * 8, nw = 2 * nin;
    const uint64_t* d0 = (const uint64_t*)dev_in(c, S, t0, nin, &rc);
    const uint64_t* d1 = rc ? nullptr : (const uint64_t*)dev_in(c, S, t1, nin, &rc);
    uint64_t* o0 = rc ? nullptr : (uint64_t*)dev_out(S, w0, nw, &rc);
    uint64_t* o1 = rc ? nullptr : (uint64_t*)dev_out(S, w1, nw, &rc);
    const uint32_t* dn = rc ? nullptr : S.upload(nonce_words(nonces, count));
    if (rc) return rc;
    if (!dn) return blb_fail(BLB_ERR_OOM, "nonce table");
    k_f2r_wrap_sim<<<dim3((N + 255) / 256, count), 256, 0, c->stream>>>(d0, d1, o0, o1, N, c->q[0], seed, dn);
    BLB_LAUNCHED();
    if (o0 != w0) BLB_TRY(copy_out(c, w0, o0, nw));
    if (o1 != w1) BLB_TRY(copy_out(c, w1, o1, nw));
    return BLB_OK;
}

extern "C" int blb_ext_wrap_sim(blb_ctx* c, const uint64_t* x0, const uint64_t* x1, uint32_t n, uint32_t count,
                                uint32_t l, uint64_t seed, const uint64_t* nonces, uint64_t* w0, uint64_t* w1)
{
    if (!c || !x0 || !x1 || !nonces || !w0 || !w1) return blb_fail(BLB_ERR_ARG, "null argument");
    if (l < 2 || l > 62) return blb_fail(BLB_ERR_ARG, "need 2 <= l <= 62");
    if (!aligned16(w0) || !aligned16(w1)) return blb_fail(BLB_ERR_ARG, "share arrays must be 16-byte aligned");
    if (count == 0 || n == 0) return BLB_OK;
    Scratch S(c);
    int rc = BLB_OK;
    const size_t nin = (size_t)count * n * 8, nw = 2 * nin;
    const uint64_t* d0 = (const uint64_t*)dev_in(c, S, x0, nin, &rc);
    const uint64_t* d1 = rc ? nullptr : (const uint64_t*)dev_in(c, S, x1, nin, &rc);
    uint64_t* o0 = rc ? nullptr : (uint64_t*)dev_out(S, w0, nw, &rc);
    uint64_t* o1 = rc ? nullptr : (uint64_t*)dev_out(S, w1, nw, &rc);
    const uint32_t* dn = rc ? nullptr : S.upload(nonce_words(nonces, count));
    if (rc) return rc;
    if (!dn) return blb_fail(BLB_ERR_OOM, "nonce table");
    k_ext_wrap_sim<<<dim3((n + 255) / 256, count), 256, 0, c->stream>>>(d0, d1, o0, o1, n, (int)l, seed, dn);
    BLB_LAUNCHED();
    if (o0 != w0) BLB_TRY(copy_out(c, w0, o0, nw));
    if (o1 != w1) BLB_TRY(copy_out(c, w1, o1, nw));
    return BLB_OK;
}

extern "C" int blb_c2m_local(blb_ctx* c, uint32_t party, const uint64_t* t, const uint64_t* wsh, uint32_t count,
                             double scale, uint32_t l, uint32_t sf, uint64_t* out)
{
    if (!c || !t || !wsh || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (party > 1) return blb_fail(BLB_ERR_ARG, "party must be 0 or 1");
    if (!aligned16(wsh)) return blb_fail(BLB_ERR_ARG, "share arrays must be 16-byte aligned");
    BLB_TRY(check_fixed(c, l, sf));
    if (!(scale > 0) || !std::isfinite(scale)) return blb_fail(BLB_ERR_ARG, "scale must be positive");
    int ex;
    const double mu = 2.0 * frexp(scale, &ex);  // scale = mu 2^e, mu in [1, 2)
    const int sh_in = (ex - 1) - FX_P;
    if (sh_in >= 64 || sh_in <= -64) return blb_fail(BLB_ERR_ARG, "scale out of range");
    if (count == 0) return BLB_OK;
    const uint32_t N = c->N, s = N / 2, logs = c->logN - 1;
    BLB_TRY(fx_tables(c));
    const int2* twist;
    BLB_TRY(fx_twist(c, 1.0 / mu, &twist));
    Scratch S(c);
    int rc = BLB_OK;
    const uint64_t* dt = (const uint64_t*)dev_in(c, S, t, (size_t)count * N * 8, &rc);
    const uint64_t* dw = rc ? nullptr : (const uint64_t*)dev_in(c, S, wsh, (size_t)count * N * 16, &rc);
    uint64_t* dout = rc ? nullptr : (uint64_t*)dev_out(S, out, (size_t)count * s * 8, &rc);
    c128* A = rc ? nullptr : (c128*)S.get((size_t)count * s * sizeof(c128));
    if (rc) return rc;
    if (!A) return blb_fail(BLB_ERR_OOM, "conversion buffer");
    const uint64_t mask = (1ull << l) - 1;
    const dim3 grid(s / FX_E, count);
    {
        ProfScope ps(c, "c2m", (uint64_t)count * (N * 24ull + s * 8ull));
        if (party)
            FX_DISPATCH(logs, k_c2m_pass1<L_, true><<<grid, FX_T, 0, c->stream>>>(dt, dw, A, c->d_fx_root, twist,
                                                                                  c->q[0], sh_in));
        else
            FX_DISPATCH(logs, k_c2m_pass1<L_, false><<<grid, FX_T, 0, c->stream>>>(dt, dw, A, c->d_fx_root, twist,
                                                                                   c->q[0], sh_in));
        BLB_LAUNCHED();
        if (party)
            FX_DISPATCH(logs, k_c2m_pass2<L_, true><<<grid, FX_T, 0, c->stream>>>(A, dout, c->d_fx_root, c->d_kinv,
                                                                                  FX_P - (int)sf, mask));
        else
            FX_DISPATCH(logs, k_c2m_pass2<L_, false><<<grid, FX_T, 0, c->stream>>>(A, dout, c->d_fx_root, c->d_kinv,
                                                                                   FX_P - (int)sf, mask));
        BLB_LAUNCHED();
    }
    if (dout != out) BLB_TRY(copy_out(c, out, dout, (size_t)count * s * 8));
    return BLB_OK;
}

extern "C" int blb_m2c_local(blb_ctx* c, uint32_t party, const uint64_t* x, const uint64_t* wsh, uint32_t n,
                             uint32_t count, uint32_t level, double scale, uint32_t l, uint32_t sf, uint64_t* out)
{
    if (!c || !out || (n && (!x || !wsh))) return blb_fail(BLB_ERR_ARG, "null argument");
    if (party > 1) return blb_fail(BLB_ERR_ARG, "party must be 0 or 1");
    if (n && !aligned16(wsh)) return blb_fail(BLB_ERR_ARG, "share arrays must be 16-byte aligned");
    BLB_TRY(check_fixed(c, l, sf));
    if (level >= c->nQ) return blb_fail(BLB_ERR_LEVEL, "level out of range");
    if (n > c->N / 2) return blb_fail(BLB_ERR_ARG, "more values than slots");
    if (!(scale > 0) || !std::isfinite(scale)) return blb_fail(BLB_ERR_ARG, "scale must be positive");
    int ex;
    const double mu = frexp(scale, &ex);  // scale = mu 2^ex, mu in [0.5, 1)
    const int sh = FX_P + FX_F - ex;
    if (sh >= 64 || sh <= -64) return blb_fail(BLB_ERR_ARG, "scale out of range");
    if (count == 0) return BLB_OK;
    const uint32_t N = c->N, s = N / 2, logs = c->logN - 1, nl = level + 1;
    BLB_TRY(fx_tables(c));
    const int2* twist;
    BLB_TRY(fx_twist(c, mu, &twist));
    R2FConsts K{};
    for (uint32_t i = 0; i < nl; i++) {
        const uint64_t q = c->q[i];
        const uint64_t two64 = (uint64_t)(((unsigned __int128)1 << 64) % q);
        K.q[i] = q;
        K.two128[i] = host_mulmod(two64, two64, q);
        const unsigned __int128 R = ~(unsigned __int128)0 / q;  // floor((2^128 - 1) / q) = floor(2^128 / q)
        K.r0[i] = (uint64_t)R;
        K.r1[i] = (uint64_t)(R >> 64);
    }
    Scratch S(c);
    int rc = BLB_OK;
    const uint64_t* dx = nullptr;
    const uint64_t* dw = nullptr;
    if (n) {
        dx = (const uint64_t*)dev_in(c, S, x, (size_t)count * n * 8, &rc);
        if (!rc) dw = (const uint64_t*)dev_in(c, S, wsh, (size_t)count * n * 16, &rc);
    } else {
        dx = dw = (const uint64_t*)S.get(16);  // never read
    }
    const size_t out_bytes = (size_t)count * nl * N * 8;
    uint64_t* dout = rc ? nullptr : (uint64_t*)dev_out(S, out, out_bytes, &rc);
    c128* A = rc ? nullptr : (c128*)S.get((size_t)count * s * sizeof(c128));
    if (rc) return rc;
    if (!A || !dx) return blb_fail(BLB_ERR_OOM, "conversion buffer");
    const dim3 grid(s / FX_E, count);
    {
        ProfScope ps(c, "m2c", (uint64_t)count * (n * 24ull + out_bytes / count));
        if (party)
            FX_DISPATCH(logs, k_m2c_pass1<L_, true><<<grid, FX_T, 0, c->stream>>>(dx, dw, A, c->d_fx_root, c->d_kinv,
                                                                                  n, (int)l, FX_P - (int)sf));
        else
            FX_DISPATCH(logs, k_m2c_pass1<L_, false><<<grid, FX_T, 0, c->stream>>>(dx, dw, A, c->d_fx_root,
                                                                                   c->d_kinv, n, (int)l,
                                                                                   FX_P - (int)sf));
        BLB_LAUNCHED();
        if (party)
            FX_DISPATCH(logs, k_m2c_pass2<L_, true><<<grid, FX_T, 0, c->stream>>>(A, dout, c->d_fx_root, twist, K,
                                                                                  nl, sh));
        else
            FX_DISPATCH(logs, k_m2c_pass2<L_, false><<<grid, FX_T, 0, c->stream>>>(A, dout, c->d_fx_root, twist, K,
                                                                                   nl, sh));
        BLB_LAUNCHED();
    }
    if (dout != out) BLB_TRY(copy_out(c, out, dout, out_bytes));
    return BLB_OK;
}
