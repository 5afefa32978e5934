// matmul_cc.cu -- ciphertext x ciphertext matrix product of Sec. 5.1 (three
// steps, multi-head packing, baby-step giant-step of App. C.1).
//
// Packing: s = N/2 slots in blocks of L; block beta = h + Hg kappa of input
// ciphertext c holds column k = c Kc + kappa of A_h (spatial-first) or row k
// of B_h (reduce-first), element i at slot beta L + i, Kc = s / (L Hg).  Output
// ciphertext j (of L/Kc) holds diagonal delta = j Kc + kappa' of C_h = A_h B_h at
// block h + Hg kappa', element i = C_h[i][(i + delta) mod L].
//
// Schedule (b1s1 | Kc, b1s2 | L, G1 = Kc/b1s1, G2 = L/b1s2):
//   1. B'_c = Rescale( sum_{g1} Rot^{g1 b1s1}( sum_{b0} m1lo(g1,b0) Rot^{b0}(B_c)
//                                               + m1hi(g1,b0) Rot^{b0-L}(B_c) ) )
//      (block kappa of B'_c holds B[k][(i + kappa) mod L]);
//   2. for t = g b1s2 + b: V_{c,t} = m2lo(g,b) Rot^{b}(B'_c) + m2hi(g,b) Rot^{b-L}(B'_c),
//      W_t = Rescale( Relin( Rescale( sum_c Rot^{-g b1s2}(A_c) (x) V_{c,t} ) ) ), A_c at
//      level-1 (one rescale of the sum over c instead of one per V_{c,t}; the
//      depth, 4, is unchanged).  The tensor product is bilinear, so the sum is
//      m2lo(t) (.) sum_c AG_{c,g} (x) BLO_{c,b} + m2hi(t) (.) sum_c AG_{c,g} (x) BHI_{c,b}:
//      one kernel forms both sums and applies the masks (k_cc_step2);
//   3. C_j = Rescale( sum_t m3(t,j) Rot^{g b1s2 - (t mod Kc) Hg L}(W_t) ).
// Masks are 0/1 slot vectors encoded at scale q_l of the level they are applied
// at (so masking and its rescale leave the scale unchanged):
//   m1lo(g1,b0) = Rot^{-g1 b1s1}[kappa(slot) = g1 b1s1 + b0, i < L - kappa]   (hi: i >= L - kappa)
//   m2lo(g,b)   = Rot^{-g b1s2}[i < L - t]                                    (hi: i >= L - t)
//   m3(t,j)     = [the block landing at kappa' comes from kappa = (kappa' - t) mod Kc and
//                  carries diagonal (t + kappa) mod L of output j]
// m3(t,j) is constant on every block and depends on the block's kappa' only;
// for t = a Kc + r it is [kappa' >= r] for j = a and [kappa' < r] for
// j = a + 1 (mod L/Kc), so the L^2/Kc step-3 masks hold at most 2 Kc distinct
// plaintexts and each is encoded and stored once.
// Depth 4: step-1 masks, step-2 masks, the tensor product, step-3 masks.
#include <algorithm>
#include <cstring>
#include <map>

#include "common.cuh"

struct blb_cc_plan {
    blb_ctx* ctx;
    uint32_t L, Hg, R, level, Kc, n_c, nout, b1s1, b1s2, G1, G2;
    uint32_t c_chunk, t_chunk;  // input ciphertexts and diagonals per pass of steps 1-2
    uint64_t* d_m1;  // [G1][b1s1][2] at level, (level+1) x N each
    uint64_t* d_m2;  // [G2][b1s2][2] at level-1
    uint64_t* d_m3;  // [n3] distinct step-3 masks at level-3
    std::vector<uint8_t> nz1, nz2;
    std::vector<int32_t> m3_index;  // [L][nout]: row of d_m3, -1 for an all-zero mask
    size_t b1, b2, b3, bytes;
};

namespace {
constexpr int kT = 256;

struct MaskSpec {
    uint32_t L, Hg, Kc, s, b1s1, b1s2, nout;
};

// mask value at slot (before the giant-step rotation) for mask id of `type`
__host__ __device__ inline bool mask_pred(const MaskSpec& m, int type, uint32_t id, uint32_t slot)
{
    const uint32_t i = slot % m.L, kap = (slot / m.L) / m.Hg;
    if (type == 1) {  // id = (g1 b1s1 + b0) * 2 + hi
        const uint32_t kappa = id >> 1, hi = id & 1;
        if (kap != kappa) return false;
        return hi ? i >= m.L - kappa : i < m.L - kappa;
    }
    if (type == 2) {  // id = t * 2 + hi
        const uint32_t t = id >> 1, hi = id & 1;
        return hi ? i >= m.L - t : i < m.L - t;
    }
    // type 3: id = t * nout + j
    const uint32_t t = id / m.nout, j = id % m.nout;
    const uint32_t kappa = (uint32_t)(((int64_t)kap - (int64_t)t) % (int64_t)m.Kc + m.Kc) % m.Kc;
    const uint32_t delta = (t + kappa) % m.L;
    return delta / m.Kc == j;
}

__host__ __device__ inline uint32_t mask_shift(const MaskSpec& m, int type, uint32_t id)
{
    if (type == 1) return ((id >> 1) / m.b1s1) * m.b1s1;  // g1 b1s1
    if (type == 2) return ((id >> 1) / m.b1s2) * m.b1s2;  // g b1s2
    return 0;
}

// z[m][slot] = mask(type, id) at slot (slot - shift) mod s, id = ids[first + m]
// (first + m without a table)
__global__ void k_cc_masks(double* __restrict__ z, MaskSpec spec, int type, uint32_t first,
                           const uint32_t* __restrict__ ids)
{
    const uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y;
    if (slot >= spec.s) return;
    const uint32_t id = ids ? ids[first + m] : first + m;
    const uint32_t src = (slot + spec.s - mask_shift(spec, type, id) % spec.s) % spec.s;
    z[(size_t)m * spec.s + slot] = mask_pred(spec, type, id, src) ? 1.0 : 0.0;
}

// out[o] = sum_{t in [start[o], start[o+1])} ct[t] (.) pt[t]  (2 polynomials, n limbs)
struct LcTerm {
    const uint64_t* ct;
    const uint64_t* pt;
};
__global__ void k_lincomb(uint64_t* __restrict__ out, const uint32_t* __restrict__ start,
                          const LcTerm* __restrict__ terms, uint32_t n, uint32_t N, const uint64_t* __restrict__ qs,
                          const uint64_t* __restrict__ bar)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y, o = blockIdx.z;
    if (c >= N) return;
    const uint64_t q = qs[i], r0 = bar[2 * i], r1 = bar[2 * i + 1];
    const size_t nN = (size_t)n * N, off = (size_t)i * N + c;
    acc128 a0{0, 0}, a1{0, 0};
    const uint32_t t0 = start[o], t1 = start[o + 1];
    for (uint32_t t = t0; t < t1; t++) {
        const uint64_t w = terms[t].pt[off];
        mad128(a0, terms[t].ct[off], w);
        mad128(a1, terms[t].ct[nN + off], w);
        if (((t - t0) & 7) == 7) {
            a0 = acc128{barrett128(a0.lo, a0.hi, q, r0, r1), 0};
            a1 = acc128{barrett128(a1.lo, a1.hi, q, r0, r1), 0};
        }
    }
    uint64_t* dst = out + (size_t)o * 2 * nN + off;
    dst[0] = barrett128(a0.lo, a0.hi, q, r0, r1);
    dst[nN] = barrett128(a1.lo, a1.hi, q, r0, r1);
}

// Step 2 for diagonals t in [t0, t0 + gridDim.x): with g = t / b1s2, b = t % b1s2,
//   X = sum_{c < cn} AG[c][g] (x) BLO[c][b],  Y = sum_{c < cn} AG[c][g] (x) BHI[c][b]
//   U[t] (+)= mlo(t) (.) X + mhi(t) (.) Y
// (x) = (a0 b0, a0 b1 + a1 b0, a1 b1); the middle term by Karatsuba as
// (a0 + a1)(b0 + b1) - a0 b0 - a1 b1 (three products, operand sums < 2q, lazy
// 128-bit sums reduced every 8 terms: at most 8 (2q)^2 + q < 2^126 for q < 2^60).
// AG, BLO, BHI: stacks of 2-polynomial ciphertexts of n limbs (stride 2 n N),
// indexed c G2 + g and c b1s2 + b; U: 3-polynomial ciphertexts, U[t - t0] at
// U + (t - t0) 3 n N.  The diagonal is the fastest grid index so that the
// blocks running together share their AG / BLO / BHI tiles in L2.
struct MaskPair {
    const uint64_t* lo;  // (n) x N words at the mask level, nullptr = all-zero mask
    const uint64_t* hi;
};
constexpr int kS2 = 128;
__global__ void __launch_bounds__(kS2) k_cc_step2(uint64_t* __restrict__ U, const uint64_t* __restrict__ AG,
                                                  const uint64_t* __restrict__ BLO, const uint64_t* __restrict__ BHI,
                                                  const MaskPair* __restrict__ masks, uint32_t t0, uint32_t cn,
                                                  uint32_t b1s2, uint32_t G2, uint32_t n, uint32_t N,
                                                  const uint64_t* __restrict__ qs, const uint64_t* __restrict__ bar,
                                                  bool accumulate)
{
    const uint32_t t = t0 + blockIdx.x, k = blockIdx.y * kS2 + threadIdx.x, i = blockIdx.z;
    if (k >= N) return;
    const uint32_t g = t / b1s2, b = t % b1s2;
    const uint64_t q = qs[i], r0 = bar[2 * i], r1 = bar[2 * i + 1];
    // lazy 128-bit sums: every product is below (2q)^2; for q < 2^50 that is
    // 2^102, so any count of input ciphertexts below 2^25 sums without a
    // reduction; larger primes reduce every 8 terms (8 (2q)^2 < 2^128 for q < 2^62)
    const bool reduce8 = q >= (1ull << 50);
    const size_t nN = (size_t)n * N, off = (size_t)i * N + k, cw = 2 * nN;
    const MaskPair mp = masks[t];
    const bool use_lo = mp.lo != nullptr, use_hi = mp.hi != nullptr;
    const size_t sa = (size_t)G2 * cw, sb = (size_t)b1s2 * cw;
    // one pass over the input ciphertexts per mask (three 128-bit sums live at
    // a time): sum_c AG (x) V for V = BLO, then V = BHI
    auto tensor_sum = [&](const uint64_t* pv, uint64_t& Z0, uint64_t& Z1, uint64_t& Z2) {
        acc128 z0{0, 0}, zs{0, 0}, z2{0, 0};
        const uint64_t* pa = AG + (size_t)g * cw + off;
        for (uint32_t c = 0; c < cn; c++) {
            const uint64_t a0 = pa[0], a1 = pa[nN], v0 = pv[0], v1 = pv[nN];
            mad128(z0, a0, v0);
            mad128(z2, a1, v1);
            mad128(zs, a0 + a1, v0 + v1);
            if (reduce8 && (c & 7) == 7) {
                z0 = acc128{barrett128(z0.lo, z0.hi, q, r0, r1), 0};
                zs = acc128{barrett128(zs.lo, zs.hi, q, r0, r1), 0};
                z2 = acc128{barrett128(z2.lo, z2.hi, q, r0, r1), 0};
            }
            pa += sa;
            pv += sb;
        }
        Z0 = barrett128(z0.lo, z0.hi, q, r0, r1);
        Z2 = barrett128(z2.lo, z2.hi, q, r0, r1);
        Z1 = sub_mod(sub_mod(barrett128(zs.lo, zs.hi, q, r0, r1), Z0, q), Z2, q);
    };
    uint64_t X0 = 0, X1 = 0, X2 = 0, Y0 = 0, Y1 = 0, Y2 = 0;
    if (use_lo) tensor_sum(BLO + (size_t)b * cw + off, X0, X1, X2);
    if (use_hi) tensor_sum(BHI + (size_t)b * cw + off, Y0, Y1, Y2);
    const uint64_t ml = use_lo ? mp.lo[off] : 0, mh = use_hi ? mp.hi[off] : 0;
    uint64_t* dst = U + (size_t)blockIdx.x * 3 * nN + off;
    const uint64_t Xv[3] = {X0, X1, X2}, Yv[3] = {Y0, Y1, Y2};
#pragma unroll
    for (int poly = 0; poly < 3; poly++) {
        acc128 u{accumulate ? dst[poly * nN] : 0, 0};
        mad128(u, ml, Xv[poly]);
        mad128(u, mh, Yv[poly]);
        dst[poly * nN] = barrett128(u.lo, u.hi, q, r0, r1);
    }
}

// copy polynomials from `from` limbs per polynomial to `to` limbs (drop the top limbs)
__global__ void k_drop(uint64_t* __restrict__ out, const uint64_t* __restrict__ in, uint32_t from, uint32_t to,
                       uint32_t N)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y, poly = blockIdx.z;
    if (c >= N) return;
    out[((size_t)poly * to + i) * N + c] = in[((size_t)poly * from + i) * N + c];
}

// Device copy of a host table.  Under stream capture the copy goes to a buffer
// the context keeps (a graph replays the launches that read it) and *bytes is
// 0, so free_table leaves it alone.
template <class T>
int upload_table(blb_ctx* c, const std::vector<T>& v, T** d, size_t* bytes)
{
    if (capturing(c)) {
        *bytes = 0;
        return persist_upload(c, v.data(), v.size() * sizeof(T), (void**)d);
    }
    *bytes = std::max<size_t>(v.size() * sizeof(T), 16);
    *d = (T*)dev_alloc(c, *bytes);
    if (!*d) return blb_fail(BLB_ERR_OOM, "table allocation failed");
    BLB_CUDA(cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return BLB_OK;
}

void free_table(blb_ctx* c, void* d, size_t bytes)
{
    if (d && bytes) dev_free(c, d, bytes);
}

// Device buffer holding `count` ciphertexts of 2 polynomials at `level`
struct Stack {
    blb_ctx* c = nullptr;
    uint64_t* d = nullptr;
    size_t bytes = 0, words_per = 0;
    int alloc(blb_ctx* ctx, uint32_t count, uint32_t level, uint32_t npolys = 2)
    {
        c = ctx;
        words_per = (size_t)npolys * (level + 1) * ctx->N;
        bytes = std::max<size_t>((size_t)count * words_per * 8, 16);
        d = (uint64_t*)dev_alloc(ctx, bytes);
        return d ? BLB_OK : blb_fail(BLB_ERR_OOM, "matmul_cc workspace");
    }
    uint64_t* at(size_t k) const { return d + k * words_per; }
    ~Stack()
    {
        if (d) dev_free(c, d, bytes);
    }
};

}  // namespace

// Rescale `count` ciphertexts of npolys polynomials stored back to back (in:
// level l, out: level l-1).
static int rescale_many(blb_ctx* c, uint64_t* out, const uint64_t* in, uint32_t level, uint32_t count,
                        uint32_t npolys)
{
    // the rescale kernels treat count * npolys polynomials as one stack
    return launch_rescale_stack(c, out, in, level, count * npolys);
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
static MaskSpec spec_of(const blb_cc_plan* P)
{
    return MaskSpec{P->L, P->Hg, P->Kc, P->ctx->N / 2, P->b1s1, P->b1s2, P->nout};
}

static int encode_masks(blb_ctx* c, const MaskSpec& spec, int type, uint32_t count, uint32_t level, uint64_t* out,
                        const uint32_t* d_ids = nullptr)
{
    const uint32_t s = spec.s, n = level + 1;
    const uint32_t chunk = std::max<uint32_t>(1, std::min<uint32_t>(count, (uint32_t)((32ull << 20) / ((uint64_t)s * 8))));
    double* z = (double*)dev_alloc(c, (size_t)chunk * s * 8);
    if (!z) return blb_fail(BLB_ERR_OOM, "mask buffer");
    int rc = BLB_OK;
    for (uint32_t first = 0; !rc && first < count; first += chunk) {
        const uint32_t cnt = std::min(chunk, count - first);
        k_cc_masks<<<dim3((s + kT - 1) / kT, cnt), kT, 0, c->stream>>>(z, spec, type, first, d_ids);
        if (cudaGetLastError() != cudaSuccess) rc = blb_fail(BLB_ERR_CUDA, "mask kernel launch failed");
        else {
            blb_count_launch();
            rc = encode_slots(c, z, cnt, s, level, (double)c->q[level], out + (size_t)first * n * c->N);
        }
    }
    dev_free(c, z, (size_t)chunk * s * 8);
    return rc;
}

extern "C" int blb_cc_plan_create(blb_ctx* c, uint32_t L, uint32_t Hg, uint32_t R, uint32_t level,
                                  const blb_cc_sched* sched, blb_cc_plan** out)
{
    if (!c || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    *out = nullptr;
    BLB_TRY(refuse_capture(c, "plan creation"));
    const uint32_t s = c->N / 2;
    if (L == 0 || Hg == 0 || (L & (L - 1)) || (Hg & (Hg - 1)) || s % (L * Hg))
        return blb_fail(BLB_ERR_ARG, "L and Hg must be powers of two with L Hg dividing N/2");
    const uint32_t Kc = s / (L * Hg);
    if (Kc == 0 || Kc > L) return blb_fail(BLB_ERR_ARG, "need Kc = N/2/(L Hg) <= L");
    if (R == 0 || R > L) return blb_fail(BLB_ERR_ARG, "R must be in [1, L]");
    if (level < 4 || level >= c->nQ) return blb_fail(BLB_ERR_LEVEL, "matmul_cc needs 4 levels");
    uint32_t b1s1 = sched ? sched->b1s1 : 0, b1s2 = sched ? sched->b1s2 : 0;
    if (b1s1 == 0) {
        b1s1 = 1;
        while (2 * b1s1 * b1s1 * 2 <= Kc) b1s1 <<= 1;  // about sqrt(Kc/2)
    }
    if (b1s2 == 0) {
        b1s2 = 1;
        while (2 * b1s2 * b1s2 * 2 <= L) b1s2 <<= 1;
    }
    if (Kc % b1s1 || L % b1s2) return blb_fail(BLB_ERR_ARG, "b1s1 must divide Kc and b1s2 must divide L");
    blb_cc_plan* P = new blb_cc_plan();
    P->ctx = c;
    ctx_retain(c);
    P->L = L;
    P->Hg = Hg;
    P->R = R;
    P->level = level;
    P->Kc = Kc;
    P->n_c = (R + Kc - 1) / Kc;
    P->nout = L / Kc;
    P->b1s1 = b1s1;
    P->b1s2 = b1s2;
    P->G1 = Kc / b1s1;
    P->G2 = L / b1s2;
    P->d_m1 = P->d_m2 = P->d_m3 = nullptr;
    const uint32_t N = c->N;
    {  // chunking of steps 1-2 under the workspace budget
        const uint64_t l0 = level + 1, l1 = level, l2 = level - 1;
        const uint64_t per_c = 16ull * N * ((2ull * b1s1 + P->G1 + 1) * l0 + (2ull + 2ull * b1s2 + P->G2) * l1);
        (void)l2;
        const uint64_t budget = (sched && sched->workspace_bytes) ? sched->workspace_bytes : (24ull << 30);
        uint32_t Cc = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(P->n_c, budget / per_c)), Tc = L;
        if (sched && sched->c_chunk) Cc = std::min(sched->c_chunk, P->n_c);
        if (sched && sched->t_chunk) Tc = std::min(sched->t_chunk, L);
        P->c_chunk = Cc;
        P->t_chunk = Tc;
    }
    const MaskSpec spec = spec_of(P);
    // distinct step-3 masks: the predicate depends on the block's kappa' only,
    // so a mask is identified by its values on the Kc blocks (slot kappa' Hg L)
    std::vector<uint32_t> rep3;
    {
        std::map<std::vector<uint8_t>, int32_t> seen;
        P->m3_index.assign((size_t)L * P->nout, -1);
        std::vector<uint8_t> sig(Kc);
        for (uint32_t t = 0; t < L; t++)
            for (uint32_t j = 0; j < P->nout; j++) {
                const uint32_t id = t * P->nout + j;
                bool any = false;
                for (uint32_t kap = 0; kap < Kc; kap++) {
                    sig[kap] = mask_pred(spec, 3, id, kap * Hg * L) ? 1 : 0;
                    any |= sig[kap] != 0;
                }
                if (!any) continue;
                auto it = seen.find(sig);
                if (it == seen.end()) {
                    it = seen.emplace(sig, (int32_t)rep3.size()).first;
                    rep3.push_back(id);
                }
                P->m3_index[id] = it->second;
            }
    }
    const size_t n1 = 2ull * Kc, n2 = 2ull * L, n3 = rep3.size();
    P->b1 = n1 * (level + 1) * N * 8;
    P->b2 = n2 * level * N * 8;
    P->b3 = std::max<size_t>(n3 * (level - 2) * N * 8, 16);
    P->bytes = P->b1 + P->b2 + P->b3;
    P->d_m1 = (uint64_t*)dev_alloc(c, P->b1);
    P->d_m2 = (uint64_t*)dev_alloc(c, P->b2);
    P->d_m3 = (uint64_t*)dev_alloc(c, P->b3);
    int rc = (P->d_m1 && P->d_m2 && P->d_m3) ? BLB_OK : blb_fail(BLB_ERR_OOM, "mask plaintexts do not fit");
    // which masks are non-zero (host evaluation of the same predicates)
    auto nonzero = [&](int type, uint32_t id) {
        for (uint32_t slot = 0; slot < s; slot++)
            if (mask_pred(spec, type, id, slot)) return (uint8_t)1;
        return (uint8_t)0;
    };
    P->nz1.resize(n1);
    P->nz2.resize(n2);
    for (size_t k = 0; k < n1; k++) P->nz1[k] = nonzero(1, (uint32_t)k);
    for (size_t k = 0; k < n2; k++) P->nz2[k] = nonzero(2, (uint32_t)k);
    if (!rc) rc = encode_masks(c, spec, 1, (uint32_t)n1, level, P->d_m1);
    if (!rc) rc = encode_masks(c, spec, 2, (uint32_t)n2, level - 1, P->d_m2);
    if (!rc && n3) {
        uint32_t* d_ids = nullptr;
        size_t bi = 0;
        rc = upload_table(c, rep3, &d_ids, &bi);
        if (!rc) rc = encode_masks(c, spec, 3, (uint32_t)n3, level - 3, P->d_m3, d_ids);
        free_table(c, d_ids, bi);
    }
    if (rc) {
        blb_cc_plan_free(P);
        return rc;
    }
    *out = P;
    return BLB_OK;
}

extern "C" void blb_cc_plan_free(blb_cc_plan* P)
{
    if (!P) return;
    blb_ctx* c = P->ctx;
    dev_free(c, P->d_m1, P->b1);
    dev_free(c, P->d_m2, P->b2);
    dev_free(c, P->d_m3, P->b3);
    delete P;
    ctx_release(c);
}

static int32_t step3_rot(const blb_cc_plan* P, uint32_t t)
{
    const int64_t s = P->ctx->N / 2;
    const int64_t g = t / P->b1s2;
    return (int32_t)((((int64_t)g * P->b1s2 - (int64_t)(t % P->Kc) * P->Hg * P->L) % s + s) % s);
}

static std::vector<int32_t> plan_rotations(const blb_cc_plan* P)
{
    std::vector<int32_t> r;
    auto add = [&](int64_t x) {
        const int64_t s = P->ctx->N / 2;
        int32_t v = (int32_t)x;
        if (((x % s) + s) % s == 0) return;
        if (std::find(r.begin(), r.end(), v) == r.end()) r.push_back(v);
    };
    for (uint32_t b0 = 1; b0 < P->b1s1; b0++) add(b0);
    for (uint32_t b0 = 0; b0 < P->b1s1; b0++) add((int64_t)b0 - P->L);
    for (uint32_t g1 = 1; g1 < P->G1; g1++) add((int64_t)g1 * P->b1s1);
    for (uint32_t b = 1; b < P->b1s2; b++) add(b);
    for (uint32_t b = 0; b < P->b1s2; b++) add((int64_t)b - P->L);
    for (uint32_t g = 1; g < P->G2; g++) add(-(int64_t)g * P->b1s2);
    for (uint32_t t = 1; t < P->L; t++) add(step3_rot(P, t));
    return r;
}

extern "C" int blb_cc_plan_info(const blb_cc_plan* P, uint32_t* n_c, uint32_t* Kc, uint32_t* nout, uint32_t* b1s1,
                                uint32_t* b1s2, uint64_t* mask_bytes, uint32_t* c_chunk, uint32_t* t_chunk)
{
    if (!P) return blb_fail(BLB_ERR_ARG, "null plan");
    if (n_c) *n_c = P->n_c;
    if (Kc) *Kc = P->Kc;
    if (nout) *nout = P->nout;
    if (b1s1) *b1s1 = P->b1s1;
    if (b1s2) *b1s2 = P->b1s2;
    if (mask_bytes) *mask_bytes = P->bytes;
    if (c_chunk) *c_chunk = P->c_chunk;
    if (t_chunk) *t_chunk = P->t_chunk;
    return BLB_OK;
}

extern "C" int blb_cc_plan_rotations(const blb_cc_plan* P, int32_t* out, uint32_t cap, uint32_t* count)
{
    if (!P || !count) return blb_fail(BLB_ERR_ARG, "null argument");
    std::vector<int32_t> r = plan_rotations(P);
    *count = (uint32_t)r.size();
    if (out) {
        if (cap < r.size()) return blb_fail(BLB_ERR_ARG, "rotation buffer too small");
        memcpy(out, r.data(), r.size() * 4);
    }
    return BLB_OK;
}

// ---------------------------------------------------------------------------
// run
// ---------------------------------------------------------------------------
static int lincomb(blb_ctx* c, uint64_t* out, uint32_t nout, const std::vector<uint32_t>& start,
                   const std::vector<LcTerm>& terms, uint32_t level)
{
    uint32_t* d_start = nullptr;
    LcTerm* d_terms = nullptr;
    size_t bs = 0, bt = 0;
    int rc = upload_table(c, start, &d_start, &bs);
    if (!rc) rc = upload_table(c, terms, &d_terms, &bt);
    if (!rc) {
        k_lincomb<<<dim3((c->N + kT - 1) / kT, level + 1, nout), kT, 0, c->stream>>>(out, d_start, d_terms, level + 1,
                                                                                   c->N, c->d_q, c->d_bar);
        if (cudaGetLastError() != cudaSuccess) rc = blb_fail(BLB_ERR_CUDA, "lincomb launch failed");
        else blb_count_launch();
    }
    free_table(c, d_start, bs);
    free_table(c, d_terms, bt);
    return rc;
}

static const uint64_t* key_for(const blb_keys* K, uint32_t N, int32_t rot, int* rc)
{
    const KeyEntry* k = K->find(galois_element(N, rot));
    if (!k) *rc = blb_fail(BLB_ERR_NO_KEY, "no Galois key for rotation " + std::to_string(rot));
    return k ? k->d : nullptr;
}

// Hoisted rotations: every source ciphertext srcs[i] (2 polynomials at `level`)
// rotated by every amount rots[j] into out(i, j); one ModUp per source.
template <typename Out>
static int rotate_hoisted(blb_ctx* c, const blb_keys* K, uint32_t level, const std::vector<const uint64_t*>& srcs,
                          const std::vector<int32_t>& rots, Out out)
{
    if (srcs.empty() || rots.empty()) return BLB_OK;
    const size_t pw = (size_t)(level + 1) * c->N;
    int rc = BLB_OK;
    std::vector<const uint64_t*> keys(rots.size());
    std::vector<uint64_t> gal(rots.size());
    for (size_t j = 0; j < rots.size() && !rc; j++) {
        keys[j] = key_for(K, c->N, rots[j], &rc);
        gal[j] = galois_element(c->N, rots[j]);
    }
    if (rc) return rc;
    std::vector<KsSource> src;
    std::vector<KsProduct> prod;
    std::vector<KsGroup> grp;
    std::vector<KsAdd> adds;
    for (uint32_t i = 0; i < srcs.size(); i++) {
        src.push_back(KsSource{srcs[i] + pw, 1});
        for (uint32_t j = 0; j < rots.size(); j++) {
            uint64_t* o = out(i, j);
            grp.push_back(KsGroup{o, o + pw, (uint32_t)prod.size(), (uint32_t)prod.size() + 1, (uint32_t)adds.size(),
                                  (uint32_t)adds.size() + 1});
            prod.push_back(KsProduct{i, gal[j], keys[j]});
            adds.push_back(KsAdd{srcs[i], gal[j], 0});
        }
    }
    return ks_run(c, level, src.data(), (uint32_t)src.size(), prod.data(), grp.data(), (uint32_t)grp.size(),
                  adds.data(), 0);
}

// out[i] = base[i] + sum_{j >= 1} Rot^{rots[j-1]}(T(i, j)), the inner products of
// all terms of one output summed over Q_l u P before one ModDown.
template <typename Term>
static int rotate_sum(blb_ctx* c, const blb_keys* K, uint32_t level, const std::vector<const uint64_t*>& base,
                      const std::vector<uint64_t*>& out, const std::vector<int32_t>& rots, Term T)
{
    if (base.empty()) return BLB_OK;
    const size_t pw = (size_t)(level + 1) * c->N;
    int rc = BLB_OK;
    std::vector<const uint64_t*> keys(rots.size());
    std::vector<uint64_t> gal(rots.size());
    for (size_t j = 0; j < rots.size() && !rc; j++) {
        keys[j] = key_for(K, c->N, rots[j], &rc);
        gal[j] = galois_element(c->N, rots[j]);
    }
    if (rc) return rc;
    std::vector<KsSource> src;
    std::vector<KsProduct> prod;
    std::vector<KsGroup> grp;
    std::vector<KsAdd> adds;
    for (uint32_t i = 0; i < base.size(); i++) {
        KsGroup G{out[i], out[i] + pw, (uint32_t)prod.size(), 0, (uint32_t)adds.size(), 0};
        adds.push_back(KsAdd{base[i], 1, 0});
        adds.push_back(KsAdd{base[i] + pw, 1, 1});
        for (uint32_t j = 0; j < rots.size(); j++) {
            const uint64_t* t = T(i, j + 1);
            prod.push_back(KsProduct{(uint32_t)src.size(), 1, keys[j]});
            src.push_back(KsSource{t + pw, gal[j]});
            adds.push_back(KsAdd{t, gal[j], 0});
        }
        G.prod1 = (uint32_t)prod.size();
        G.add1 = (uint32_t)adds.size();
        grp.push_back(G);
    }
    return ks_run(c, level, src.data(), (uint32_t)src.size(), prod.data(), grp.data(), (uint32_t)grp.size(),
                  adds.data(), 0);
}

extern "C" int blb_matmul_cc_plan(blb_ctx* c, const blb_keys* K, const blb_cc_plan* P, blb_ct* const* A,
                                  blb_ct* const* B, uint32_t n_in, blb_ct** C)
{
    if (!c || !K || !P || !A || !B || !C) return blb_fail(BLB_ERR_ARG, "null argument");
    if (n_in != P->n_c) return blb_fail(BLB_ERR_ARG, "number of input ciphertexts does not match the plan");
    for (uint32_t i = 0; i < n_in; i++) {
        if (!A[i] || !B[i] || A[i]->level != P->level || B[i]->level != P->level || A[i]->npolys != 2 ||
            B[i]->npolys != 2)
            return blb_fail(BLB_ERR_LEVEL, "input ciphertexts must be 2-polynomial ciphertexts at the plan's level");
        if (std::fabs(A[i]->scale - A[0]->scale) > 1e-9 * A[0]->scale ||
            std::fabs(B[i]->scale - B[0]->scale) > 1e-9 * B[0]->scale)
            return blb_fail(BLB_ERR_SCALE, "inputs have different scales");
    }
    if (!K->find(0)) return blb_fail(BLB_ERR_NO_KEY, "matmul_cc needs the relinearization key");
    for (uint32_t j = 0; j < P->nout; j++) C[j] = nullptr;
    const uint32_t N = c->N, n_c = P->n_c, L = P->L, l0 = P->level;
    const uint32_t l1 = l0 - 1, l2 = l0 - 2, l3 = l0 - 3;
    const size_t pw0 = (size_t)(l0 + 1) * N, pw1 = (size_t)(l1 + 1) * N, pw2 = (size_t)(l2 + 1) * N,
                 pw3 = (size_t)(l3 + 1) * N;
    int rc = BLB_OK;
    std::vector<KsItem> items;

    // Steps 1 and 2 run over chunks of Cc input ciphertexts; the step-2 sums of
    // every chunk are added into U mod q, so the result does not depend on the
    // chunking.  Step 2 is launched for Tc diagonals at a time.
    const uint32_t Cc = P->c_chunk, Tc = P->t_chunk;
    Stack LO, HI, INNER, ACC, BP, BLO, BHI, A1, AG, U, U2, WP, W;
    rc = LO.alloc(c, Cc * P->b1s1, l0);
    if (!rc) rc = HI.alloc(c, Cc * P->b1s1, l0);
    if (!rc) rc = INNER.alloc(c, Cc * P->G1, l0);
    if (!rc) rc = ACC.alloc(c, Cc, l0);
    if (!rc) rc = BP.alloc(c, Cc, l1);
    if (!rc) rc = BLO.alloc(c, Cc * P->b1s2, l1);
    if (!rc) rc = BHI.alloc(c, Cc * P->b1s2, l1);
    if (!rc) rc = A1.alloc(c, Cc, l1);
    if (!rc) rc = AG.alloc(c, Cc * P->G2, l1);
    if (!rc) rc = U.alloc(c, L, l1, 3);
    if (!rc) rc = U2.alloc(c, L, l2, 3);
    std::vector<MaskPair> mpairs(L);
    for (uint32_t t = 0; t < L; t++)
        mpairs[t] = MaskPair{P->nz2[2 * t] ? P->d_m2 + (size_t)(2 * t) * pw1 : nullptr,
                             P->nz2[2 * t + 1] ? P->d_m2 + (size_t)(2 * t + 1) * pw1 : nullptr};
    MaskPair* d_mpairs = nullptr;
    size_t bmp = 0;
    if (!rc) rc = upload_table(c, mpairs, &d_mpairs, &bmp);
    if (!rc) rc = WP.alloc(c, L, l2);
    if (!rc) rc = W.alloc(c, L, l3);
    for (uint32_t c0 = 0; !rc && c0 < n_c; c0 += Cc) {
        const uint32_t cn = std::min(Cc, n_c - c0);
        // ---- step 1 ----
        {  // baby steps: Rot^{b0}(B_c) (b0 >= 1) and Rot^{b0 - L}(B_c), hoisted per B_c
            std::vector<const uint64_t*> srcs;
            std::vector<int32_t> rots;
            for (uint32_t ci = 0; ci < cn; ci++) srcs.push_back(B[c0 + ci]->d);
            for (uint32_t b0 = 1; b0 < P->b1s1; b0++) rots.push_back((int32_t)b0);
            for (uint32_t b0 = (P->G1 > 1 ? 0 : 1); b0 < P->b1s1; b0++) rots.push_back((int32_t)b0 - (int32_t)L);
            for (uint32_t ci = 0; !rc && ci < cn; ci++)
                if (cudaMemcpyAsync(LO.at((size_t)ci * P->b1s1), B[c0 + ci]->d, 2 * pw0 * 8, cudaMemcpyDeviceToDevice,
                                    c->stream))
                    rc = blb_fail(BLB_ERR_CUDA, "copy failed");
            if (!rc)
                rc = rotate_hoisted(c, K, l0, srcs, rots, [&](uint32_t i, uint32_t j) {
                    const int32_t r = rots[j];
                    return r > 0 ? LO.at((size_t)i * P->b1s1 + r) : HI.at((size_t)i * P->b1s1 + (r + (int32_t)L));
                });
        }
        if (!rc) {  // inner[c][g1] = sum_b0 m1lo LO + m1hi HI
            std::vector<uint32_t> start{0};
            std::vector<LcTerm> terms;
            for (uint32_t ci = 0; ci < cn; ci++)
                for (uint32_t g1 = 0; g1 < P->G1; g1++) {
                    for (uint32_t b0 = 0; b0 < P->b1s1; b0++) {
                        const uint32_t kappa = g1 * P->b1s1 + b0;
                        for (uint32_t hi = 0; hi < 2; hi++) {
                            const uint32_t id = kappa * 2 + hi;
                            if (!P->nz1[id]) continue;
                            const uint64_t* ct = (hi ? HI : LO).at((size_t)ci * P->b1s1 + b0);
                            terms.push_back(LcTerm{ct, P->d_m1 + (size_t)id * pw0});
                        }
                    }
                    start.push_back((uint32_t)terms.size());
                }
            rc = lincomb(c, INNER.d, cn * P->G1, start, terms, l0);
        }
        if (!rc) {  // ACC[c] = INNER[c][0] + sum_{g1 >= 1} Rot^{g1 b1s1}(INNER[c][g1]), one ModDown per c
            std::vector<const uint64_t*> base;
            std::vector<uint64_t*> out;
            std::vector<int32_t> rots;
            for (uint32_t ci = 0; ci < cn; ci++) {
                base.push_back(INNER.at((size_t)ci * P->G1));
                out.push_back(ACC.at(ci));
            }
            for (uint32_t g1 = 1; g1 < P->G1; g1++) rots.push_back((int32_t)(g1 * P->b1s1));
            if (P->G1 == 1) {
                for (uint32_t ci = 0; !rc && ci < cn; ci++)
                    if (cudaMemcpyAsync(ACC.at(ci), base[ci], 2 * pw0 * 8, cudaMemcpyDeviceToDevice, c->stream))
                        rc = blb_fail(BLB_ERR_CUDA, "copy failed");
            } else {
                rc = rotate_sum(c, K, l0, base, out, rots,
                                [&](uint32_t i, uint32_t j) { return INNER.at((size_t)i * P->G1 + j); });
            }
        }
        if (!rc) rc = rescale_many(c, BP.d, ACC.d, l0, cn, 2);

        // ---- step 2 ----
        if (!rc) {  // baby steps: Rot^{b}(B'_c) (b >= 1) and Rot^{b - L}(B'_c), hoisted per B'_c
            std::vector<const uint64_t*> srcs;
            std::vector<int32_t> rots;
            for (uint32_t ci = 0; ci < cn; ci++) srcs.push_back(BP.at(ci));
            for (uint32_t b = 1; b < P->b1s2; b++) rots.push_back((int32_t)b);
            for (uint32_t b = (P->G2 > 1 ? 0 : 1); b < P->b1s2; b++) rots.push_back((int32_t)b - (int32_t)L);
            for (uint32_t ci = 0; !rc && ci < cn; ci++)
                if (cudaMemcpyAsync(BLO.at((size_t)ci * P->b1s2), BP.at(ci), 2 * pw1 * 8, cudaMemcpyDeviceToDevice,
                                    c->stream))
                    rc = blb_fail(BLB_ERR_CUDA, "copy failed");
            if (!rc)
                rc = rotate_hoisted(c, K, l1, srcs, rots, [&](uint32_t i, uint32_t j) {
                    const int32_t r = rots[j];
                    return r > 0 ? BLO.at((size_t)i * P->b1s2 + r) : BHI.at((size_t)i * P->b1s2 + (r + (int32_t)L));
                });
        }
        for (uint32_t ci = 0; !rc && ci < cn; ci++) {  // A at level l1, then its giant-step rotations
            k_drop<<<dim3((N + kT - 1) / kT, l1 + 1, 2), kT, 0, c->stream>>>(A1.at(ci), A[c0 + ci]->d, l0 + 1, l1 + 1,
                                                                             N);
            if (cudaGetLastError() != cudaSuccess) rc = blb_fail(BLB_ERR_CUDA, "drop launch failed");
            else blb_count_launch();
            if (!rc && cudaMemcpyAsync(AG.at((size_t)ci * P->G2), A1.at(ci), 2 * pw1 * 8, cudaMemcpyDeviceToDevice,
                                       c->stream))
                rc = blb_fail(BLB_ERR_CUDA, "copy failed");
        }
        if (!rc) {  // giant steps of A: Rot^{-g b1s2}(A_c), hoisted per A_c
            std::vector<const uint64_t*> srcs;
            std::vector<int32_t> rots;
            for (uint32_t ci = 0; ci < cn; ci++) srcs.push_back(A1.at(ci));
            for (uint32_t g = 1; g < P->G2; g++) rots.push_back(-(int32_t)(g * P->b1s2));
            rc = rotate_hoisted(c, K, l1, srcs, rots,
                                [&](uint32_t i, uint32_t j) { return AG.at((size_t)i * P->G2 + j + 1); });
        }
        for (uint32_t t0 = 0; !rc && t0 < L; t0 += Tc) {  // U[t] (+)= masked tensor sums of this chunk
            const uint32_t tn = std::min(Tc, L - t0);
            k_cc_step2<<<dim3(tn, (N + kS2 - 1) / kS2, l1 + 1), kS2, 0, c->stream>>>(
                U.at(t0), AG.d, BLO.d, BHI.d, d_mpairs, t0, cn, P->b1s2, P->G2, l1 + 1, N, c->d_q, c->d_bar, c0 > 0);
            if (cudaGetLastError() != cudaSuccess) rc = blb_fail(BLB_ERR_CUDA, "step-2 launch failed");
            else blb_count_launch();
        }
    }
    if (!rc) rc = rescale_many(c, U2.d, U.d, l1, L, 3);
    if (!rc) {  // relinearize: (d0, d1, d2) -> (d0 + k0, d1 + k1)
        items.clear();
        const uint64_t* rk = K->find(0)->d;
        for (uint32_t t = 0; t < L; t++) {
            const uint64_t* u = U2.at(t);
            uint64_t* o = WP.at(t);
            items.push_back(KsItem{u, u + 2 * pw2, u + pw2, rk, o, o + pw2, 1});
        }
        rc = keyswitch_batch(c, l2, items.data(), (uint32_t)items.size(), 0);
    }
    if (!rc) rc = rescale_many(c, W.d, WP.d, l2, L, 2);
    free_table(c, d_mpairs, bmp);

    // ---- step 3 ----
    Stack RT, CP;
    if (!rc) rc = RT.alloc(c, L, l3);
    if (!rc) rc = CP.alloc(c, P->nout, l3);
    items.clear();
    for (uint32_t t = 0; !rc && t < L; t++) {
        const int32_t r = step3_rot(P, t);
        if (r == 0) {
            if (cudaMemcpyAsync(RT.at(t), W.at(t), 2 * pw3 * 8, cudaMemcpyDeviceToDevice, c->stream))
                rc = blb_fail(BLB_ERR_CUDA, "copy failed");
            continue;
        }
        const uint64_t* k = key_for(K, N, r, &rc);
        if (k) items.push_back(KsItem{W.at(t), W.at(t) + pw3, nullptr, k, RT.at(t), RT.at(t) + pw3, galois_element(N, r)});
    }
    if (!rc) rc = keyswitch_batch(c, l3, items.data(), (uint32_t)items.size(), 0);
    if (!rc) {
        std::vector<uint32_t> start{0};
        std::vector<LcTerm> terms;
        for (uint32_t j = 0; j < P->nout; j++) {
            for (uint32_t t = 0; t < L; t++) {
                const int32_t m = P->m3_index[(size_t)t * P->nout + j];
                if (m >= 0) terms.push_back(LcTerm{RT.at(t), P->d_m3 + (size_t)m * pw3});
            }
            start.push_back((uint32_t)terms.size());
        }
        rc = lincomb(c, CP.d, P->nout, start, terms, l3);
    }
    const double out_scale = A[0]->scale * B[0]->scale / (double)c->q[l2];
    for (uint32_t j = 0; !rc && j < P->nout; j++) {
        blb_ct* y = nullptr;
        rc = new_ciphertext(c, l3 - 1, 2, out_scale, &y);
        if (!rc) rc = launch_rescale(c, y->d, CP.at(j), l3, 2);
        C[j] = y;
    }
    if (rc) {
        for (uint32_t j = 0; j < P->nout; j++) {
            blb_ct_free(C[j]);
            C[j] = nullptr;
        }
    }
    return rc;
}

extern "C" int blb_matmul_cc(blb_ctx* c, const blb_keys* K, blb_ct* const* A, blb_ct* const* B, uint32_t n_in,
                             uint32_t L, uint32_t R, uint32_t Hg, const blb_cc_sched* sched, blb_ct** C)
{
    if (!c || !A || n_in == 0 || !A[0]) return blb_fail(BLB_ERR_ARG, "null argument");
    blb_cc_plan* P = nullptr;
    BLB_TRY(blb_cc_plan_create(c, L, Hg, R, A[0]->level, sched, &P));
    int rc = blb_matmul_cc_plan(c, K, P, A, B, n_in, C);
    blb_cc_plan_free(P);
    return rc;
}
