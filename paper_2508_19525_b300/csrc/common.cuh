// common.cuh -- shared definitions of the B300 RNS-CKKS library (device
// arithmetic, context / object layouts, launcher declarations).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/blb.h"

#define BLB_MAXP 32

// ---------------------------------------------------------------------------
// error plumbing: every entry point returns a code; the message is kept per
// thread.
// ---------------------------------------------------------------------------
void blb_set_error(const std::string& msg);
int blb_fail(int code, const std::string& msg);
#define BLB_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return blb_fail(BLB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define BLB_TRY(expr)                  \
    do {                               \
        int rc_ = (expr);              \
        if (rc_ != BLB_OK) return rc_; \
    } while (0)
// launch check: catches configuration errors without synchronizing; counts
// the library's kernel launches
void blb_count_launch();
#define BLB_LAUNCHED()            \
    do {                          \
        blb_count_launch();       \
        BLB_CUDA(cudaGetLastError()); \
    } while (0)

// ---------------------------------------------------------------------------
// device modular arithmetic (all primes < 2^62)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q)
{
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q)
{
    return a >= b ? a - b : a + q - b;
}
__device__ __forceinline__ uint64_t neg_mod(uint64_t a, uint64_t q) { return a ? q - a : 0; }

// x * w mod q for a constant w with companion wp = floor(w 2^64 / q) (Shoup).
// Valid for any 64-bit x; result in [0, q).
__device__ __forceinline__ uint64_t mul_shoup(uint64_t x, uint64_t w, uint64_t wp, uint64_t q)
{
    uint64_t qt = __umul64hi(x, wp);
    uint64_t r = x * w - qt * q;
    return r >= q ? r - q : r;
}

// Barrett reduction of a 128-bit x = x1 2^64 + x0 with R = floor(2^128 / q)
// = r1 2^64 + r0.  x R / 2^128 = x1 r1 + (x1 r0 + x0 r1) / 2^64 + x0 r0 / 2^128;
// qhat keeps the whole first term and the integer parts of the second, so it
// misses at most 2 (three dropped fractions below 1 each) of floor(x R / 2^128),
// which is itself at least floor(x / q) - 1 and at most x / q.  Hence
// floor(x / q) - 3 <= qhat <= floor(x / q), r = x - qhat q lies in [0, 4q)
// (below 2^64 for q < 2^62, so it is exact mod 2^64), and two conditional
// subtractions land in [0, q).  Any x below 2^128.
__device__ __forceinline__ uint64_t barrett128(uint64_t x0, uint64_t x1, uint64_t q, uint64_t r0,
                                               uint64_t r1)
{
    const uint64_t qhat = x1 * r1 + __umul64hi(x1, r0) + __umul64hi(x0, r1);
    uint64_t r = x0 - qhat * q;
    const uint64_t q2 = q << 1;
    r = r >= q2 ? r - q2 : r;
    return r >= q ? r - q : r;
}

// x mod q for any 64-bit x, with rb = floor(2^64 / q) (the high word of the
// Barrett constant floor(2^128 / q)): floor(x rb / 2^64) is at least
// floor(x / q) - 1 and at most x / q, so one conditional subtraction lands in
// [0, q).  No division.
__device__ __forceinline__ uint64_t reduce64(uint64_t x, uint64_t q, uint64_t rb)
{
    const uint64_t r = x - __umul64hi(x, rb) * q;
    return r >= q ? r - q : r;
}
// a signed 64-bit v mod q, in [0, q)
__device__ __forceinline__ uint64_t signed_mod(int64_t v, uint64_t q, uint64_t rb)
{
    return v >= 0 ? reduce64((uint64_t)v, q, rb) : q - 1 - reduce64((uint64_t)(-(v + 1)), q, rb);
}

__device__ __forceinline__ uint64_t mul_mod(uint64_t a, uint64_t b, uint64_t q, uint64_t r0, uint64_t r1)
{
    return barrett128(a * b, __umul64hi(a, b), q, r0, r1);
}

// Programmatic dependent launch (launch_pdl below): a kernel launched this way
// may be scheduled while the previous kernel of its stream drains, so it must
// call pdl_begin before touching memory; pdl_begin also lets the next such
// kernel be scheduled early.  Both instructions are no-ops for kernels
// launched the ordinary way.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// 128-bit accumulator for lazy sums of products
struct acc128 {
    uint64_t lo, hi;
};
// acc += a b (mod 2^128): the low word with carry out, the high word with the
// carry in, as one multiply-add pair (the additions ride on the multiplies)
__device__ __forceinline__ void mad128(acc128& acc, uint64_t a, uint64_t b)
{
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(a), "l"(b));
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11); key = (seed lo, seed hi)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

enum { PURPOSE_SECRET = 1, PURPOSE_KEY_A = 2, PURPOSE_KEY_E = 3, PURPOSE_ENC_A = 4, PURPOSE_ENC_E = 5,
       PURPOSE_MASK = 6, PURPOSE_WRAP = 7 };

// one Philox draw with counter (coefficient i, sub-index j, object, purpose)
__device__ __forceinline__ uint4 philox_draw(uint64_t seed, uint32_t i, uint32_t j, uint32_t obj, uint32_t purpose)
{
    return philox4x32_10(make_uint4(i, j, obj, purpose), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// ---------------------------------------------------------------------------
// limb -> prime maps passed by value to kernels: row r of a polynomial stack uses
// prime p[r % n].
// ---------------------------------------------------------------------------
struct LimbMap {
    uint8_t p[BLB_MAXP];
    uint32_t n;
};

// Base-conversion constants for one (source set -> target set) conversion:
//   out_t = sum_i [x_i * hat_inv_i]_{s_i} * hat[i][t] mod t
struct ConvTable {
    uint32_t ns, nt;
    uint8_t src[BLB_MAXP];             // prime indices of the sources
    uint8_t dst[BLB_MAXP];             // prime indices of the targets
    uint8_t dst_row[BLB_MAXP];         // output row of each target
    uint64_t hat_inv[BLB_MAXP];        // (S/s_i)^-1 mod s_i
    uint64_t hat_inv_sh[BLB_MAXP];     // Shoup companions
    uint64_t hat[BLB_MAXP][BLB_MAXP];  // [i][t] = S/s_i mod t
    uint64_t prod_mod_t[BLB_MAXP];     // S mod t
    uint64_t neg_prod_mod_t[BLB_MAXP]; // (t - S mod t) mod t
};

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------
struct blb_ctx {
    uint32_t logN, N, nQ, nP, dnum, alpha, np;
    double scale;
    cudaStream_t stream;
    std::vector<uint64_t> q, psi;     // np primes, roots
    // device tables
    uint64_t* d_q = nullptr;          // [np]
    uint64_t* d_bar = nullptr;        // [np][2]: floor(2^128/q) lo, hi
    uint64_t* d_tw = nullptr;         // [np][2][N] pairs (w, shoup): psi^brv(k), then psi^-brv(k)
    uint64_t* d_ninv = nullptr;       // [np][2]: N^-1, shoup
    // [level][np][2]: N^-1 (S/s)^-1 mod s and its Shoup companion, where S is the
    // product of the conversion sources s belongs to at that level (its ModUp
    // digit for a ciphertext prime, P for a special prime): the inverse NTT
    // that feeds a base conversion applies the conversion's first factor
    uint64_t* d_ninv_conv = nullptr;
    uint64_t* d_ql_inv = nullptr;     // [l][i][2]: q_l^-1 mod q_i and its Shoup companion (i < l < nQ)
    double2* d_zeta = nullptr;        // [N]: (cos, sin)(pi k / N)
    uint64_t* d_cdt = nullptr;        // [19]
    uint32_t* d_kperm = nullptr;      // [N/2]: k_j = (5^j mod 2N - 1)/4
    int* d_flag = nullptr;            // device status word (encoding overflow)
    // deferred encoding checks: the overflow flag of every encoding accumulates
    // here and blb_ctx_sync reports it (no host wait per encoding)
    bool encode_deferred = false;
    int* d_flag_deferred = nullptr;
    uint32_t* d_status = nullptr;     // set by a kernel whose bounded wait expired
    uint64_t wait_ns = 0;             // limit of the bounded device waits (0: the 2 s default)
    uint32_t mac_withhold = 0;        // test hook: the plaintext streamer issues nothing (waits run out)
    int batch_mac = 0;                // MAC kernel of batches: 0 automatic, 1 mma.sync, 2 tcgen05
    uint64_t* noalloc_scratch = nullptr;  // device address of the allocation-free key switch's array
    // conversions between CKKS and shares (built on first use): fixed-point
    // roots zeta^k (k < N), the inverse slot permutation, and twist tables
    // round(2^30 c zeta^t) (t < N/2) for the last multipliers c used
    int2* d_fx_root = nullptr;
    uint32_t* d_kinv = nullptr;
    struct FxTwist {
        double mul;
        int2* d;
    };
    std::vector<FxTwist> fx_twist;
    // host-side constants
    std::vector<uint64_t> P_mod_q;              // [nQ]  P mod q_i
    std::vector<uint64_t> P_inv_mod_q;          // [nQ]  P^-1 mod q_i
    std::vector<std::vector<uint64_t>> ql_inv;  // [l][i] q_l^-1 mod q_i
    // conversion tables: ModUp per (level, digit), ModDown P -> Q
    std::vector<ConvTable> h_modup;             // index level * dnum + j
    std::vector<ConvTable*> d_modup;            // pointers into d_modup_all
    ConvTable* d_modup_all = nullptr;
    ConvTable h_moddown;
    ConvTable* d_moddown = nullptr;
    // optional CUDA-event timing of named launch sites (bench / profiling)
    bool profiling = false;
    struct ProfSite {
        std::string name;
        std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
        double ms = 0;
        uint64_t count = 0;
        uint64_t bytes = 0;  // algorithmic bytes of the bracketed calls
        // arithmetic of the bracketed calls, where the site counts it: 64 x 64
        // -> 128-bit multiply-adds, reductions of a 128-bit sum mod a prime,
        // NTT butterflies (and Shoup products by a constant)
        uint64_t mad128 = 0, reductions = 0, butterflies = 0;
    };
    std::vector<ProfSite> prof;
    std::string prof_only;  // when not empty, only this site is bracketed
    std::vector<cudaEvent_t> event_pool;
    // grow-only arena for batched key switching (stream-ordered reuse)
    uint64_t* batch = nullptr;
    size_t batch_words = 0;
    // scratch arena (stream-ordered reuse)
    uint64_t* scratch = nullptr;
    size_t scratch_words = 0;
    size_t bytes_in_use = 0;
    // CUDA-graph capture of the context's stream: tables uploaded during a
    // capture live in buffers of their own (graph_keep, freed with the
    // context), filled through a private non-blocking stream; once anything
    // was captured, a grown key-switch arena keeps the old one alive too
    cudaStream_t upload_stream = nullptr;
    std::vector<std::pair<void*, size_t>> graph_keep;  // (pointer, bytes); bytes 0 = cudaMalloc'd
    bool captured = false;
    int ntt_split = 0;  // split of the two-pass NTT around the middle (-1, 0, +1), see ntt.cu
    int ntt_radix = 8;  // largest radix of the NTT's register rounds (8 or 16), see ntt.cu
    // lifetime: objects (keys, plaintexts, ciphertexts, plans) hold the
    // context; blb_ctx_free releases it once the last of them is freed
    uint64_t live_objects = 0;
    bool closing = false;

    LimbMap qmap(uint32_t nlimbs, uint32_t first = 0) const;  // limbs -> q_first..
    LimbMap extmap(uint32_t level) const;                     // q_0..q_l, p_0..p_{nP-1}
    LimbMap pmap() const;                                     // p_0..p_{nP-1}
    // scratch regions (words): key switching uses [0, ks_words), operations
    // above it
    size_t ks_words() const;
    uint64_t* op_scratch() const { return scratch + ks_words(); }
};

struct blb_ct {
    blb_ctx* ctx;
    uint32_t level, npolys;
    double scale;
    uint64_t* d;   // npolys x (level+1) x N, NTT domain
    size_t bytes;
};

struct blb_pt {
    blb_ctx* ctx;
    uint32_t level;
    double scale;
    uint64_t* d;   // (level+1) x N, NTT domain
    size_t bytes;
};

struct KeyEntry {
    uint64_t galois;   // Galois element (0 = relinearization)
    uint64_t* d;       // dnum x 2 x np x N, NTT domain (b then a)
};

struct blb_keys {
    blb_ctx* ctx;
    uint64_t seed;
    uint64_t* d_s;     // np x N, NTT domain
    int64_t* d_s_coef; // N signed coefficients
    std::vector<KeyEntry> keys;
    size_t bytes;
    const KeyEntry* find(uint64_t g) const
    {
        for (auto& k : keys)
            if (k.galois == g) return &k;
        return nullptr;
    }
};

struct blb_cp_plan {
    blb_ctx* ctx;
    uint32_t m, d, d_out, level, k, nX, nY, b1, G;
    uint32_t KT, NEB;           // 16-term tiles, 16-output blocks of the (e, g) x (c, b) contraction
    uint8_t* d_ptb;             // byte-sliced plaintext diagonals, NTT domain (layout in mac_tc.cu)
    std::vector<uint8_t> nb;    // bytes per word of each limb
    std::vector<uint64_t> off;  // byte offset of each limb's region in d_ptb
    size_t bytes;
};

bool capturing(blb_ctx* ctx);
int persist_upload(blb_ctx* ctx, const void* host, size_t bytes, void** dev);

// stream-ordered temporary device buffers of one call, freed at scope exit
struct Scratch {
    blb_ctx* c;
    std::vector<std::pair<void*, size_t>> bufs;
    explicit Scratch(blb_ctx* ctx) : c(ctx) {}
    void* get(size_t bytes);
    // a device copy of a host table; under stream capture it goes to a buffer
    // the context keeps, since a replay reads it after the host vector is gone
    template <typename T>
    T* upload(const std::vector<T>& v)
    {
        if (capturing(c)) {
            void* p = nullptr;
            return persist_upload(c, v.data(), v.size() * sizeof(T), &p) == BLB_OK ? (T*)p : nullptr;
        }
        T* d = (T*)get(v.size() * sizeof(T));
        if (d && !v.empty() &&
            cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return nullptr;
        return d;
    }
    ~Scratch();
};

// RAII timer around a launch site (no-op unless the context is profiling)
struct ProfScope {
    blb_ctx* c;
    int site;
    cudaEvent_t b = nullptr, e = nullptr;
    ProfScope(blb_ctx* ctx, const char* name, uint64_t algorithmic_bytes);
    ~ProfScope();
    void ops(uint64_t mad128, uint64_t reductions, uint64_t butterflies);
};

// ---------------------------------------------------------------------------
// memory / host helpers
// ---------------------------------------------------------------------------
void* dev_alloc(blb_ctx* ctx, size_t bytes);
void ctx_retain(blb_ctx* ctx);
void ctx_release(blb_ctx* ctx);
void dev_free(blb_ctx* ctx, void* p, size_t bytes);
bool is_device_ptr(const void* p);
// is the context's stream being captured into a CUDA graph?
bool capturing(blb_ctx* ctx);
// host data into a device buffer that outlives every replay of the graph being
// captured (freed with the context); synchronous
int persist_upload(blb_ctx* ctx, const void* host, size_t bytes, void** dev);

uint64_t host_mulmod(uint64_t a, uint64_t b, uint64_t q);
uint64_t host_powmod(uint64_t b, uint64_t e, uint64_t q);
uint64_t host_invmod(uint64_t a, uint64_t q);
uint64_t shoup_companion(uint64_t w, uint64_t q);
uint64_t galois_element(uint32_t N, int32_t rot);

// ---------------------------------------------------------------------------
// launchers (all on ctx->stream)
// ---------------------------------------------------------------------------
// NTT of `rows` rows of N words; row r uses prime map.p[r % map.n]
// The rescale's forward transform with its elementwise steps fused into it:
// rows are (polynomial p, prime i < level), row p level + i; the first pass
// reads the centered lift of the q_level limb of polynomial p (coefficient
// form, `last`) reduced mod q_i instead of the row, and the last pass writes
// (in_i - result) q_level^-1 mod q_i to row p level + i of `out` instead of
// the row (in: polynomial p of a stack of ciphertexts of ppc polynomials,
// `stride` words apart).  `data` holds the rows between the two passes.
struct RescaleIO {
    const uint64_t* last;
    const uint64_t* in;
    uint64_t* out;
    const uint64_t* inv;  // [i][2]: q_level^-1 mod q_i and its Shoup companion (device)
    size_t stride;
    uint32_t level, ppc;
};
int ntt_forward_rescale(blb_ctx* ctx, uint64_t* data, uint32_t rows, const RescaleIO& rs);
// A key-switch source: its c1 rows (evaluation domain) and the Galois element
// applied as they are read.
struct GatherSrc {
    const uint64_t* c1;
    uint64_t g;
};
// The key switch's gather fused into the inverse transform of its sources:
// rows are (source s, prime i < n), row s n + i; the first pass reads
// c1[i][perm(k, g)] of source s instead of the row and also writes that value
// to row i of the source's extended digit j = i / alpha
// (ext[((s beta + j) E + i) N + k], the digit's own rows in the evaluation
// domain).  `data` receives the rows in coefficient form.
struct GatherIO {
    const GatherSrc* srcs;  // device array, one per source
    uint64_t* ext;
    uint32_t n, E, beta, alpha;
};
int ntt_inverse_gather(blb_ctx* ctx, uint64_t* data, uint32_t rows, const GatherIO& ga, const uint64_t* ninv);

// Evaluation-domain position read for output position k under the Galois
// element g (the forward transform's output order is bit-reversed odd powers
// of psi: A[k] = a(psi^(2 bitrev(k) + 1))).
__device__ __forceinline__ uint32_t perm_index(uint32_t k, uint32_t logN, uint64_t g)
{
    if (g == 1) return k;
    const uint32_t N = 1u << logN;
    const uint64_t e = 2 * (uint64_t)(__brev(k) >> (32 - logN)) + 1;
    const uint32_t ge = (uint32_t)((g * e) & (2ull * N - 1));
    return __brev((ge - 1) >> 1) >> (32 - logN);
}
int ntt_forward(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map);
int ntt_inverse(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map);
// same on an explicit device row list: entry = row index | prime index << 24
int ntt_forward_list(blb_ctx* ctx, uint64_t* data, uint32_t rows, const uint32_t* d_rowlist);
int ntt_inverse_list(blb_ctx* ctx, uint64_t* data, uint32_t rows, const uint32_t* d_rowlist);
// inverse NTT whose last pass multiplies by ninv[2 pi] (Shoup companion at
// ninv[2 pi + 1]) instead of N^-1 mod q_pi
int ntt_inverse_scaled(blb_ctx* ctx, uint64_t* data, uint32_t rows, const LimbMap& map, const uint64_t* ninv);
int ntt_inverse_list_scaled(blb_ctx* ctx, uint64_t* data, uint32_t rows, const uint32_t* d_rowlist,
                            const uint64_t* ninv);

// element-wise (row r uses prime map.p[r % map.n]; operand b repeats every
// b_rows rows)
int launch_mul_rows(blb_ctx* ctx, uint64_t* out, const uint64_t* a, const uint64_t* b, uint32_t rows,
                    const LimbMap& map, uint32_t b_rows);
int launch_mac_rows(blb_ctx* ctx, uint64_t* acc, const uint64_t* a, const uint64_t* b, uint32_t rows,
                    const LimbMap& map, uint32_t b_rows);
int launch_add_rows(blb_ctx* ctx, uint64_t* out, const uint64_t* a, const uint64_t* b, uint32_t rows,
                    const LimbMap& map);
int launch_sub_rows(blb_ctx* ctx, uint64_t* out, const uint64_t* a, const uint64_t* b, uint32_t rows,
                    const LimbMap& map);
int launch_neg_rows(blb_ctx* ctx, uint64_t* out, const uint64_t* a, uint32_t rows, const LimbMap& map);
int launch_mul_const_rows(blb_ctx* ctx, uint64_t* out, const uint64_t* a, uint32_t rows, const LimbMap& map,
                          const uint64_t* consts_per_row_host);
int launch_automorph_ntt(blb_ctx* ctx, uint64_t* out, const uint64_t* in, uint32_t rows, uint64_t g);
int launch_signed_to_rows(blb_ctx* ctx, uint64_t* out, const int64_t* in, uint32_t rows, const LimbMap& map);
int launch_rescale(blb_ctx* ctx, uint64_t* out, const uint64_t* in, uint32_t level, uint32_t npolys);
int launch_rescale_strided(blb_ctx* ctx, uint64_t* out, const uint64_t* in, uint32_t level, uint32_t npolys,
                           uint32_t ppc, size_t stride);
int launch_rescale_stack(blb_ctx* ctx, uint64_t* out, const uint64_t* in, uint32_t level, uint32_t npolys);
// new ciphertext object (retains the context)
int new_ciphertext(blb_ctx* ctx, uint32_t level, uint32_t npolys, double scale, blb_ct** out);
int new_ct(blb_ctx* c, uint32_t level, uint32_t npolys, double scale, blb_ct** out);
uint64_t* op_row(blb_ctx* c, size_t r);                             // row r of the operation scratch
// a host table of the library into device memory on the stream; under stream
// capture through a buffer the context keeps (a replay copies it from there)
int host_upload(blb_ctx* c, void* dst, const void* src, size_t bytes);
// an error if the context's stream is being captured (for calls that read
// results back on the host, create cached tables or plans, or take caller host
// memory)
int refuse_capture(blb_ctx* c, const char* what);

// launch with programmatic stream serialization (the kernel calls pdl_begin first)
template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
// caller buffers: host or device; a host buffer is refused while the stream is
// being captured (a graph cannot keep reading or writing caller host memory)
int copy_in(blb_ctx* c, void* dst, const void* src, size_t bytes);  // host or device source
int copy_out(blb_ctx* c, void* dst, const void* src, size_t bytes); // host (synchronises) or device target
int launch_tensor(blb_ctx* ctx, uint64_t* out, const uint64_t* a, const uint64_t* b, uint32_t level);

// sampling: counter (coefficient, j, obj, purpose), key = seed
int launch_sample_ternary(blb_ctx* ctx, int64_t* out, uint64_t seed, uint32_t obj, uint32_t purpose, uint32_t j);
int launch_sample_gauss(blb_ctx* ctx, int64_t* out, uint64_t seed, uint32_t obj, uint32_t purpose, uint32_t j);
// rows of uniform residues: row r mod prime map.p[r % map.n], sub-index j_of_row[r]
int launch_sample_uniform(blb_ctx* ctx, uint64_t* out, uint32_t rows, const LimbMap& map, uint64_t seed,
                          uint32_t obj, uint32_t purpose, const uint32_t* j_of_row);

// key switching of d (NTT domain, level+1 rows) with key (dnum x 2 x np x N)
int keyswitch(blb_ctx* ctx, const uint64_t* d_ntt, uint32_t level, const uint64_t* key, uint64_t* out0,
              uint64_t* out1);

// Batched key switching with fused automorphism: for each item,
//   (k0, k1) = KeySwitch(sigma_g(c1), key)
//   out0 = [out0 +] sigma_g(c0) + k0          (c0 may be null)
//   out1 = [out1 +] sigma_g(add1) + k1        (add1 may be null)
// g = 1 means no automorphism.  All items are at `level`; accumulate != 0 adds
// into the outputs instead of overwriting them (items of one call must then
// have distinct outputs).
struct KsItem {
    const uint64_t* c0;
    const uint64_t* c1;
    const uint64_t* add1;
    const uint64_t* key;
    uint64_t* out0;
    uint64_t* out1;
    uint64_t g;
};
int keyswitch_batch(blb_ctx* ctx, uint32_t level, const KsItem* items, uint32_t count, int accumulate);
// resolves, with the context's device current, the device address of the
// allocation-free key switch's array and loads that entry point's kernels
// (called by blb_ctx_create, where allocating is allowed)
int keyswitch_noalloc_prepare(blb_ctx* ctx);

// General key-switching pass (keyswitch.cu): sources are ModUp'd once (after
// the automorphism g), products apply g to the extended digits and multiply by
// a key, groups sum their products, divide by P once and add their addends.
struct KsSource {
    const uint64_t* c1;
    uint64_t g;
};
struct KsProduct {
    uint32_t src;
    uint64_t g;
    const uint64_t* key;
};
struct KsAdd {
    const uint64_t* ptr;  // (level+1) x N, NTT domain, read through sigma_g
    uint64_t g;
    uint32_t poly;        // added to out0 (0) or out1 (1)
};
struct KsGroup {
    uint64_t* out0;
    uint64_t* out1;
    uint32_t prod0, prod1;  // products [prod0, prod1)
    uint32_t add0, add1;    // addends [add0, add1)
};
int ks_run(blb_ctx* ctx, uint32_t level, const KsSource* sources, uint32_t n_src, const KsProduct* prods,
           const KsGroup* groups, uint32_t n_groups, const KsAdd* adds, int accumulate);

// encoding (Eq. 2)
int encode_slots(blb_ctx* ctx, const double* d_z, uint32_t npts, uint32_t n, uint32_t level, double scale,
                 uint64_t* d_out /* npts x (level+1) x N, NTT domain */);
int decode_limb0(blb_ctx* ctx, const uint64_t* d_coef0, double scale, double* d_slots);
// matmul_cp plaintext diagonals for pts [first, first+count) of a plan (slot vectors)
int cp_build_diagonals(blb_ctx* ctx, const blb_cp_plan* plan, const double* d_W, uint32_t first, uint32_t count,
                       double* d_z, const int32_t* d_head = nullptr, const int32_t* d_delta = nullptr,
                       uint32_t Dh = 0);
int launch_cp_mac(blb_ctx* ctx, const blb_cp_plan* plan, const uint64_t* baby, uint64_t* T, uint32_t S);
// the batched MAC on tcgen05 (mac_umma.cu); *used = false when the plan's
// shape does not fit it
int launch_cp_mac_umma(blb_ctx* c, const blb_cp_plan* P, const uint64_t* baby, uint64_t* T, uint32_t S, bool* used);
int cp_plan_layout(blb_ctx* ctx, blb_cp_plan* plan);
int cp_plan_store_block(blb_ctx* ctx, blb_cp_plan* plan, const uint64_t* src, uint32_t eblk);
