// ctx.cu -- context creation: primes, NTT twiddles, base-conversion and encoding
// tables, allocator hooks, error strings.  Host code only.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"

typedef unsigned __int128 u128_t;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;
void blb_set_error(const std::string& msg) { g_err = msg; }
int blb_fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}
extern "C" const char* blb_last_error(void) { return g_err.c_str(); }
extern "C" const char* blb_version(void) { return "blb-b300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// launch counting and event timing of launch sites
// ---------------------------------------------------------------------------
static std::atomic<uint64_t> g_launches{0};
void blb_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
extern "C" uint64_t blb_kernel_launches(void) { return g_launches.load(); }

static cudaEvent_t pool_event(blb_ctx* c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfScope::ProfScope(blb_ctx* ctx, const char* name, uint64_t algorithmic_bytes) : c(ctx), site(-1)
{
    if (!c || !c->profiling || capturing(c)) return;  // a captured launch has no time of its own
    if (!c->prof_only.empty() && c->prof_only != name) return;
    for (size_t i = 0; i < c->prof.size(); i++)
        if (c->prof[i].name == name) site = (int)i;
    if (site < 0) {
        c->prof.push_back(blb_ctx::ProfSite{name, {}, 0, 0, 0, 0, 0, 0});
        site = (int)c->prof.size() - 1;
    }
    c->prof[site].bytes += algorithmic_bytes;
    b = pool_event(c);
    e = pool_event(c);
    cudaEventRecord(b, c->stream);
}
void ProfScope::ops(uint64_t mad128, uint64_t reductions, uint64_t butterflies)
{
    if (site < 0) return;
    c->prof[site].mad128 += mad128;
    c->prof[site].reductions += reductions;
    c->prof[site].butterflies += butterflies;
}
ProfScope::~ProfScope()
{
    if (site < 0) return;
    cudaEventRecord(e, c->stream);
    c->prof[site].ev.push_back({b, e});
}

static void prof_collect(blb_ctx* c)
{
    cudaStreamSynchronize(c->stream);
    for (auto& s : c->prof) {
        for (auto& p : s.ev) {
            float ms = 0;
            cudaEventElapsedTime(&ms, p.first, p.second);
            s.ms += ms;
            s.count++;
            c->event_pool.push_back(p.first);
            c->event_pool.push_back(p.second);
        }
        s.ev.clear();
    }
}

extern "C" int blb_profile_enable(blb_ctx* c, int on)
{
    if (!c) return blb_fail(BLB_ERR_ARG, "null context");
    prof_collect(c);
    c->prof.clear();
    c->profiling = on != 0;
    return BLB_OK;
}

extern "C" int blb_profile_select(blb_ctx* c, const char* site)
{
    if (!c) return blb_fail(BLB_ERR_ARG, "null context");
    c->prof_only = site ? site : "";
    return BLB_OK;
}

extern "C" int blb_profile_read(blb_ctx* c, const char* site, double* ms, uint64_t* count, uint64_t* bytes)
{
    if (!c || !site) return blb_fail(BLB_ERR_ARG, "null argument");
    prof_collect(c);
    if (ms) *ms = 0;
    if (count) *count = 0;
    if (bytes) *bytes = 0;
    for (auto& s : c->prof)
        if (s.name == site) {
            if (ms) *ms = s.ms;
            if (count) *count = s.count;
            if (bytes) *bytes = s.bytes;
        }
    return BLB_OK;
}

extern "C" int blb_profile_read_ops(blb_ctx* c, const char* site, uint64_t* mad128, uint64_t* reductions,
                                    uint64_t* butterflies)
{
    if (!c || !site) return blb_fail(BLB_ERR_ARG, "null argument");
    if (mad128) *mad128 = 0;
    if (reductions) *reductions = 0;
    if (butterflies) *butterflies = 0;
    for (auto& s : c->prof)
        if (s.name == site) {
            if (mad128) *mad128 = s.mad128;
            if (reductions) *reductions = s.reductions;
            if (butterflies) *butterflies = s.butterflies;
        }
    return BLB_OK;
}

// ---------------------------------------------------------------------------
// allocator
// ---------------------------------------------------------------------------
static std::mutex g_alloc_mu;
static blb_alloc_fn g_alloc = nullptr;
static blb_free_fn g_free = nullptr;
static void* g_alloc_user = nullptr;

extern "C" int blb_set_allocator(blb_alloc_fn alloc, blb_free_fn free_fn, void* user)
{
    if ((alloc == nullptr) != (free_fn == nullptr))
        return blb_fail(BLB_ERR_ARG, "blb_set_allocator: give both functions or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_user = user;
    return BLB_OK;
}

void* dev_alloc(blb_ctx* ctx, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    blb_alloc_fn a;
    void* u;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        u = g_alloc_user;
    }
    if (a) {
        p = a(bytes, (void*)ctx->stream, u);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) ctx->bytes_in_use += bytes;
    return p;
}

void dev_free(blb_ctx* ctx, void* p, size_t bytes)
{
    if (!p) return;
    if (bytes == 0) bytes = 256;
    blb_free_fn f;
    void* u;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        f = g_free;
        u = g_alloc_user;
    }
    if (f) f(p, bytes, (void*)ctx->stream, u);
    else cudaFree(p);
    ctx->bytes_in_use -= bytes;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// host number theory
// ---------------------------------------------------------------------------
uint64_t host_mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128_t)a * b) % q); }
uint64_t host_powmod(uint64_t b, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    b %= q;
    for (; e; e >>= 1) {
        if (e & 1) r = host_mulmod(r, b, q);
        b = host_mulmod(b, b, q);
    }
    return r;
}
uint64_t host_invmod(uint64_t a, uint64_t q) { return host_powmod(a % q, q - 2, q); }
uint64_t shoup_companion(uint64_t w, uint64_t q) { return (uint64_t)(((u128_t)w << 64) / q); }

// Strong-probable-prime test to the first 12 prime bases: exact below 3.3e24.
static bool is_prime_u64(uint64_t n)
{
    static const uint64_t B[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t b : B) {
        if (n == b) return true;
        if (n % b == 0) return false;
    }
    uint64_t d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        s++;
    }
    for (uint64_t b : B) {
        uint64_t x = host_powmod(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int r = 1; r < s && witness; r++) {
            x = host_mulmod(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// Left rotation by rot slots <-> X -> X^(5^rot mod 2N); 5 has order N/2.
uint64_t galois_element(uint32_t N, int32_t rot)
{
    int64_t h = N / 2;
    int64_t e = ((int64_t)rot % h + h) % h;
    return host_powmod(5, (uint64_t)e, 2ull * N);
}

static int select_primes(const blb_params* p, std::vector<uint64_t>& primes)
{
    if (!p) return blb_fail(BLB_ERR_ARG, "null parameters");
    if (p->logN < 10 || p->logN > 17) return blb_fail(BLB_ERR_ARG, "logN must be in [10, 17]");
    if (p->nQ < 1 || p->nP < 1 || p->nQ + p->nP > BLB_MAXP)
        return blb_fail(BLB_ERR_ARG, "need 1 <= nQ, 1 <= nP, nQ + nP <= 32");
    if (!p->q_bits || !p->p_bits) return blb_fail(BLB_ERR_ARG, "null bit-size array");
    if (p->dnum < 1 || p->dnum > p->nQ) return blb_fail(BLB_ERR_ARG, "dnum must be in [1, nQ]");
    uint32_t alpha = (p->nQ + p->dnum - 1) / p->dnum;
    if (p->nP < alpha) return blb_fail(BLB_ERR_ARG, "nP must be >= ceil(nQ/dnum)");
    const uint64_t m = 2ull << p->logN;
    primes.clear();
    for (uint32_t i = 0; i < p->nQ + p->nP; i++) {
        uint32_t bits = i < p->nQ ? p->q_bits[i] : p->p_bits[i - p->nQ];
        if (bits < p->logN + 2 || bits > 61) return blb_fail(BLB_ERR_PARAM, "prime bit size out of [logN+2, 61]");
        uint64_t lim = (1ull << bits) - 1;
        uint64_t c = lim - ((lim - 1) % m);  // largest value < 2^bits congruent to 1 mod 2N
        for (;;) {
            if (c <= m) return blb_fail(BLB_ERR_PARAM, "no prime of the requested size");
            bool taken = false;
            for (uint64_t x : primes) taken |= (x == c);
            if (!taken && is_prime_u64(c)) break;
            c -= m;
        }
        primes.push_back(c);
    }
    return BLB_OK;
}

extern "C" int blb_params_primes(const blb_params* params, uint64_t* out)
{
    if (!out) return blb_fail(BLB_ERR_ARG, "null output");
    std::vector<uint64_t> pr;
    BLB_TRY(select_primes(params, pr));
    memcpy(out, pr.data(), pr.size() * 8);
    return BLB_OK;
}

// psi: the first x = 2, 3, ... with x^((q-1)/2N) of order exactly 2N.
static uint64_t find_psi(uint64_t q, uint32_t N)
{
    for (uint64_t x = 2;; x++) {
        uint64_t w = host_powmod(x, (q - 1) / (2ull * N), q);
        if (host_powmod(w, N, q) == q - 1) return w;
    }
}

static uint32_t brv(uint32_t x, uint32_t bits)
{
    uint32_t r = 0;
    for (uint32_t i = 0; i < bits; i++) r = (r << 1) | ((x >> i) & 1);
    return r;
}

LimbMap blb_ctx::qmap(uint32_t nlimbs, uint32_t first) const
{
    LimbMap m{};
    for (uint32_t i = 0; i < nlimbs; i++) m.p[i] = (uint8_t)(first + i);
    m.n = nlimbs;
    return m;
}
LimbMap blb_ctx::extmap(uint32_t level) const
{
    LimbMap m{};
    uint32_t n = level + 1;
    for (uint32_t i = 0; i < n; i++) m.p[i] = (uint8_t)i;
    for (uint32_t k = 0; k < nP; k++) m.p[n + k] = (uint8_t)(nQ + k);
    m.n = n + nP;
    return m;
}
LimbMap blb_ctx::pmap() const { return qmap(nP, nQ); }

size_t blb_ctx::ks_words() const
{
    // coefficients n + extended digits beta*E + accumulators 2E + ModDown 2n rows
    size_t E = nQ + nP;
    return ((size_t)nQ + (size_t)dnum * E + 2 * E + 2 * (size_t)nQ) * N;
}

template <class T>
static int upload(blb_ctx* ctx, T** dptr, const T* host, size_t count)
{
    *dptr = (T*)dev_alloc(ctx, count * sizeof(T));
    if (!*dptr) return blb_fail(BLB_ERR_OOM, "table allocation failed");
    BLB_CUDA(cudaMemcpyAsync(*dptr, host, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return BLB_OK;
}

static void build_conv(const blb_ctx* c, const std::vector<uint32_t>& src, const std::vector<uint32_t>& dst,
                       const std::vector<uint32_t>& dst_row, ConvTable& t)
{
    memset(&t, 0, sizeof(t));
    t.ns = (uint32_t)src.size();
    t.nt = (uint32_t)dst.size();
    for (uint32_t i = 0; i < t.ns; i++) t.src[i] = (uint8_t)src[i];
    for (uint32_t k = 0; k < t.nt; k++) {
        t.dst[k] = (uint8_t)dst[k];
        t.dst_row[k] = (uint8_t)dst_row[k];
    }
    for (uint32_t i = 0; i < t.ns; i++) {
        uint64_t si = c->q[src[i]];
        uint64_t h = 1 % si;
        for (uint32_t k = 0; k < t.ns; k++)
            if (k != i) h = host_mulmod(h, c->q[src[k]] % si, si);
        t.hat_inv[i] = host_invmod(h, si);
        t.hat_inv_sh[i] = shoup_companion(t.hat_inv[i], si);
        for (uint32_t k = 0; k < t.nt; k++) {
            uint64_t tq = c->q[dst[k]];
            uint64_t v = 1 % tq;
            for (uint32_t l = 0; l < t.ns; l++)
                if (l != i) v = host_mulmod(v, c->q[src[l]] % tq, tq);
            t.hat[i][k] = v;
        }
    }
    for (uint32_t k = 0; k < t.nt; k++) {
        uint64_t tq = c->q[dst[k]], v = 1 % tq;
        for (uint32_t l = 0; l < t.ns; l++) v = host_mulmod(v, c->q[src[l]] % tq, tq);
        t.prod_mod_t[k] = v;
        t.neg_prod_mod_t[k] = (tq - v) % tq;
    }
}

extern "C" int blb_ctx_create(const blb_params* params, void* stream, blb_ctx** out)
{
    if (!out) return blb_fail(BLB_ERR_ARG, "null output");
    *out = nullptr;
    std::vector<uint64_t> primes;
    BLB_TRY(select_primes(params, primes));
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return blb_fail(BLB_ERR_CUDA, "no CUDA device");
    }
    blb_ctx* c = new blb_ctx();
    c->logN = params->logN;
    c->N = 1u << params->logN;
    c->nQ = params->nQ;
    c->nP = params->nP;
    c->dnum = params->dnum;
    c->alpha = (c->nQ + c->dnum - 1) / c->dnum;
    c->np = c->nQ + c->nP;
    c->scale = params->scale;
    c->stream = (cudaStream_t)stream;
    c->q = primes;
    const uint32_t N = c->N, np = c->np;
    auto fail = [&](int rc) {
        std::string msg = blb_last_error();
        blb_ctx_free(c);
        blb_set_error(msg);
        return rc;
    };

    // NTT tables
    std::vector<uint64_t> tw((size_t)np * 4 * N), bar(np * 2), ninv(np * 2);
    c->psi.resize(np);
    for (uint32_t i = 0; i < np; i++) {
        uint64_t q = c->q[i];
        uint64_t psi = find_psi(q, N), psi_inv = host_invmod(psi, q);
        c->psi[i] = psi;
        // [forward, inverse][k] pairs (psi^brv, Shoup companion): successive
        // powers of psi (psi^-1) placed at bit-reversed positions k
        uint64_t* T = &tw[(size_t)i * 4 * N];
        uint64_t pw = 1, pwi = 1;
        for (uint32_t e = 0; e < N; e++) {
            uint32_t k = brv(e, c->logN);
            T[2 * k] = pw;
            T[2 * k + 1] = shoup_companion(pw, q);
            T[2 * N + 2 * k] = pwi;
            T[2 * N + 2 * k + 1] = shoup_companion(pwi, q);
            pw = host_mulmod(pw, psi, q);
            pwi = host_mulmod(pwi, psi_inv, q);
        }
        u128_t R = (~(u128_t)0) / q;  // == floor(2^128 / q) for odd q
        bar[2 * i] = (uint64_t)R;
        bar[2 * i + 1] = (uint64_t)(R >> 64);
        ninv[2 * i] = host_invmod(N, q);
        ninv[2 * i + 1] = shoup_companion(ninv[2 * i], q);
    }
    int rc;
    if ((rc = upload(c, &c->d_q, c->q.data(), np))) return fail(rc);
    if ((rc = upload(c, &c->d_bar, bar.data(), bar.size()))) return fail(rc);
    if ((rc = upload(c, &c->d_tw, tw.data(), tw.size()))) return fail(rc);
    if ((rc = upload(c, &c->d_ninv, ninv.data(), ninv.size()))) return fail(rc);

    // encoding: zeta^k = (cos, sin)(pi k / N), k < N
    std::vector<double2> zeta(N);
    for (uint32_t k = 0; k < N; k++) {
        double ang = M_PI * (double)k / (double)N;
        zeta[k] = make_double2(cos(ang), sin(ang));
    }
    if ((rc = upload(c, &c->d_zeta, zeta.data(), N))) return fail(rc);

    // slot permutation of the canonical embedding and a status word
    {
        const uint32_t s = N / 2;
        std::vector<uint32_t> kp(s);
        uint64_t g = 1;
        for (uint32_t j = 0; j < s; j++) {
            kp[j] = (uint32_t)((g - 1) / 4);
            g = (g * 5) % (2ull * N);
        }
        if ((rc = upload(c, &c->d_kperm, kp.data(), s))) return fail(rc);
        int zero = 0;
        if ((rc = upload(c, &c->d_flag, &zero, 1))) return fail(rc);
        if ((rc = upload(c, &c->d_flag_deferred, &zero, 1))) return fail(rc);
        uint32_t uzero = 0;
        if ((rc = upload(c, &c->d_status, &uzero, 1))) return fail(rc);
    }
    if ((rc = keyswitch_noalloc_prepare(c))) return fail(rc);

    // discrete Gaussian table: floor(2^64 P(|e| <= k)), sigma 3.2, |e| <= 19
    {
        const double sigma = 3.2;
        double part[20];
        double z = 1.0;
        part[0] = z;
        for (int x = 1; x <= 19; x++) {
            z += 2.0 * exp(-(double)(x * x) / (2.0 * sigma * sigma));
            part[x] = z;
        }
        uint64_t cdt[19];
        for (int k = 0; k < 19; k++) {
            double cdf = part[k] / z;
            cdt[k] = cdf < 1.0 ? (uint64_t)ldexp(cdf, 64) : UINT64_MAX;
        }
        if ((rc = upload(c, &c->d_cdt, cdt, 19))) return fail(rc);
    }

    // RNS constants
    c->P_mod_q.resize(c->nQ);
    c->P_inv_mod_q.resize(c->nQ);
    for (uint32_t i = 0; i < c->nQ; i++) {
        uint64_t v = 1 % c->q[i];
        for (uint32_t k = 0; k < c->nP; k++) v = host_mulmod(v, c->q[c->nQ + k] % c->q[i], c->q[i]);
        c->P_mod_q[i] = v;
        c->P_inv_mod_q[i] = host_invmod(v, c->q[i]);
    }
    c->ql_inv.assign(c->nQ, std::vector<uint64_t>(c->nQ, 0));
    for (uint32_t l = 1; l < c->nQ; l++)
        for (uint32_t i = 0; i < l; i++) c->ql_inv[l][i] = host_invmod(c->q[l] % c->q[i], c->q[i]);

    // ModUp tables per (level, digit): sources D_j, targets Q_l u P minus D_j,
    // output rows in the extended basis order (q_0..q_l, p_0..)
    c->h_modup.assign((size_t)c->nQ * c->dnum, ConvTable{});
    c->d_modup.assign((size_t)c->nQ * c->dnum, nullptr);
    for (uint32_t l = 0; l < c->nQ; l++) {
        uint32_t n = l + 1, beta = (n + c->alpha - 1) / c->alpha;
        for (uint32_t j = 0; j < beta; j++) {
            uint32_t lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, n);
            std::vector<uint32_t> src, dst, row;
            for (uint32_t i = lo; i < hi; i++) src.push_back(i);
            for (uint32_t t = 0; t < n; t++)
                if (t < lo || t >= hi) {
                    dst.push_back(t);
                    row.push_back(t);
                }
            for (uint32_t k = 0; k < c->nP; k++) {
                dst.push_back(c->nQ + k);
                row.push_back(n + k);
            }
            build_conv(c, src, dst, row, c->h_modup[(size_t)l * c->dnum + j]);
        }
    }
    // one contiguous device array [level][digit]
    if ((rc = upload(c, &c->d_modup_all, c->h_modup.data(), c->h_modup.size()))) return fail(rc);
    for (size_t i = 0; i < c->h_modup.size(); i++) c->d_modup[i] = c->d_modup_all + i;
    {
        std::vector<uint32_t> src, dst, row;
        for (uint32_t k = 0; k < c->nP; k++) src.push_back(c->nQ + k);
        for (uint32_t i = 0; i < c->nQ; i++) {
            dst.push_back(i);
            row.push_back(i);
        }
        build_conv(c, src, dst, row, c->h_moddown);
        if ((rc = upload(c, &c->d_moddown, &c->h_moddown, 1))) return fail(rc);
    }
    {
        std::vector<uint64_t> nc((size_t)c->nQ * np * 2);
        for (uint32_t l = 0; l < c->nQ; l++)
            for (uint32_t pi = 0; pi < np; pi++) {
                const uint64_t q = c->q[pi], ni = host_invmod(N, q);
                uint64_t f = 1;
                if (pi >= c->nQ) f = c->h_moddown.hat_inv[pi - c->nQ];
                else if (pi <= l) f = c->h_modup[(size_t)l * c->dnum + pi / c->alpha].hat_inv[pi % c->alpha];
                const uint64_t w = host_mulmod(ni, f, q);
                nc[((size_t)l * np + pi) * 2] = w;
                nc[((size_t)l * np + pi) * 2 + 1] = shoup_companion(w, q);
            }
        if ((rc = upload(c, &c->d_ninv_conv, nc.data(), nc.size()))) return fail(rc);
    }
    {  // the rescale's q_l^-1 mod q_i with Shoup companions, [l][i][2]
        std::vector<uint64_t> qi((size_t)c->nQ * c->nQ * 2, 0);
        for (uint32_t l = 1; l < c->nQ; l++)
            for (uint32_t i = 0; i < l; i++) {
                qi[((size_t)l * c->nQ + i) * 2] = c->ql_inv[l][i];
                qi[((size_t)l * c->nQ + i) * 2 + 1] = shoup_companion(c->ql_inv[l][i], c->q[i]);
            }
        if ((rc = upload(c, &c->d_ql_inv, qi.data(), qi.size()))) return fail(rc);
    }

    // scratch arena: key-switch region + operation temporaries
    {
        size_t op_rows = 6 * (size_t)c->nQ + 2 * np + 4;
        size_t words = c->ks_words() + op_rows * N;
        c->scratch = (uint64_t*)dev_alloc(c, words * 8);
        if (!c->scratch) {
            blb_fail(BLB_ERR_OOM, "scratch arena allocation failed");
            return fail(BLB_ERR_OOM);
        }
        c->scratch_words = words;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        blb_fail(BLB_ERR_CUDA, "context table upload failed");
        return fail(BLB_ERR_CUDA);
    }
    *out = c;
    return BLB_OK;
}

static void ctx_destroy(blb_ctx* c);

void ctx_retain(blb_ctx* c) { c->live_objects++; }

void ctx_release(blb_ctx* c)
{
    if (--c->live_objects == 0 && c->closing) ctx_destroy(c);
}

// A context freed while objects created from it are alive (the order in which
// a garbage collector finalizes handles is arbitrary) is destroyed when the
// last of those objects is freed.
extern "C" void blb_ctx_free(blb_ctx* c)
{
    if (!c || c->closing) return;
    c->closing = true;
    if (c->live_objects == 0) ctx_destroy(c);
}

static void ctx_destroy(blb_ctx* c)
{
    prof_collect(c);
    for (auto e : c->event_pool) cudaEventDestroy(e);
    cudaStreamSynchronize(c->stream);
    dev_free(c, c->d_q, c->np * 8);
    dev_free(c, c->d_bar, c->np * 16);
    dev_free(c, c->d_tw, (size_t)c->np * 4 * c->N * 8);
    dev_free(c, c->d_ninv, c->np * 16);
    dev_free(c, c->d_ninv_conv, (size_t)c->nQ * c->np * 16);
    dev_free(c, c->d_ql_inv, (size_t)c->nQ * c->nQ * 16);
    dev_free(c, c->d_zeta, (size_t)c->N * sizeof(double2));
    dev_free(c, c->d_cdt, 19 * 8);
    dev_free(c, c->d_kperm, (size_t)c->N / 2 * 4);
    dev_free(c, c->d_flag, sizeof(int));
    dev_free(c, c->d_flag_deferred, sizeof(int));
    dev_free(c, c->d_status, sizeof(uint32_t));
    for (auto& k : c->graph_keep) {
        if (k.second) dev_free(c, k.first, k.second);
        else cudaFree(k.first);
    }
    if (c->upload_stream) cudaStreamDestroy(c->upload_stream);
    dev_free(c, c->d_fx_root, (size_t)c->N * sizeof(int2));
    dev_free(c, c->d_kinv, (size_t)c->N / 2 * 4);
    for (auto& t : c->fx_twist) dev_free(c, t.d, (size_t)c->N / 2 * sizeof(int2));
    dev_free(c, c->d_modup_all, c->h_modup.size() * sizeof(ConvTable));
    dev_free(c, c->d_moddown, sizeof(ConvTable));
    dev_free(c, c->scratch, c->scratch_words * 8);
    dev_free(c, c->batch, c->batch_words * 8);
    delete c;
}

extern "C" int blb_ctx_info(const blb_ctx* c, uint32_t* logN, uint32_t* nQ, uint32_t* nP, uint32_t* dnum)
{
    if (!c) return blb_fail(BLB_ERR_ARG, "null context");
    if (logN) *logN = c->logN;
    if (nQ) *nQ = c->nQ;
    if (nP) *nP = c->nP;
    if (dnum) *dnum = c->dnum;
    return BLB_OK;
}

extern "C" int blb_ctx_primes(const blb_ctx* c, uint64_t* out)
{
    if (!c || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    memcpy(out, c->q.data(), c->np * 8);
    return BLB_OK;
}

extern "C" int blb_ctx_sync(blb_ctx* c)
{
    if (!c) return blb_fail(BLB_ERR_ARG, "null context");
    BLB_CUDA(cudaStreamSynchronize(c->stream));
    uint32_t st = 0;
    BLB_CUDA(cudaMemcpy(&st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st) {
        BLB_CUDA(cudaMemset(c->d_status, 0, sizeof(st)));
        return blb_fail(BLB_ERR_TIMEOUT, "a bounded device wait expired (plaintext product pipeline)");
    }
    int ov = 0;
    BLB_CUDA(cudaMemcpy(&ov, c->d_flag_deferred, sizeof(ov), cudaMemcpyDeviceToHost));
    if (ov) {
        BLB_CUDA(cudaMemset(c->d_flag_deferred, 0, sizeof(ov)));
        return blb_fail(BLB_ERR_ARG, "an encoding with deferred checks overflowed: value * scale too large");
    }
    return BLB_OK;
}

extern "C" int blb_ctx_set_deferred_encode_check(blb_ctx* c, int on)
{
    if (!c) return blb_fail(BLB_ERR_ARG, "null context");
    c->encode_deferred = on != 0;
    return BLB_OK;
}

extern "C" uint64_t blb_ctx_bytes_in_use(const blb_ctx* c) { return c ? c->bytes_in_use : 0; }

extern "C" int blb_ctx_set_wait_limit(blb_ctx* c, uint64_t limit_ns)
{
    if (!c) return blb_fail(BLB_ERR_ARG, "null context");
    c->wait_ns = limit_ns;
    return BLB_OK;
}

extern "C" int blb_ctx_set_batch_mac(blb_ctx* c, int kind)
{
    if (!c || kind < 0 || kind > 2) return blb_fail(BLB_ERR_ARG, "kind must be 0, 1 or 2");
    c->batch_mac = kind;
    return BLB_OK;
}

extern "C" int blb_ctx_test_withhold_copies(blb_ctx* c, int withhold)
{
    if (!c) return blb_fail(BLB_ERR_ARG, "null context");
    c->mac_withhold = withhold ? 1u : 0u;
    return BLB_OK;
}
