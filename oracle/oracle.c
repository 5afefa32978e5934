/*
 * oracle.c -- plain CPU oracle of BLB's RNS-CKKS linear path.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Written for a reader checking it
 * against the paper by eye: one function per operation, steps in the order
 * the operation is defined, modular products as (__int128)a*b % q.
 *
 * Paper passages followed (arXiv 2508.19525):
 *   Sec. 2.1  notation: A_{N,q} = Z_q[X]/(X^N+1), centered Z_q
 *   Sec. 2.4  CKKS plaintext/ciphertext, rescale, HomAdd/HomMul, Rot_l / Rot_r
 *   Sec. 6.1  Eq. 2: Encode(m) = round(Delta * pi^-1(m)), Decode = pi(Delta^-1 m)
 *   Sec. 4.2.1 spatial-first packing; Sec. 5 matmul protocols (BOLT's ct-pt
 *             product is cited there, not restated; the reading implemented
 *             here is the standard diagonal method with baby-step giant-step,
 *             App. C.1)
 *   Sec. 6.3 / Alg. 1  secure CKKS-to-MPC masking with a uniform mask
 *   Sec. 4.2.1 rotate-and-sum sum / broadcast packing; the HE steps of the
 *             secure LayerNorm before rsqrt (Alg. LayerNorm lines 1-6)
 *   Alg. 1 steps 3-4, Alg. 2, App. C.3  the parties' local steps of the
 *             conversions: field to ring, ring to field, fixed-point decoding
 *             and encoding of shares with local truncations
 * Where the paper is silent (key switching, sampling, prime choice, rounding
 * modes) the readings are the ones listed in the design notes; each function
 * below states the one it implements.
 */
#include "oracle.h"

#define ORC_MAX_ROT 512  /* rotations per hoisted call in matmul_cc */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------- */
/* modular arithmetic                                                          */
/* ------------------------------------------------------------------------- */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) { uint64_t s = a + b; return s >= q ? s - q : s; }
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) { return a >= b ? a - b : a + q - b; }
static uint64_t negmod(uint64_t a, uint64_t q) { return a ? q - a : 0; }
static uint64_t powmod(uint64_t b, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}
/* q prime: a^(q-2) is the inverse (Fermat). */
static uint64_t invmod(uint64_t a, uint64_t q) { return powmod(a % q, q - 2, q); }
/* signed integer -> residue in [0, q) */
static uint64_t from_signed(int64_t v, uint64_t q)
{
    if (v >= 0) return (uint64_t)v % q;
    uint64_t r = (uint64_t)(-(v + 1)) % q; /* -(v+1) avoids overflow at INT64_MIN */
    return q - 1 - r;
}

/* Deterministic Miller-Rabin: the first twelve primes as bases decide every
 * n < 3.3e24, which covers all 64-bit n. */
int orc_is_prime(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int k = 1; k < r; k++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

static uint32_t bitrev(uint32_t x, uint32_t bits)
{
    uint32_t r = 0;
    for (uint32_t i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

/* ------------------------------------------------------------------------- */
/* parameters                                                                  */
/* ------------------------------------------------------------------------- */
/* Prime rule (the paper fixes only bit widths, Table 4 / Sec. 7.1): for each
 * requested bit size b, in the order q_0, q_1, ..., p_0, p_1, ..., take the
 * largest prime below 2^b that is 1 mod 2N and not already taken.
 * psi rule: the first x = 2, 3, ... whose power x^((q-1)/2N) has order exactly
 * 2N (i.e. its N-th power is -1); that power is psi. */
int orc_params_init(orc_params* p, uint32_t logN, uint32_t nQ, uint32_t nP,
                    const uint32_t* q_bits, const uint32_t* p_bits, uint32_t dnum)
{
    memset(p, 0, sizeof(*p));
    if (logN < 2 || logN > 17 || nQ < 1 || nP < 1 || nQ + nP > ORC_MAX_PRIMES || dnum < 1) return -1;
    p->logN = logN;
    p->N = 1u << logN;
    p->nQ = nQ;
    p->nP = nP;
    p->dnum = dnum;
    p->alpha = (nQ + dnum - 1) / dnum;
    const uint64_t twoN = 2ull * p->N;
    for (uint32_t i = 0; i < nQ + nP; i++) {
        uint32_t b = i < nQ ? q_bits[i] : p_bits[i - nQ];
        if (b < logN + 2 || b > 62) return -2;
        uint64_t top = (1ull << b) - 1;
        uint64_t c = top - (top - 1) % twoN; /* largest value <= 2^b - 1 that is 1 mod 2N */
        for (;;) {
            if (c <= twoN) return -3;
            int used = 0;
            for (uint32_t k = 0; k < i; k++) used |= (p->prime[k] == c);
            if (!used && orc_is_prime(c)) break;
            c -= twoN;
        }
        p->prime[i] = c;
        for (uint64_t x = 2;; x++) {
            uint64_t w = powmod(x, (c - 1) / twoN, c);
            if (powmod(w, p->N, c) == c - 1) { p->psi[i] = w; break; }
        }
    }
    return 0;
}

/* Rot_l^r is the automorphism X -> X^g with g = 5^r mod 2N; a right rotation
 * by r is a left rotation by -r, and 5 has order N/2 (Sec. 2.4). */
uint64_t orc_galois_elt(const orc_params* p, int32_t r)
{
    int64_t s = p->N / 2;
    int64_t e = ((int64_t)r % s + s) % s;
    return powmod(5, (uint64_t)e, 2ull * p->N);
}

/* ------------------------------------------------------------------------- */
/* NTT                                                                         */
/* ------------------------------------------------------------------------- */
/* Forward negacyclic NTT, Cooley-Tukey butterflies with the psi powers in
 * bit-reversed order, natural-order input, output A[k] = a(psi^(2 brv(k)+1)).
 * (The tests check this statement against the O(N^2) definition.) */
void orc_ntt(const orc_params* p, uint32_t pi, uint64_t* a)
{
    const uint32_t N = p->N, logN = p->logN;
    const uint64_t q = p->prime[pi], psi = p->psi[pi];
    for (uint32_t m = 1, t = N / 2; m < N; m <<= 1, t >>= 1) {
        for (uint32_t i = 0; i < m; i++) {
            uint64_t S = powmod(psi, bitrev(m + i, logN), q);
            for (uint32_t j = 2 * i * t; j < 2 * i * t + t; j++) {
                uint64_t U = a[j], V = mulmod(a[j + t], S, q);
                a[j] = addmod(U, V, q);
                a[j + t] = submod(U, V, q);
            }
        }
    }
}

/* Inverse of orc_ntt: Gentleman-Sande butterflies with psi^-1 powers, then
 * multiplication by N^-1. */
void orc_intt(const orc_params* p, uint32_t pi, uint64_t* a)
{
    const uint32_t N = p->N, logN = p->logN;
    const uint64_t q = p->prime[pi], psi_inv = invmod(p->psi[pi], q);
    for (uint32_t m = N, t = 1; m > 1; m >>= 1, t <<= 1) {
        uint32_t h = m / 2;
        for (uint32_t i = 0; i < h; i++) {
            uint64_t S = powmod(psi_inv, bitrev(h + i, logN), q);
            for (uint32_t j = 2 * i * t; j < 2 * i * t + t; j++) {
                uint64_t U = a[j], V = a[j + t];
                a[j] = addmod(U, V, q);
                a[j + t] = mulmod(submod(U, V, q), S, q);
            }
        }
    }
    uint64_t n_inv = invmod(N, q);
    for (uint32_t j = 0; j < N; j++) a[j] = mulmod(a[j], n_inv, q);
}

/* a*b in Z_q[X]/(X^N+1) via forward NTT, pointwise product, inverse NTT. */
void orc_negacyclic_mul(const orc_params* p, uint32_t pi, const uint64_t* a, const uint64_t* b,
                        uint64_t* out)
{
    const uint32_t N = p->N;
    const uint64_t q = p->prime[pi];
    uint64_t* A = malloc(sizeof(uint64_t) * N);
    uint64_t* B = malloc(sizeof(uint64_t) * N);
    memcpy(A, a, sizeof(uint64_t) * N);
    memcpy(B, b, sizeof(uint64_t) * N);
    orc_ntt(p, pi, A);
    orc_ntt(p, pi, B);
    for (uint32_t j = 0; j < N; j++) A[j] = mulmod(A[j], B[j], q);
    orc_intt(p, pi, A);
    memcpy(out, A, sizeof(uint64_t) * N);
    free(A);
    free(B);
}

/* ------------------------------------------------------------------------- */
/* sampling                                                                    */
/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * published multipliers and Weyl key increments. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One 128-bit draw for coefficient i: counter (i, j, obj, purpose), key = seed. */
static void draw(uint64_t seed, uint32_t i, uint32_t j, uint32_t obj, uint32_t purpose, uint32_t out[4])
{
    uint32_t ctr[4] = {i, j, obj, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

/* Cumulative table of |e| for the discrete Gaussian rho(x) = exp(-x^2/(2 sigma^2)),
 * sigma = 3.2 (the usual CKKS error width), support cut at |x| <= 19:
 * table[k] = floor(2^64 * P(|e| <= k)) for k = 0..18. */
void orc_cdt_table(uint64_t table[19])
{
    const double sigma = 3.2;
    double partial[20];
    double acc = 1.0; /* rho(0) */
    partial[0] = acc;
    for (int x = 1; x <= 19; x++) {
        acc += 2.0 * exp(-(double)(x * x) / (2.0 * sigma * sigma));
        partial[x] = acc;
    }
    for (int k = 0; k < 19; k++) {
        double cdf = partial[k] / acc;
        table[k] = cdf < 1.0 ? (uint64_t)ldexp(cdf, 64) : UINT64_MAX;
    }
}

/* Ternary secret: (u32 mod 3) - 1. */
void orc_sample_ternary(uint32_t N, uint64_t seed, uint32_t obj, uint32_t purpose, uint32_t j,
                        int64_t* out)
{
    for (uint32_t i = 0; i < N; i++) {
        uint32_t r[4];
        draw(seed, i, j, obj, purpose, r);
        out[i] = (int64_t)(r[0] % 3u) - 1;
    }
}

/* Discrete Gaussian by cumulative-table inversion: magnitude = number of table
 * entries <= the 64-bit draw (words 0,1), sign from bit 0 of word 2. */
void orc_sample_gauss(uint32_t N, uint64_t seed, uint32_t obj, uint32_t purpose, uint32_t j,
                      int64_t* out)
{
    uint64_t T[19];
    orc_cdt_table(T);
    for (uint32_t i = 0; i < N; i++) {
        uint32_t r[4];
        draw(seed, i, j, obj, purpose, r);
        uint64_t u = (uint64_t)r[0] | ((uint64_t)r[1] << 32);
        int64_t k = 0;
        for (int t = 0; t < 19; t++) k += (u >= T[t]);
        out[i] = (r[2] & 1u) ? -k : k;
    }
}

/* Uniform residue: the full 128-bit draw (word 3 most significant) mod q. */
void orc_sample_uniform(uint32_t N, uint64_t q, uint64_t seed, uint32_t obj, uint32_t purpose,
                        uint32_t j, uint64_t* out)
{
    for (uint32_t i = 0; i < N; i++) {
        uint32_t r[4];
        draw(seed, i, j, obj, purpose, r);
        u128 v = ((u128)r[3] << 96) | ((u128)r[2] << 64) | ((u128)r[1] << 32) | (u128)r[0];
        out[i] = (uint64_t)(v % q);
    }
}

/* ------------------------------------------------------------------------- */
/* encode / decode (Sec. 6.1, Eq. 2)                                           */
/* ------------------------------------------------------------------------- */
/* Slot j of a real polynomial m is m(zeta^(5^j)), zeta = exp(i pi / N), j < N/2
 * (real slots only, as in the footnote to Eq. 2).  With s = N/2 and
 * v_t = m_t + i m_{t+s}, slot j equals sum_t v_t zeta^(t 5^j), an s-point DFT
 * (root omega = zeta^4) of v_t zeta^t read at index k_j = (5^j - 1)/4.
 * Encode inverts it: V[k_j] = z_j, a = inverse DFT (no 1/s), c_t = a_t zeta^-t,
 * m_t = round(Re c_t * Delta/s), m_{t+s} = round(Im c_t * Delta/s), round half
 * to even.  The DFT is the iterative radix-2 decimation-in-time FFT on
 * bit-reversed input with the complex product (ac - bd, ad + bc) and
 * zeta^k = (cos(pi k/N), sin(pi k/N)) from the C library; no fused multiply-add
 * (this file is built with -ffp-contract=off). */
typedef struct { double re, im; } cplx;

static cplx cmul(cplx x, cplx w)
{
    double t1 = x.re * w.re, t2 = x.im * w.im, t3 = x.re * w.im, t4 = x.im * w.re;
    cplx r = {t1 - t2, t3 + t4};
    return r;
}

static cplx zeta_pow(uint32_t N, uint32_t k)
{
    double ang = M_PI * (double)k / (double)N;
    cplx r = {cos(ang), sin(ang)};
    return r;
}

/* In-place radix-2 DIT DFT of length s on A (already bit-reversed):
 * sign = -1 computes sum_k A[k] omega^(-k t), sign = +1 uses omega^(+k t). */
static void fft_dit(cplx* A, uint32_t s, uint32_t N, int sign)
{
    for (uint32_t len = 2; len <= s; len <<= 1) {
        uint32_t half = len / 2, step = s / len;
        for (uint32_t i = 0; i < s; i += len) {
            for (uint32_t j = 0; j < half; j++) {
                cplx w = zeta_pow(N, 4 * j * step);
                if (sign < 0) w.im = -w.im;
                cplx u = A[i + j];
                cplx v = cmul(A[i + j + half], w);
                A[i + j].re = u.re + v.re;
                A[i + j].im = u.im + v.im;
                A[i + j + half].re = u.re - v.re;
                A[i + j + half].im = u.im - v.im;
            }
        }
    }
}

int orc_encode_int(const orc_params* p, const double* z, uint32_t n, double scale, int64_t* out)
{
    const uint32_t N = p->N, s = N / 2, logs = p->logN - 1;
    if (n > s) return -1;
    cplx* V = calloc(s, sizeof(cplx));
    cplx* A = calloc(s, sizeof(cplx));
    uint64_t g = 1;
    for (uint32_t j = 0; j < s; j++) {
        uint32_t k = (uint32_t)((g - 1) / 4);
        V[k].re = j < n ? z[j] : 0.0;
        V[k].im = 0.0;
        g = (g * 5) % (2ull * N);
    }
    for (uint32_t k = 0; k < s; k++) A[bitrev(k, logs)] = V[k];
    fft_dit(A, s, N, -1);
    const double f = scale / (double)s;
    int rc = 0;
    for (uint32_t t = 0; t < s; t++) {
        cplx w = zeta_pow(N, t);
        w.im = -w.im;
        cplx c = cmul(A[t], w);
        double re = rint(c.re * f), im = rint(c.im * f);
        if (fabs(re) >= 9.2e18 || fabs(im) >= 9.2e18) rc = -2;
        out[t] = (int64_t)re;
        out[t + s] = (int64_t)im;
    }
    free(V);
    free(A);
    return rc;
}

int orc_encode(const orc_params* p, const double* z, uint32_t n, uint32_t level, double scale,
               uint64_t* out)
{
    const uint32_t N = p->N;
    int64_t* m = malloc(sizeof(int64_t) * N);
    int rc = orc_encode_int(p, z, n, scale, m);
    for (uint32_t i = 0; i <= level; i++)
        for (uint32_t t = 0; t < N; t++) out[(size_t)i * N + t] = from_signed(m[t], p->prime[i]);
    free(m);
    return rc;
}

/* Decode: z_j = (1/Delta) sum_t m_t zeta^(t 5^j) for signed coefficients m. */
void orc_decode(const orc_params* p, const int64_t* coef, double scale, double* z)
{
    const uint32_t N = p->N, s = N / 2, logs = p->logN - 1;
    cplx* A = calloc(s, sizeof(cplx));
    for (uint32_t t = 0; t < s; t++) {
        cplx v = {(double)coef[t], (double)coef[t + s]};
        A[bitrev(t, logs)] = cmul(v, zeta_pow(N, t));
    }
    fft_dit(A, s, N, +1);
    uint64_t g = 1;
    for (uint32_t j = 0; j < s; j++) {
        z[j] = A[(g - 1) / 4].re / scale;
        g = (g * 5) % (2ull * N);
    }
    free(A);
}

/* ------------------------------------------------------------------------- */
/* keys                                                                        */
/* ------------------------------------------------------------------------- */
uint64_t orc_ksk_words(const orc_params* p)
{
    return (uint64_t)p->dnum * 2 * (p->nQ + p->nP) * p->N;
}

void orc_keygen_secret(const orc_params* p, uint64_t seed, int64_t* s)
{
    orc_sample_ternary(p->N, seed, 0, ORC_SECRET, 0, s);
}

/* Hybrid key-switching key from s' to s (standard hybrid key switching; the
 * paper uses rotations and relinearization, Sec. 2.4, without restating them).
 * Digit j covers ciphertext primes D_j = {j*alpha, ..., min((j+1)*alpha, nQ)-1}.
 * For every prime t of Q u P:
 *   a_j[t] uniform (purpose KEY_A, sub-index 64*j + t),
 *   e_j    Gaussian, shared by all primes of the digit (purpose KEY_E, sub-index j),
 *   b_j[t] = -a_j[t]*s + e_j + [t in D_j] * (P mod q_t) * s'   (mod prime t).
 * The gadget factor P*(Q/Q_j)*[(Q/Q_j)^-1 mod Q_j] is P mod q_t on the digit's
 * own primes and 0 on every other prime, which is what the last term writes. */
void orc_keygen_ksk(const orc_params* p, uint64_t seed, const int64_t* s, const int64_t* s_prime,
                    uint32_t obj, uint64_t* ksk)
{
    const uint32_t N = p->N, L = p->nQ + p->nP;
    int64_t* e = malloc(sizeof(int64_t) * N);
    uint64_t* a = malloc(sizeof(uint64_t) * N);
    uint64_t* sq = malloc(sizeof(uint64_t) * N);
    uint64_t* as = malloc(sizeof(uint64_t) * N);
    for (uint32_t j = 0; j < p->dnum; j++) {
        orc_sample_gauss(N, seed, obj, ORC_KEY_E, j, e);
        for (uint32_t t = 0; t < L; t++) {
            const uint64_t q = p->prime[t];
            uint64_t* B = ksk + ((size_t)(j * 2 + 0) * L + t) * N;
            uint64_t* A = ksk + ((size_t)(j * 2 + 1) * L + t) * N;
            orc_sample_uniform(N, q, seed, obj, ORC_KEY_A, 64 * j + t, a);
            for (uint32_t i = 0; i < N; i++) sq[i] = from_signed(s[i], q);
            orc_negacyclic_mul(p, t, a, sq, as);
            int in_digit = t < p->nQ && t >= j * p->alpha && t < (j + 1) * p->alpha;
            uint64_t Pmod = 1 % q;
            for (uint32_t k = 0; k < p->nP; k++) Pmod = mulmod(Pmod, p->prime[p->nQ + k] % q, q);
            for (uint32_t i = 0; i < N; i++) {
                uint64_t v = addmod(negmod(as[i], q), from_signed(e[i], q), q);
                if (in_digit) v = addmod(v, mulmod(Pmod, from_signed(s_prime[i], q), q), q);
                B[i] = v;
                A[i] = a[i];
            }
        }
    }
    free(e); free(a); free(sq); free(as);
}

/* s^2 as a signed integer polynomial (coefficients are tiny for ternary s). */
static void square_secret(uint32_t N, const int64_t* s, int64_t* s2)
{
    for (uint32_t k = 0; k < N; k++) s2[k] = 0;
    for (uint32_t i = 0; i < N; i++) {
        if (!s[i]) continue;
        for (uint32_t j = 0; j < N; j++) {
            if (!s[j]) continue;
            uint32_t k = i + j;
            int64_t v = s[i] * s[j];
            if (k >= N) { k -= N; v = -v; }
            s2[k] += v;
        }
    }
}

void orc_keygen_relin(const orc_params* p, uint64_t seed, const int64_t* s, uint64_t* ksk)
{
    int64_t* s2 = malloc(sizeof(int64_t) * p->N);
    square_secret(p->N, s, s2);
    orc_keygen_ksk(p, seed, s, s2, 0, ksk);
    free(s2);
}

/* sigma_g on signed coefficients: X^i -> X^(i g mod 2N), negated past N. */
static void automorph_signed(uint32_t N, const int64_t* in, uint64_t g, int64_t* out)
{
    for (uint32_t i = 0; i < N; i++) {
        uint64_t k = ((uint64_t)i * g) % (2ull * N);
        if (k < N) out[k] = in[i];
        else out[k - N] = -in[i];
    }
}

void orc_keygen_galois(const orc_params* p, uint64_t seed, const int64_t* s, uint64_t g, uint64_t* ksk)
{
    int64_t* sg = malloc(sizeof(int64_t) * p->N);
    automorph_signed(p->N, s, g, sg);
    orc_keygen_ksk(p, seed, s, sg, (uint32_t)g, ksk);
    free(sg);
}

/* ------------------------------------------------------------------------- */
/* ciphertext operations                                                       */
/* ------------------------------------------------------------------------- */
/* Secret-key encryption c = (-a*s + m + e, a): a uniform per prime (ENC_A,
 * sub-index = prime index), e Gaussian shared by all primes (ENC_E), both keyed
 * by the caller's nonce. */
void orc_encrypt(const orc_params* p, const int64_t* s, const uint64_t* pt, uint32_t level,
                 uint64_t seed, uint32_t nonce, uint64_t* ct)
{
    const uint32_t N = p->N, n = level + 1;
    int64_t* e = malloc(sizeof(int64_t) * N);
    orc_sample_gauss(N, seed, nonce, ORC_ENC_E, 0, e);
    #pragma omp parallel for
    for (uint32_t i = 0; i < n; i++) {
        const uint64_t q = p->prime[i];
        uint64_t* a = malloc(sizeof(uint64_t) * N);
        uint64_t* sq = malloc(sizeof(uint64_t) * N);
        uint64_t* as = malloc(sizeof(uint64_t) * N);
        orc_sample_uniform(N, q, seed, nonce, ORC_ENC_A, i, a);
        for (uint32_t k = 0; k < N; k++) sq[k] = from_signed(s[k], q);
        orc_negacyclic_mul(p, i, a, sq, as);
        uint64_t* c0 = ct + (size_t)i * N;
        uint64_t* c1 = ct + ((size_t)n + i) * N;
        for (uint32_t k = 0; k < N; k++) {
            c0[k] = addmod(addmod(negmod(as[k], q), pt[(size_t)i * N + k], q), from_signed(e[k], q), q);
            c1[k] = a[k];
        }
        free(a); free(sq); free(as);
    }
    free(e);
}

/* m = sum_k c_k * s^k over the ciphertext's polynomials (2, or 3 before
 * relinearization). */
void orc_decrypt(const orc_params* p, const int64_t* s, const uint64_t* ct, uint32_t level,
                 uint32_t npolys, uint64_t* m)
{
    const uint32_t N = p->N, n = level + 1;
    #pragma omp parallel for
    for (uint32_t i = 0; i < n; i++) {
        const uint64_t q = p->prime[i];
        uint64_t* sp = malloc(sizeof(uint64_t) * N);
        uint64_t* tmp = malloc(sizeof(uint64_t) * N);
        for (uint32_t k = 0; k < N; k++) sp[k] = from_signed(s[k], q);
        /* Horner: ((c_{np-1}) s + c_{np-2}) s + ... + c_0 */
        uint64_t* h = malloc(sizeof(uint64_t) * N);
        memcpy(h, ct + ((size_t)(npolys - 1) * n + i) * N, sizeof(uint64_t) * N);
        for (int k = (int)npolys - 2; k >= 0; k--) {
            orc_negacyclic_mul(p, i, h, sp, tmp);
            const uint64_t* ck = ct + ((size_t)k * n + i) * N;
            for (uint32_t t = 0; t < N; t++) h[t] = addmod(tmp[t], ck[t], q);
        }
        memcpy(m + (size_t)i * N, h, sizeof(uint64_t) * N);
        free(sp); free(tmp); free(h);
    }
}

void orc_automorphism(const orc_params* p, const uint64_t* in, uint32_t nlimbs, uint64_t g, uint64_t* out)
{
    const uint32_t N = p->N;
    for (uint32_t l = 0; l < nlimbs; l++) {
        const uint64_t* a = in + (size_t)l * N;
        uint64_t* b = out + (size_t)l * N;
        for (uint32_t i = 0; i < N; i++) {
            uint64_t k = ((uint64_t)i * g) % (2ull * N);
            if (k < N) b[k] = a[i];
            else b[k - N] = negmod(a[i], p->prime[l]);
        }
    }
}

/* Fast base conversion (approximate, no overflow correction) from the primes
 * src[0..ns) to prime t, for every coefficient c:
 *   Conv(x)_t = sum_i [x_i * (S/s_i)^-1]_{s_i} * (S/s_i mod t)   mod t,
 * S = prod_i s_i.  x holds ns limbs of N residues, limb i mod src[i]. */
static void base_convert(uint32_t N, const uint64_t* const* x, const uint64_t* src, uint32_t ns,
                         uint64_t t, uint64_t* out)
{
    uint64_t hat_inv[ORC_MAX_PRIMES], hat_t[ORC_MAX_PRIMES];
    for (uint32_t i = 0; i < ns; i++) {
        uint64_t hat_mod_si = 1 % src[i], h_t = 1 % t;
        for (uint32_t k = 0; k < ns; k++) {
            if (k == i) continue;
            hat_mod_si = mulmod(hat_mod_si, src[k] % src[i], src[i]);
            h_t = mulmod(h_t, src[k] % t, t);
        }
        hat_inv[i] = invmod(hat_mod_si, src[i]);
        hat_t[i] = h_t;
    }
    for (uint32_t c = 0; c < N; c++) {
        uint64_t acc = 0;
        for (uint32_t i = 0; i < ns; i++) {
            uint64_t y = mulmod(x[i][c], hat_inv[i], src[i]);
            acc = addmod(acc, mulmod(y % t, hat_t[i], t), t);
        }
        out[c] = acc;
    }
}

/* Multi-word unsigned integers (little-endian 64-bit words), used only by the
 * exact CRT of ModDown below: P, a product of at most ORC_MP_WORDS - 1 primes
 * below 2^64, and sums of nP multiples of P/p_k fit with room to spare. */
#define ORC_MP_WORDS 8
typedef struct {
    uint64_t w[ORC_MP_WORDS];
} mpint;

static void mp_set(mpint* a, uint64_t v)
{
    memset(a, 0, sizeof *a);
    a->w[0] = v;
}
static void mp_mul_u64(mpint* a, uint64_t m)
{
    u128 carry = 0;
    for (int i = 0; i < ORC_MP_WORDS; i++) {
        u128 t = (u128)a->w[i] * m + carry;
        a->w[i] = (uint64_t)t;
        carry = t >> 64;
    }
}
static void mp_add(mpint* a, const mpint* b)
{
    uint64_t carry = 0;
    for (int i = 0; i < ORC_MP_WORDS; i++) {
        u128 t = (u128)a->w[i] + b->w[i] + carry;
        a->w[i] = (uint64_t)t;
        carry = (uint64_t)(t >> 64);
    }
}
static void mp_sub(mpint* a, const mpint* b) /* requires a >= b */
{
    uint64_t borrow = 0;
    for (int i = 0; i < ORC_MP_WORDS; i++) {
        uint64_t bi = b->w[i] + borrow;
        uint64_t nb = (bi < borrow) || (a->w[i] < bi);
        a->w[i] -= bi;
        borrow = nb;
    }
}
static int mp_cmp(const mpint* a, const mpint* b)
{
    for (int i = ORC_MP_WORDS - 1; i >= 0; i--)
        if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
    return 0;
}
static uint64_t mp_mod_u64(const mpint* a, uint64_t q)
{
    int top = ORC_MP_WORDS - 1;
    while (top > 0 && a->w[top] == 0) top--;
    u128 r = 0;
    for (int i = top; i >= 0; i--) r = ((r << 64) | a->w[i]) % q;
    return (uint64_t)r;
}

/* ModDown: divide a polynomial pair given over Q_l u P (coefficient form,
 * 2 x (n + nP) rows, Q rows first) by P with rounding:
 *   out_i = (x_i - X) * P^-1 mod q_i = round(x / P) mod q_i,
 * where X is the representative of x mod P in (-P/2, P/2] (P is odd, so no
 * value sits exactly between two integers).  X is computed exactly, by the
 * Chinese remainder theorem in multi-word integers:
 *   [x]_P = sum_k [x_k (P/p_k)^-1]_{p_k} (P/p_k)  reduced into [0, P),
 * minus P when twice it exceeds P. */
void orc_moddown(const orc_params* p, const uint64_t* acc, uint32_t level, uint64_t* out)
{
    const uint32_t N = p->N, n = level + 1, nP = p->nP, ext = n + nP;
    const uint64_t* pp = p->prime + p->nQ;
    if (nP >= ORC_MP_WORDS) abort(); /* P would not fit the multi-word integers */
    mpint P, hat[ORC_MAX_PRIMES];
    uint64_t hat_inv[ORC_MAX_PRIMES], P_q[ORC_MAX_PRIMES], Pinv[ORC_MAX_PRIMES];
    mp_set(&P, 1);
    for (uint32_t k = 0; k < nP; k++) mp_mul_u64(&P, pp[k]);
    for (uint32_t k = 0; k < nP; k++) {
        mp_set(&hat[k], 1);
        for (uint32_t l = 0; l < nP; l++)
            if (l != k) mp_mul_u64(&hat[k], pp[l]);
        hat_inv[k] = invmod(mp_mod_u64(&hat[k], pp[k]), pp[k]);
    }
    for (uint32_t i = 0; i < n; i++) {
        P_q[i] = mp_mod_u64(&P, p->prime[i]);
        Pinv[i] = invmod(P_q[i], p->prime[i]);
    }
    for (uint32_t poly = 0; poly < 2; poly++) {
        const uint64_t* A = acc + (size_t)poly * ext * N;
        #pragma omp parallel for
        for (uint32_t c = 0; c < N; c++) {
            mpint X, t;
            mp_set(&X, 0);
            for (uint32_t k = 0; k < nP; k++) {
                t = hat[k];
                mp_mul_u64(&t, mulmod(A[(size_t)(n + k) * N + c], hat_inv[k], pp[k]));
                mp_add(&X, &t);
            }
            while (mp_cmp(&X, &P) >= 0) mp_sub(&X, &P);
            t = X;
            mp_add(&t, &X);
            const int negative = mp_cmp(&t, &P) > 0; /* X > P/2: the representative is X - P */
            for (uint32_t i = 0; i < n; i++) {
                const uint64_t q = p->prime[i];
                uint64_t Xq = mp_mod_u64(&X, q);
                if (negative) Xq = submod(Xq, P_q[i], q);
                out[((size_t)poly * n + i) * N + c] = mulmod(submod(A[(size_t)i * N + c], Xq, q), Pinv[i], q);
            }
        }
    }
}

/* sigma_g on one limb mod q: X^i -> X^(i g mod 2N), negated past N. */
static void automorph_limb(uint32_t N, const uint64_t* in, uint64_t g, uint64_t q, uint64_t* out)
{
    for (uint32_t i = 0; i < N; i++) {
        uint64_t k = ((uint64_t)i * g) % (2ull * N);
        if (k < N) out[k] = in[i];
        else out[k - N] = negmod(in[i], q);
    }
}

/* Prime index of limb e of the extended basis Q_l u P (e < n: q_e, else p_{e-n}). */
static uint32_t ext_prime(const orc_params* p, uint32_t n, uint32_t e) { return e < n ? e : p->nQ + (e - n); }

/* Steps 1-2 of hybrid key switching for a polynomial d (coefficient form, level
 * l): decompose d into beta = ceil((l+1)/alpha) digits over the primes
 * D_j = {j alpha, ..., min((j+1) alpha, l+1) - 1} and extend each digit to
 * every prime of Q_l u P by fast base conversion; the digit's own primes keep
 * d's residues.  ext: [beta][l+1+nP][N]. */
void orc_modup(const orc_params* p, const uint64_t* d, uint32_t level, uint64_t* ext)
{
    const uint32_t N = p->N, n = level + 1, E = n + p->nP;
    const uint32_t beta = (n + p->alpha - 1) / p->alpha;
    #pragma omp parallel for collapse(2)
    for (uint32_t j = 0; j < beta; j++) {
        for (uint32_t e = 0; e < E; e++) {
            uint32_t lo = j * p->alpha, hi = (j + 1) * p->alpha;
            if (hi > n) hi = n;
            uint64_t* x = ext + ((size_t)j * E + e) * N;
            if (e >= lo && e < hi) {
                memcpy(x, d + (size_t)e * N, sizeof(uint64_t) * N);
            } else {
                uint64_t src[ORC_MAX_PRIMES];
                const uint64_t* xs[ORC_MAX_PRIMES];
                for (uint32_t i = lo; i < hi; i++) {
                    src[i - lo] = p->prime[i];
                    xs[i - lo] = d + (size_t)i * N;
                }
                base_convert(N, xs, src, hi - lo, p->prime[ext_prime(p, n, e)], x);
            }
        }
    }
}

/* Step 3 of hybrid key switching, accumulated: for every limb e of Q_l u P,
 *   acc[0][e] += sum_j sigma_g(x_j[e]) * b_j[e],  acc[1][e] += sum_j sigma_g(x_j[e]) * a_j[e]
 * with the key's digits (b_j, a_j); g = 1 applies no automorphism.  Applying
 * sigma_g to the extended digits of d instead of extending the digits of
 * sigma_g(d) is the hoisted form of a rotation: the decomposition and ModUp of
 * one ciphertext then serve all its rotations. */
void orc_ks_accumulate(const orc_params* p, const uint64_t* ext, uint32_t level, uint64_t g, const uint64_t* ksk,
                       uint64_t* acc)
{
    const uint32_t N = p->N, n = level + 1, E = n + p->nP, L = p->nQ + p->nP;
    const uint32_t beta = (n + p->alpha - 1) / p->alpha;
    #pragma omp parallel for
    for (uint32_t e = 0; e < E; e++) {
        const uint32_t pi = ext_prime(p, n, e);
        const uint64_t t = p->prime[pi];
        uint64_t* x = malloc(sizeof(uint64_t) * N);
        uint64_t* xb = malloc(sizeof(uint64_t) * N);
        uint64_t* xa = malloc(sizeof(uint64_t) * N);
        for (uint32_t j = 0; j < beta; j++) {
            const uint64_t* xj = ext + ((size_t)j * E + e) * N;
            if (g == 1) memcpy(x, xj, sizeof(uint64_t) * N);
            else automorph_limb(N, xj, g, t, x);
            orc_negacyclic_mul(p, pi, x, ksk + ((size_t)(j * 2 + 0) * L + pi) * N, xb);
            orc_negacyclic_mul(p, pi, x, ksk + ((size_t)(j * 2 + 1) * L + pi) * N, xa);
            uint64_t* a0 = acc + (size_t)e * N;
            uint64_t* a1 = acc + ((size_t)E + e) * N;
            for (uint32_t c = 0; c < N; c++) {
                a0[c] = addmod(a0[c], xb[c], t);
                a1[c] = addmod(a1[c], xa[c], t);
            }
        }
        free(x); free(xb); free(xa);
    }
}

/* Hybrid key switching of one polynomial d (coefficient form, level l) with a
 * key from s' to s; returns (k0, k1) with k0 + k1 s ~ d s' (mod Q_l):
 * ModUp (orc_modup), the inner product with the key over Q_l u P
 * (orc_ks_accumulate), and ModDown k_i = round(acc / P) mod q_i (orc_moddown). */
void orc_keyswitch(const orc_params* p, const uint64_t* d, uint32_t level, const uint64_t* ksk,
                   uint64_t* out)
{
    const uint32_t N = p->N, n = level + 1, E = n + p->nP;
    const uint32_t beta = (n + p->alpha - 1) / p->alpha;
    uint64_t* ext = malloc(sizeof(uint64_t) * (size_t)beta * E * N);
    uint64_t* acc = calloc((size_t)2 * E * N, sizeof(uint64_t));
    orc_modup(p, d, level, ext);
    orc_ks_accumulate(p, ext, level, 1, ksk, acc);
    orc_moddown(p, acc, level, out);
    free(ext);
    free(acc);
}

/* Rot_l^r: apply X -> X^g (g = 5^r) to both polynomials, then switch the
 * second from sigma_g(s) back to s and add. */
void orc_rotate(const orc_params* p, const uint64_t* ct, uint32_t level, int32_t r,
                const uint64_t* galois_ksk, uint64_t* out)
{
    const uint32_t N = p->N, n = level + 1;
    const uint64_t g = orc_galois_elt(p, r);
    uint64_t* rc = malloc(sizeof(uint64_t) * 2 * n * N);
    uint64_t* ks = malloc(sizeof(uint64_t) * 2 * n * N);
    orc_automorphism(p, ct, n, g, rc);
    orc_automorphism(p, ct + (size_t)n * N, n, g, rc + (size_t)n * N);
    orc_keyswitch(p, rc + (size_t)n * N, level, galois_ksk, ks);
    for (uint32_t l = 0; l < n; l++) {
        const uint64_t q = p->prime[l];
        for (uint32_t i = 0; i < N; i++) {
            out[(size_t)l * N + i] = addmod(rc[(size_t)l * N + i], ks[(size_t)l * N + i], q);
            out[((size_t)n + l) * N + i] = ks[((size_t)n + l) * N + i];
        }
    }
    free(rc);
    free(ks);
}

/* Hoisted rotations of one ciphertext (c0, c1) by r_0..r_{k-1} (Halevi and
 * Shoup 2018): c1 is decomposed and extended once; rotation r is
 *   (sigma_g(c0) + k0, k1),  (k0, k1) = ModDown( sum_j sigma_g(x_j) (b_j, a_j) ),
 * g = 5^r, x_j the extended digits of c1 and (b_j, a_j) the key for r.
 * out: k ciphertexts of 2 x (l+1) x N words. */
void orc_rotate_hoisted(const orc_params* p, const uint64_t* ct, uint32_t level, uint32_t k, const int32_t* r,
                        const uint64_t* const* galois_ksk, uint64_t* out)
{
    const uint32_t N = p->N, n = level + 1, E = n + p->nP;
    const uint32_t beta = (n + p->alpha - 1) / p->alpha;
    uint64_t* ext = malloc(sizeof(uint64_t) * (size_t)beta * E * N);
    uint64_t* acc = malloc(sizeof(uint64_t) * (size_t)2 * E * N);
    uint64_t* ks = malloc(sizeof(uint64_t) * (size_t)2 * n * N);
    uint64_t* r0 = malloc(sizeof(uint64_t) * (size_t)n * N);
    orc_modup(p, ct + (size_t)n * N, level, ext);
    for (uint32_t x = 0; x < k; x++) {
        const uint64_t g = orc_galois_elt(p, r[x]);
        memset(acc, 0, sizeof(uint64_t) * (size_t)2 * E * N);
        orc_ks_accumulate(p, ext, level, g, galois_ksk[x], acc);
        orc_moddown(p, acc, level, ks);
        orc_automorphism(p, ct, n, g, r0);
        uint64_t* o = out + (size_t)x * 2 * n * N;
        for (uint32_t l = 0; l < n; l++) {
            const uint64_t q = p->prime[l];
            for (uint32_t i = 0; i < N; i++) {
                o[(size_t)l * N + i] = addmod(r0[(size_t)l * N + i], ks[(size_t)l * N + i], q);
                o[((size_t)n + l) * N + i] = ks[((size_t)n + l) * N + i];
            }
        }
    }
    free(ext); free(acc); free(ks); free(r0);
}

/* Sum of rotations with one ModDown (the giant-step sum of a BSGS product):
 *   base + sum_x Rot^{r_x}(T_x)
 * = base + sum_x (sigma_{g_x}(T_x.c0), 0) + ModDown( sum_x sum_j y_{x,j} (b_{x,j}, a_{x,j}) ),
 * y_{x,j} the extended digits of sigma_{g_x}(T_x.c1).  The inner products are
 * summed over Q_l u P before a single division by P.  base may be NULL. */
void orc_rotate_sum(const orc_params* p, const uint64_t* base, const uint64_t* T, uint32_t level, uint32_t k,
                    const int32_t* r, const uint64_t* const* galois_ksk, uint64_t* out)
{
    const uint32_t N = p->N, n = level + 1, E = n + p->nP;
    const uint32_t beta = (n + p->alpha - 1) / p->alpha;
    const size_t ctw = (size_t)2 * n * N;
    uint64_t* ext = malloc(sizeof(uint64_t) * (size_t)beta * E * N);
    uint64_t* acc = calloc((size_t)2 * E * N, sizeof(uint64_t));
    uint64_t* ks = malloc(sizeof(uint64_t) * ctw);
    uint64_t* rc = malloc(sizeof(uint64_t) * ctw);
    if (base) memcpy(out, base, sizeof(uint64_t) * ctw);
    else memset(out, 0, sizeof(uint64_t) * ctw);
    for (uint32_t x = 0; x < k; x++) {
        const uint64_t g = orc_galois_elt(p, r[x]);
        orc_automorphism(p, T + (size_t)x * ctw, n, g, rc);
        orc_automorphism(p, T + (size_t)x * ctw + (size_t)n * N, n, g, rc + (size_t)n * N);
        orc_modup(p, rc + (size_t)n * N, level, ext);
        orc_ks_accumulate(p, ext, level, 1, galois_ksk[x], acc);
        orc_add(p, out, rc, n, out);
    }
    if (k) {
        orc_moddown(p, acc, level, ks);
        orc_add(p, out, ks, n, out);
        orc_add(p, out + (size_t)n * N, ks + (size_t)n * N, n, out + (size_t)n * N);
    }
    free(ext); free(acc); free(ks); free(rc);
}

/* Rescale (Sec. 2.4): divide by the last prime q_l with rounding,
 * c_i <- (c_i - [c]_{q_l}) * q_l^-1 mod q_i, where [c]_{q_l} is the residue
 * mod q_l lifted to the centered range (-q_l/2, q_l/2]. */
void orc_rescale(const orc_params* p, const uint64_t* ct, uint32_t level, uint32_t npolys, uint64_t* out)
{
    const uint32_t N = p->N, n = level + 1;
    const uint64_t ql = p->prime[level];
    for (uint32_t poly = 0; poly < npolys; poly++) {
        const uint64_t* last = ct + ((size_t)poly * n + level) * N;
        for (uint32_t i = 0; i < level; i++) {
            const uint64_t q = p->prime[i];
            const uint64_t inv = invmod(ql % q, q);
            const uint64_t* ci = ct + ((size_t)poly * n + i) * N;
            uint64_t* o = out + ((size_t)poly * level + i) * N;
            for (uint32_t c = 0; c < N; c++) {
                uint64_t v = last[c];
                int64_t centered = v > ql / 2 ? -(int64_t)(ql - v) : (int64_t)v;
                o[c] = mulmod(submod(ci[c], from_signed(centered, q), q), inv, q);
            }
        }
    }
}

/* Limb-wise sum of two polynomials with limbs over primes q_0..q_{nlimbs-1}. */
void orc_add(const orc_params* p, const uint64_t* a, const uint64_t* b, uint32_t nlimbs, uint64_t* out)
{
    const uint32_t N = p->N;
    for (uint32_t l = 0; l < nlimbs; l++)
        for (uint32_t i = 0; i < N; i++)
            out[(size_t)l * N + i] = addmod(a[(size_t)l * N + i], b[(size_t)l * N + i], p->prime[l]);
}

static void ct_add_inplace(const orc_params* p, uint64_t* acc, const uint64_t* b, uint32_t level, uint32_t npolys)
{
    const uint32_t N = p->N, n = level + 1;
    for (uint32_t poly = 0; poly < npolys; poly++)
        for (uint32_t l = 0; l < n; l++) {
            uint64_t* a = acc + ((size_t)poly * n + l) * N;
            const uint64_t* c = b + ((size_t)poly * n + l) * N;
            for (uint32_t i = 0; i < N; i++) a[i] = addmod(a[i], c[i], p->prime[l]);
        }
}

/* ct (x) pt: both polynomials times the plaintext (HomMul with a plaintext). */
void orc_mul_plain(const orc_params* p, const uint64_t* ct, const uint64_t* pt, uint32_t level, uint64_t* out)
{
    const uint32_t N = p->N, n = level + 1;
    #pragma omp parallel for
    for (uint32_t l = 0; l < n; l++)
        for (uint32_t poly = 0; poly < 2; poly++)
            orc_negacyclic_mul(p, l, ct + ((size_t)poly * n + l) * N, pt + (size_t)l * N,
                               out + ((size_t)poly * n + l) * N);
}

/* ct (x) ct before relinearization: (a0 b0, a0 b1 + a1 b0, a1 b1). */
void orc_tensor(const orc_params* p, const uint64_t* a, const uint64_t* b, uint32_t level, uint64_t* out)
{
    const uint32_t N = p->N, n = level + 1;
    #pragma omp parallel for
    for (uint32_t l = 0; l < n; l++) {
        const uint64_t q = p->prime[l];
        uint64_t* t1 = malloc(sizeof(uint64_t) * N);
        uint64_t* t2 = malloc(sizeof(uint64_t) * N);
        const uint64_t *a0 = a + (size_t)l * N, *a1 = a + ((size_t)n + l) * N;
        const uint64_t *b0 = b + (size_t)l * N, *b1 = b + ((size_t)n + l) * N;
        orc_negacyclic_mul(p, l, a0, b0, out + (size_t)l * N);
        orc_negacyclic_mul(p, l, a0, b1, t1);
        orc_negacyclic_mul(p, l, a1, b0, t2);
        for (uint32_t i = 0; i < N; i++) out[((size_t)n + l) * N + i] = addmod(t1[i], t2[i], q);
        orc_negacyclic_mul(p, l, a1, b1, out + ((size_t)2 * n + l) * N);
        free(t1); free(t2);
    }
}

/* (d0, d1, d2) -> (d0 + k0, d1 + k1) with (k0, k1) = KeySwitch_{s^2 -> s}(d2). */
void orc_relinearize(const orc_params* p, const uint64_t* ct3, uint32_t level, const uint64_t* relin_ksk, uint64_t* out)
{
    const uint32_t N = p->N, n = level + 1;
    uint64_t* ks = malloc(sizeof(uint64_t) * 2 * n * N);
    orc_keyswitch(p, ct3 + (size_t)2 * n * N, level, relin_ksk, ks);
    for (uint32_t poly = 0; poly < 2; poly++)
        for (uint32_t l = 0; l < n; l++)
            for (uint32_t i = 0; i < N; i++) {
                size_t o = ((size_t)poly * n + l) * N + i;
                out[o] = addmod(ct3[o], ks[o], p->prime[l]);
            }
    free(ks);
}

/* ------------------------------------------------------------------------- */
/* matmul_cp: ciphertext X (m x d) times plaintext W (d x d_out)               */
/* ------------------------------------------------------------------------- */
/* Packing (spatial-first, Sec. 4.2.1): with s = N/2 slots and k = s/m columns
 * per ciphertext, ciphertext c holds X[i][c*k + b] at slot i + m*b.  Output
 * ciphertext e holds Y[i][e*k + b] the same way.
 * Diagonal method (the ct-pt product of BOLT that Sec. 4.2.1 and 5.2 build on):
 *   Y_e = sum_c sum_{tau<k} Rot_l^{tau m}(X_c) (.) D_{c,e,tau},
 *   D_{c,e,tau}[i + m b] = W[c k + (b + tau) mod k][e k + b].
 * Baby-step giant-step (App. C.1) with tau = g*b1 + b, G = k/b1:
 *   Y_e = sum_g Rot_l^{g b1 m}( sum_c sum_b Rot_l^{b m}(X_c) (.) D'_{c,e,g,b} ),
 *   D'_{c,e,g,b}[i + m beta] = W[c k + (beta + b) mod k][e k + (beta - g b1) mod k],
 * zero outside W.  Plaintexts are encoded at the level of X with scale q_l (the
 * prime the final rescale drops), so Y_e returns to the scale of X. */
uint32_t orc_cp_num_rotations(uint32_t nX, uint32_t nY, uint32_t b1, uint32_t G)
{
    return nX * (b1 - 1) + nY * (G - 1);
}

static const uint64_t* find_galois(const orc_params* p, const orc_galois_set* gk, int32_t r)
{
    uint64_t g = orc_galois_elt(p, r);
    for (uint32_t i = 0; i < gk->n; i++)
        if (gk->gal[i] == g) return gk->ksk[i];
    return NULL;
}

/* Weight at row i of input column r and output column col of a BSGS diagonal;
 * the plain product's weight does not depend on i. */
typedef double (*cp_weight_fn)(const void* w, uint32_t i, uint32_t r, uint32_t col);

typedef struct {
    const double* W;
    uint32_t d, d_out;
} plain_weights;

static double plain_weight(const void* w, uint32_t i, uint32_t r, uint32_t col)
{
    const plain_weights* P = (const plain_weights*)w;
    (void)i;
    return (r < P->d && col < P->d_out) ? P->W[(size_t)r * P->d_out + col] : 0.0;
}

/* Baby steps of the BSGS product (App. C.1): baby[c][b] = Rot^{b m}(X_c) for
 * b < b1 (b = 0 is X_c itself), the b1 - 1 rotations of X_c hoisted (one
 * decomposition and ModUp of X_c serves all of them).  The inputs c are
 * independent (OpenMP over c). */
int orc_cp_baby_steps(const orc_params* p, const orc_galois_set* gk, const uint64_t* X, uint32_t nX,
                      uint32_t level, uint32_t m, uint32_t b1, uint64_t* baby)
{
    const uint32_t N = p->N, s = N / 2, n = level + 1;
    if (level < 1 || m == 0 || s % m || b1 == 0 || (s / m) % b1) return -1;
    const size_t ctw = (size_t)2 * n * N;
    int32_t* rots = malloc(sizeof(int32_t) * b1);
    const uint64_t** keys = malloc(sizeof(uint64_t*) * b1);
    int rc = 0;
    for (uint32_t b = 1; b < b1; b++) {
        rots[b - 1] = (int32_t)(b * m);
        keys[b - 1] = find_galois(p, gk, rots[b - 1]);
        if (!keys[b - 1]) rc = -2;
    }
    if (!rc) {
        #pragma omp parallel for schedule(dynamic) if (nX > 1)
        for (uint32_t c = 0; c < nX; c++) {
            memcpy(baby + ((size_t)c * b1) * ctw, X + (size_t)c * ctw, sizeof(uint64_t) * ctw);
            orc_rotate_hoisted(p, X + (size_t)c * ctw, level, b1 - 1, rots, keys, baby + ((size_t)c * b1 + 1) * ctw);
        }
    }
    free(rots); free(keys);
    return rc;
}

/* The plaintext diagonal D'_{c,e,g,b} as slot values (see above). */
static void cp_diagonal(uint32_t m, uint32_t k, uint32_t b1, cp_weight_fn wf, const void* wctx, uint32_t c,
                        uint32_t e, uint32_t g, uint32_t b, double* z)
{
    for (uint32_t beta = 0; beta < k; beta++) {
        uint32_t row = c * k + (beta + b) % k;
        uint32_t col = e * k + (beta + k - (g * b1) % k) % k;
        for (uint32_t i = 0; i < m; i++) z[i + m * beta] = wf(wctx, i, row, col);
    }
}

/* Inner sum of one giant step of one output (the baby-step sum of App. C.1):
 *   T_g = sum_c sum_b baby[c][b] (.) D'_{c,e,g,b}
 * with the plaintexts D' read from pts ([nX][b1] plaintexts of (level+1) x N
 * words) or, when pts is NULL, encoded here from wf (z and pt are scratch). */
static int cp_inner_sum(const orc_params* p, const uint64_t* baby, uint32_t nX, uint32_t level, uint32_t m,
                        uint32_t b1, const uint64_t* pts, cp_weight_fn wf, const void* wctx, uint32_t e, uint32_t g,
                        double* z, uint64_t* pt, uint64_t* prod, uint64_t* T)
{
    const uint32_t N = p->N, s = N / 2, n = level + 1, k = s / m;
    const size_t ctw = (size_t)2 * n * N, ptw = (size_t)n * N;
    int rc = 0;
    memset(T, 0, sizeof(uint64_t) * ctw);
    for (uint32_t c = 0; c < nX; c++) {
        for (uint32_t b = 0; b < b1; b++) {
            const uint64_t* P;
            if (pts) {
                P = pts + ((size_t)c * b1 + b) * ptw;
            } else {
                cp_diagonal(m, k, b1, wf, wctx, c, e, g, b, z);
                if (orc_encode(p, z, s, level, (double)p->prime[level], pt)) rc = -3;
                P = pt;
            }
            orc_mul_plain(p, baby + ((size_t)c * b1 + b) * ctw, P, level, prod);
            ct_add_inplace(p, T, prod, level, 2);
        }
    }
    return rc;
}

int orc_cp_inner_sum(const orc_params* p, const uint64_t* baby, uint32_t nX, uint32_t level, uint32_t b1,
                     const uint64_t* pts, uint64_t* T)
{
    if (level < 1 || !pts || b1 == 0) return -1;
    uint64_t* prod = malloc(sizeof(uint64_t) * (size_t)2 * (level + 1) * p->N);
    int rc = cp_inner_sum(p, baby, nX, level, 1, b1, pts, NULL, NULL, 0, 0, NULL, NULL, prod, T);
    free(prod);
    return rc;
}

/* Giant steps of the BSGS product for the outputs out_idx[0..n_out):
 *   T_g = the inner sum of giant step g (above), g < G
 *   Y_e = Rescale( T_0 + sum_{g >= 1} Rot^{g b1 m}(T_g) )  (one ModDown for the sum)
 * The plaintexts are read from pts ([n_out][G][nX][b1] plaintexts) when pts is
 * not NULL, else encoded from wf as they are used. */
static int cp_outputs(const orc_params* p, const orc_galois_set* gk, const uint64_t* baby, uint32_t nX,
                      uint32_t level, uint32_t m, uint32_t b1, cp_weight_fn wf, const void* wctx,
                      const uint32_t* out_idx, const uint64_t* pts, uint32_t n_out, uint64_t* Y)
{
    const uint32_t N = p->N, s = N / 2, n = level + 1;
    const uint32_t k = s / m, G = k / b1;
    const size_t ctw = (size_t)2 * n * N, ptw = (size_t)n * N;
    int32_t* rots = malloc(sizeof(int32_t) * G);
    const uint64_t** keys = malloc(sizeof(uint64_t*) * G);
    int rc = 0;
    for (uint32_t g = 1; g < G; g++) {
        rots[g - 1] = (int32_t)(g * b1 * m);
        keys[g - 1] = find_galois(p, gk, rots[g - 1]);
        if (!keys[g - 1]) rc = -2;
    }
    uint64_t* T = malloc(sizeof(uint64_t) * ctw * G);
    uint64_t* acc = malloc(sizeof(uint64_t) * ctw);
    double* z = malloc(sizeof(double) * s);
    uint64_t* pt = malloc(sizeof(uint64_t) * ptw);
    uint64_t* prod = malloc(sizeof(uint64_t) * ctw);
    for (uint32_t oi = 0; oi < n_out && !rc; oi++) {
        const uint32_t e = out_idx ? out_idx[oi] : oi;
        for (uint32_t g = 0; g < G && !rc; g++)
            rc = cp_inner_sum(p, baby, nX, level, m, b1, pts ? pts + ((size_t)oi * G + g) * nX * b1 * ptw : NULL,
                              wf, wctx, e, g, z, pt, prod, T + (size_t)g * ctw);
        if (rc) break;
        orc_rotate_sum(p, T, T + ctw, level, G - 1, rots, keys, acc);
        orc_rescale(p, acc, level, 2, Y + (size_t)oi * 2 * level * N);
    }
    free(rots); free(keys); free(T); free(acc); free(z); free(pt); free(prod);
    return rc;
}

/* BSGS diagonal product (Sec. 4.2.1 / 5.2) for any weight function:
 *   Y_e = Rescale( sum_g Rot^{g b1 m}( sum_c sum_b Rot^{b m}(X_c) (.) D'_{c,e,g,b} ) )
 * with D'_{c,e,g,b}[i + m beta] = w(i, c k + (beta + b) mod k, e k + (beta - g b1) mod k):
 * the baby steps, then the giant steps of each output with its plaintexts
 * encoded as they are used. */
static int matmul_cp_w(const orc_params* p, const orc_galois_set* gk, const uint64_t* X, uint32_t nX,
                       uint32_t level, uint32_t m, cp_weight_fn wf, const void* wctx, uint32_t b1,
                       const uint32_t* out_idx, uint32_t n_out, uint64_t* Y)
{
    const uint32_t N = p->N, s = N / 2, n = level + 1;
    if (level < 1 || m == 0 || s % m) return -1;
    const uint32_t k = s / m;
    if (b1 == 0 || k % b1) return -1;
    uint64_t* baby = malloc(sizeof(uint64_t) * (size_t)2 * n * N * nX * b1);
    int rc = orc_cp_baby_steps(p, gk, X, nX, level, m, b1, baby);
    if (!rc) rc = cp_outputs(p, gk, baby, nX, level, m, b1, wf, wctx, out_idx, NULL, n_out, Y);
    free(baby);
    return rc;
}

/* The plaintexts D'_{c,e,g,b} of the outputs out_idx[0..n_out) of X W (d x d_out,
 * row-major), encoded at `level` with scale q_level, laid out as orc_cp_outputs
 * reads them: [n_out][G][nX][b1] x (level+1) x N words. */
int orc_cp_encode_diagonals(const orc_params* p, uint32_t level, uint32_t m, uint32_t d, const double* W,
                            uint32_t d_out, uint32_t b1, const uint32_t* out_idx, uint32_t n_out, uint64_t* pts)
{
    const uint32_t N = p->N, s = N / 2, n = level + 1;
    if (level < 1 || m == 0 || s % m) return -1;
    const uint32_t k = s / m;
    if (b1 == 0 || k % b1) return -1;
    const uint32_t G = k / b1, nX = (d + k - 1) / k;
    plain_weights w = {W, d, d_out};
    int rc = 0;
    const size_t total = (size_t)n_out * G * nX * b1;
    #pragma omp parallel
    {
        double* z = malloc(sizeof(double) * s);
        #pragma omp for schedule(dynamic)
        for (size_t x = 0; x < total; x++) {
            const uint32_t b = (uint32_t)(x % b1), c = (uint32_t)((x / b1) % nX), g = (uint32_t)((x / b1 / nX) % G);
            const uint32_t oi = (uint32_t)(x / b1 / nX / G);
            cp_diagonal(m, k, b1, plain_weight, &w, c, out_idx ? out_idx[oi] : oi, g, b, z);
            if (orc_encode(p, z, s, level, (double)p->prime[level], pts + x * (size_t)n * N)) {
                #pragma omp atomic write
                rc = -3;
            }
        }
        free(z);
    }
    return rc;
}

/* Giant steps from baby steps (orc_cp_baby_steps) and pre-encoded plaintexts
 * (orc_cp_encode_diagonals): Y holds n_out ciphertexts at level - 1. */
int orc_cp_outputs(const orc_params* p, const orc_galois_set* gk, const uint64_t* baby, uint32_t nX,
                   uint32_t level, uint32_t m, uint32_t b1, const uint64_t* pts, uint32_t n_out, uint64_t* Y)
{
    const uint32_t s = p->N / 2;
    if (level < 1 || m == 0 || s % m || b1 == 0 || (s / m) % b1 || !pts) return -1;
    return cp_outputs(p, gk, baby, nX, level, m, b1, NULL, NULL, NULL, pts, n_out, Y);
}

int orc_matmul_cp(const orc_params* p, const orc_galois_set* gk, const uint64_t* X, uint32_t nX,
                  uint32_t level, uint32_t m, uint32_t d, const double* W, uint32_t d_out,
                  uint32_t b1, const uint32_t* out_idx, uint32_t n_out, uint64_t* Y)
{
    const uint32_t s = p->N / 2;
    if (m == 0 || s % m || nX != (d + s / m - 1) / (s / m)) return -1;
    plain_weights w = {W, d, d_out};
    return matmul_cp_w(p, gk, X, nX, level, m, plain_weight, &w, b1, out_idx, n_out, Y);
}

/* ------------------------------------------------------------------------- */
/* Diagonal-input matmul_cp (App. C.2): E = Concat_h(Att_h) W_O for Att_h in   */
/* the multi-head diagonal packing that matmul_cc returns.                     */
/* ------------------------------------------------------------------------- */
/* Input: for each head group (Hg heads, Kc = s/(L Hg)), the Dh/Kc ciphertexts
 * of Att_h in *dense* diagonal packing: matmul_cc's outputs j and j + Dh/Kc
 * added (V_h padded from Dh to L = 2 Dh columns makes diagonals delta and
 * delta + Dh complementary), so merged ciphertext j holds, at block
 * h + Hg kappa, element i = Att_h[i][(i + delta) mod Dh], delta = j Kc + kappa.
 * Input column r = c k + beta (k = s/L) of the product is that block; with
 * (h, delta) its head (global index) and diagonal,
 *   E[i][o] = sum_{h, delta} Att_h[i][(i + delta) mod Dh] W_O[h Dh + (i + delta) mod Dh][o],
 * i.e. the BSGS product with the row-dependent weight
 *   w(i, r, o) = W_O[h Dh + (i + delta) mod Dh][o]. */
typedef struct {
    const double* W;      /* (H Dh) x d_out */
    uint32_t Dh, d_out, ncols;
    const int32_t* head;  /* per input column: global head, -1 = unused */
    const int32_t* delta; /* per input column: diagonal */
} diag_weights;

static double diag_weight(const void* w, uint32_t i, uint32_t r, uint32_t col)
{
    const diag_weights* D = (const diag_weights*)w;
    if (r >= D->ncols || col >= D->d_out || D->head[r] < 0) return 0.0;
    const uint32_t row = (uint32_t)D->head[r] * D->Dh + (i + (uint32_t)D->delta[r]) % D->Dh;
    return D->W[(size_t)row * D->d_out + col];
}

uint32_t orc_cp_diag_inputs(uint32_t s, uint32_t L, uint32_t n_groups, const uint32_t* Hg, uint32_t Dh)
{
    uint32_t nX = 0;
    for (uint32_t g = 0; g < n_groups; g++) {
        const uint32_t Kc = s / (L * Hg[g]);
        nX += Dh / Kc;
    }
    return nX;
}

int orc_matmul_cp_diag(const orc_params* p, const orc_galois_set* gk, const uint64_t* X, uint32_t level, uint32_t L,
                       uint32_t n_groups, const uint32_t* Hg, uint32_t Dh, const double* W, uint32_t d_out,
                       uint32_t b1, const uint32_t* out_idx, uint32_t n_out, uint64_t* Y)
{
    const uint32_t s = p->N / 2;
    if (L == 0 || s % L || L != 2 * Dh) return -1;
    const uint32_t k = s / L, nX = orc_cp_diag_inputs(s, L, n_groups, Hg, Dh);
    int32_t* head = malloc(sizeof(int32_t) * nX * k);
    int32_t* delta = malloc(sizeof(int32_t) * nX * k);
    uint32_t c = 0, h0 = 0;
    int rc = 0;
    for (uint32_t g = 0; g < n_groups && !rc; g++) {
        if (s % (L * Hg[g])) { rc = -1; break; }
        const uint32_t Kc = s / (L * Hg[g]);
        if (Dh % Kc) { rc = -1; break; }
        for (uint32_t j = 0; j < Dh / Kc; j++, c++)
            for (uint32_t beta = 0; beta < k; beta++) {
                head[c * k + beta] = (int32_t)(h0 + beta % Hg[g]);
                delta[c * k + beta] = (int32_t)(j * Kc + beta / Hg[g]);
            }
        h0 += Hg[g];
    }
    if (!rc) {
        diag_weights w = {W, Dh, d_out, nX * k, head, delta};
        rc = matmul_cp_w(p, gk, X, nX, level, L, diag_weight, &w, b1, out_idx, n_out, Y);
    }
    free(head);
    free(delta);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* matmul_cc: ciphertext A (L x R per head) times ciphertext B (R x L per head) */
/* ------------------------------------------------------------------------- */
/* Multi-head packing (Sec. 5.1): s = N/2 slots in blocks of L; block
 * beta = h + Hg * kappa of input ciphertext c holds column k = c Kc + kappa of
 * A_h (spatial-first) or row k of B_h (reduce-first), Kc = s / (L Hg).
 * Output ciphertext j (of L/Kc) holds diagonal delta = j Kc + kappa' of
 * C_h = A_h B_h at block h + Hg kappa', element i = C_h[i][(i + delta) mod L].
 * Schedule (Sec. 5.1 steps 1-3, baby-step giant-step of App. C.1), with
 * b1s1 | Kc and b1s2 | L, G1 = Kc/b1s1, G2 = L/b1s2:
 *   1. B'_c = Rescale( sum_{g1} Rot^{g1 b1s1}( sum_{b0} m1lo(g1,b0) Rot^{b0}(B_c)
 *                                                + m1hi(g1,b0) Rot^{b0-L}(B_c) ) )
 *      -- block kappa = g1 b1s1 + b0 of B'_c holds B[k][(i + kappa) mod L];
 *   2. for t = g b1s2 + b:
 *      V_c = m2lo(g,b) Rot^{b}(B'_c) + m2hi(g,b) Rot^{b-L}(B'_c)     (level l-1),
 *      W_t = Rescale( Relin( Rescale( sum_c Rot^{-g b1s2}(A_c) (x) V_c ) ) )
 *      with A_c dropped to level l-1: the masked copies are multiplied before
 *      rescaling and the sum over c is rescaled once (the paper fixes the depth,
 *      4, not where the rescales fall; this placement keeps it)
 *      -- Rot^{g b1s2}(W_t) would hold diagonal (t + kappa) mod L at block kappa;
 *   3. C_j = Rescale( sum_t m3(t, j) Rot^{g b1s2 - (t mod Kc) Hg L}(W_t) ).
 * The rotations of one ciphertext in steps 1 and 2 (of B_c, B'_c and A_c) are
 * hoisted (orc_rotate_hoisted) and the giant-step sum of step 1 takes one
 * ModDown (orc_rotate_sum); step 3 and the relinearizations switch one
 * ciphertext each.
 * Masks (0/1 slot vectors, encoded at scale q_level of the level they are
 * applied at): m1lo(g1,b0) = Rot^{-g1 b1s1}([kappa(slot) = g1 b1s1 + b0 and
 * i < L - kappa]), m1hi likewise with i >= L - kappa; m2lo(g,b) =
 * Rot^{-g b1s2}([i < L - t]), m2hi with i >= L - t; m3(t, j) = [the block that
 * lands at kappa' comes from kappa = (kappa' - t) mod Kc and carries diagonal
 * (t + kappa) mod L in output j].  Depth 4 (two mask levels, the tensor, the
 * routing masks). */
static int slot_kappa(uint32_t slot, uint32_t L, uint32_t Hg) { return (int)((slot / L) / Hg); }

static void drop_limbs(const orc_params* p, const uint64_t* ct, uint32_t from_level, uint32_t to_level,
                       uint32_t npolys, uint64_t* out)
{
    const uint32_t N = p->N;
    for (uint32_t poly = 0; poly < npolys; poly++)
        memcpy(out + (size_t)poly * (to_level + 1) * N, ct + (size_t)poly * (from_level + 1) * N,
               sizeof(uint64_t) * (to_level + 1) * N);
}

/* z[slot] = mask value of slot (slot - shift) mod s, i.e. Rot^{-shift} of the
 * unrotated mask; returns whether the mask has any nonzero entry */
static int build_mask(double* z, uint32_t s, int64_t shift, int (*pred)(uint32_t, const int64_t*), const int64_t* args)
{
    int any = 0;
    for (uint32_t slot = 0; slot < s; slot++) {
        uint32_t src = (uint32_t)((((int64_t)slot - shift) % (int64_t)s + s) % s);
        z[slot] = pred(src, args) ? 1.0 : 0.0;
        any |= z[slot] != 0.0;
    }
    return any;
}

/* args: {L, Hg, kappa, hi} */
static int pred_m1(uint32_t slot, const int64_t* a)
{
    uint32_t L = (uint32_t)a[0], Hg = (uint32_t)a[1];
    int64_t kappa = a[2];
    int64_t i = slot % L;
    if (slot_kappa(slot, L, Hg) != kappa) return 0;
    return a[3] ? (i >= (int64_t)L - kappa) : (i < (int64_t)L - kappa);
}
/* args: {L, t, hi} */
static int pred_m2(uint32_t slot, const int64_t* a)
{
    int64_t L = a[0], t = a[1], i = slot % L;
    return a[2] ? (i >= L - t) : (i < L - t);
}
/* args: {L, Hg, Kc, t, j} */
static int pred_m3(uint32_t slot, const int64_t* a)
{
    int64_t L = a[0], Hg = a[1], Kc = a[2], t = a[3], j = a[4];
    int64_t kp = (slot / L) / Hg;
    int64_t kappa = ((kp - t) % Kc + Kc) % Kc;
    int64_t delta = (t + kappa) % L;
    return delta / Kc == j;
}

uint32_t orc_cc_num_rotations(uint32_t n_c, uint32_t L, uint32_t Kc, uint32_t b1s1, uint32_t b1s2)
{
    uint32_t G1 = Kc / b1s1, G2 = L / b1s2;
    uint32_t s1 = (b1s1 - 1) + (G1 > 1 ? b1s1 : b1s1 - 1) + (G1 - 1);
    uint32_t s2 = (b1s2 - 1) + b1s2 + (G2 - 1);
    return n_c * (s1 + s2) + (L - 1);
}

/* acc += ct (x) encode(mask); skipped when the mask is zero */
static int mac_mask(const orc_params* p, uint64_t* acc, const uint64_t* ct, uint32_t level, double* z,
                    uint64_t* pt, uint64_t* prod)
{
    const uint32_t s = p->N / 2;
    if (orc_encode(p, z, s, level, (double)p->prime[level], pt)) return -3;
    orc_mul_plain(p, ct, pt, level, prod);
    ct_add_inplace(p, acc, prod, level, 2);
    return 0;
}

int orc_matmul_cc(const orc_params* p, const orc_galois_set* gk, const uint64_t* relin_ksk, const uint64_t* A,
                  const uint64_t* B, uint32_t n_c, uint32_t level, uint32_t L, uint32_t Hg, uint32_t b1s1,
                  uint32_t b1s2, uint64_t* C)
{
    const uint32_t N = p->N, s = N / 2;
    if (level < 4 || L == 0 || Hg == 0 || s % (L * Hg)) return -1;
    const uint32_t Kc = s / (L * Hg);
    if (Kc == 0 || L % Kc || b1s1 == 0 || Kc % b1s1 || b1s2 == 0 || L % b1s2) return -1;
    const uint32_t G1 = Kc / b1s1, G2 = L / b1s2, nout = L / Kc;
    const uint32_t l0 = level, l1 = level - 1, l2 = level - 2, l3 = level - 3;
    const size_t w0 = (size_t)2 * (l0 + 1) * N, w1 = (size_t)2 * (l1 + 1) * N, w2 = (size_t)2 * (l2 + 1) * N;
    const size_t w3 = (size_t)2 * (l3 + 1) * N;
    double* z = malloc(sizeof(double) * s);
    uint64_t* pt = malloc(sizeof(uint64_t) * (l0 + 1) * N);
    uint64_t* prod = malloc(sizeof(uint64_t) * w0);
    uint64_t* tmp = malloc(sizeof(uint64_t) * w0);
    uint64_t* Bp = calloc((size_t)n_c * w1, sizeof(uint64_t));
    uint64_t* W = calloc((size_t)L * w3, sizeof(uint64_t));
    int rc = 0;

    /* step 1: baby steps of B_c hoisted (one ModUp), giant steps summed with one ModDown */
    {
        uint64_t* lo = malloc(sizeof(uint64_t) * w0 * b1s1);
        uint64_t* hi = malloc(sizeof(uint64_t) * w0 * b1s1);
        uint64_t* rot = malloc(sizeof(uint64_t) * w0 * 2 * b1s1);
        uint64_t* acc = malloc(sizeof(uint64_t) * w0);
        uint64_t* inner = malloc(sizeof(uint64_t) * w0 * G1);
        int32_t rs[2 * ORC_MAX_ROT];
        const uint64_t* ks[2 * ORC_MAX_ROT];
        if (2 * b1s1 > 2 * ORC_MAX_ROT || G1 > 2 * ORC_MAX_ROT) rc = -1;
        for (uint32_t c = 0; c < n_c && !rc; c++) {
            const uint64_t* Bc = B + (size_t)c * w0;
            /* rotations b0 (b0 >= 1) and b0 - L (b0 >= 1, or all b0 when G1 > 1) */
            uint32_t nr = 0;
            for (uint32_t b0 = 1; b0 < b1s1; b0++) rs[nr++] = (int32_t)b0;
            for (uint32_t b0 = (G1 > 1 ? 0 : 1); b0 < b1s1; b0++) rs[nr++] = (int32_t)b0 - (int32_t)L;
            for (uint32_t x = 0; x < nr && !rc; x++)
                if (!(ks[x] = find_galois(p, gk, rs[x]))) rc = -2;
            if (rc) break;
            orc_rotate_hoisted(p, Bc, l0, nr, rs, ks, rot);
            memcpy(lo, Bc, sizeof(uint64_t) * w0);
            for (uint32_t x = 0; x < nr; x++) {
                const int32_t r = rs[x];
                uint64_t* dst = r > 0 ? lo + (size_t)r * w0 : hi + (size_t)(r + (int32_t)L) * w0;
                memcpy(dst, rot + (size_t)x * w0, sizeof(uint64_t) * w0);
            }
            for (uint32_t g1 = 0; g1 < G1 && !rc; g1++) {
                uint64_t* in = inner + (size_t)g1 * w0;
                memset(in, 0, sizeof(uint64_t) * w0);
                for (uint32_t b0 = 0; b0 < b1s1 && !rc; b0++) {
                    int64_t args[4] = {L, Hg, (int64_t)(g1 * b1s1 + b0), 0};
                    if (build_mask(z, s, (int64_t)g1 * b1s1, pred_m1, args))
                        rc = mac_mask(p, in, lo + (size_t)b0 * w0, l0, z, pt, prod);
                    args[3] = 1;
                    if (!rc && build_mask(z, s, (int64_t)g1 * b1s1, pred_m1, args))
                        rc = mac_mask(p, in, hi + (size_t)b0 * w0, l0, z, pt, prod);
                }
            }
            for (uint32_t g1 = 1; g1 < G1 && !rc; g1++) {
                rs[g1 - 1] = (int32_t)(g1 * b1s1);
                if (!(ks[g1 - 1] = find_galois(p, gk, rs[g1 - 1]))) rc = -2;
            }
            if (rc) break;
            orc_rotate_sum(p, inner, inner + w0, l0, G1 - 1, rs, ks, acc);
            orc_rescale(p, acc, l0, 2, Bp + (size_t)c * w1);
        }
        free(lo); free(hi); free(rot); free(acc); free(inner);
    }
    if (rc) goto done;

    /* step 2: baby steps of B'_c and giant steps of A_c hoisted */
    {
        const size_t w1_3 = (size_t)3 * (l1 + 1) * N, w2_3 = (size_t)3 * (l2 + 1) * N;
        uint64_t* U = calloc((size_t)L * w1_3, sizeof(uint64_t));
        uint64_t* blo = malloc(sizeof(uint64_t) * w1 * b1s2);
        uint64_t* bhi = malloc(sizeof(uint64_t) * w1 * b1s2);
        uint64_t* rot = malloc(sizeof(uint64_t) * w1 * 2 * (b1s2 > G2 ? b1s2 : G2));
        uint64_t* Ag = malloc(sizeof(uint64_t) * w1 * G2);
        uint64_t* A1 = malloc(sizeof(uint64_t) * w1);
        int32_t rs[2 * ORC_MAX_ROT];
        const uint64_t* ks[2 * ORC_MAX_ROT];
        if (2 * b1s2 > 2 * ORC_MAX_ROT || G2 > 2 * ORC_MAX_ROT) rc = -1;
        for (uint32_t c = 0; c < n_c && !rc; c++) {
            const uint64_t* Bc = Bp + (size_t)c * w1;
            uint32_t nr = 0;
            for (uint32_t b = 1; b < b1s2; b++) rs[nr++] = (int32_t)b;
            for (uint32_t b = (G2 > 1 ? 0 : 1); b < b1s2; b++) rs[nr++] = (int32_t)b - (int32_t)L;
            for (uint32_t x = 0; x < nr && !rc; x++)
                if (!(ks[x] = find_galois(p, gk, rs[x]))) rc = -2;
            if (rc) break;
            orc_rotate_hoisted(p, Bc, l1, nr, rs, ks, rot);
            memcpy(blo, Bc, sizeof(uint64_t) * w1);
            for (uint32_t x = 0; x < nr; x++) {
                const int32_t r = rs[x];
                uint64_t* dst = r > 0 ? blo + (size_t)r * w1 : bhi + (size_t)(r + (int32_t)L) * w1;
                memcpy(dst, rot + (size_t)x * w1, sizeof(uint64_t) * w1);
            }
            drop_limbs(p, A + (size_t)c * w0, l0, l1, 2, A1);
            memcpy(Ag, A1, sizeof(uint64_t) * w1);
            for (uint32_t g = 1; g < G2 && !rc; g++) {
                rs[g - 1] = -(int32_t)(g * b1s2);
                if (!(ks[g - 1] = find_galois(p, gk, rs[g - 1]))) rc = -2;
            }
            if (rc) break;
            orc_rotate_hoisted(p, A1, l1, G2 - 1, rs, ks, Ag + w1);
            /* the L diagonals t = g b1s2 + b are independent: each adds into its own U_t */
            #pragma omp parallel
            {
                double* zt = malloc(sizeof(double) * s);
                uint64_t* ptt = malloc(sizeof(uint64_t) * (l0 + 1) * N);
                uint64_t* prodt = malloc(sizeof(uint64_t) * w0);
                uint64_t* vt = malloc(sizeof(uint64_t) * w1);
                uint64_t* T3t = malloc(sizeof(uint64_t) * w1_3);
                #pragma omp for schedule(dynamic)
                for (uint32_t t = 0; t < L; t++) {
                    const uint32_t g = t / b1s2, b = t % b1s2;
                    int trc = 0, used = 0;
                    memset(vt, 0, sizeof(uint64_t) * w1);
                    int64_t args[3] = {L, t, 0};
                    if (build_mask(zt, s, (int64_t)g * b1s2, pred_m2, args)) {
                        trc = mac_mask(p, vt, blo + (size_t)b * w1, l1, zt, ptt, prodt);
                        used = 1;
                    }
                    args[2] = 1;
                    if (!trc && build_mask(zt, s, (int64_t)g * b1s2, pred_m2, args)) {
                        trc = mac_mask(p, vt, bhi + (size_t)b * w1, l1, zt, ptt, prodt);
                        used = 1;
                    }
                    if (trc) {
                        #pragma omp atomic write
                        rc = trc;
                    }
                    if (trc || !used) continue;
                    orc_tensor(p, Ag + (size_t)g * w1, vt, l1, T3t);
                    uint64_t* Ut = U + (size_t)t * w1_3;
                    for (uint32_t poly = 0; poly < 3; poly++)
                        orc_add(p, Ut + (size_t)poly * (l1 + 1) * N, T3t + (size_t)poly * (l1 + 1) * N, l1 + 1,
                                Ut + (size_t)poly * (l1 + 1) * N);
                }
                free(zt); free(ptt); free(prodt); free(vt); free(T3t);
            }
        }
        if (!rc) {
            #pragma omp parallel for schedule(dynamic)
            for (uint32_t t = 0; t < L; t++) {
                uint64_t* U2 = malloc(sizeof(uint64_t) * w2_3);
                uint64_t* R2 = malloc(sizeof(uint64_t) * w2);
                orc_rescale(p, U + (size_t)t * w1_3, l1, 3, U2);
                orc_relinearize(p, U2, l2, relin_ksk, R2);
                orc_rescale(p, R2, l2, 2, W + (size_t)t * w3);
                free(U2);
                free(R2);
            }
        }
        free(U); free(blo); free(bhi); free(rot); free(Ag); free(A1);
    }
    if (rc) goto done;

    /* step 3 */
    {
        uint64_t* Cacc = calloc((size_t)nout * w3, sizeof(uint64_t));
        uint64_t* Rall = malloc(sizeof(uint64_t) * w3 * L);
        /* the L rotations first (independent), then the masked sums */
        for (uint32_t t = 0; t < L && !rc; t++) {
            const uint32_t g = t / b1s2;
            const int64_t r = (((int64_t)g * b1s2 - (int64_t)(t % Kc) * Hg * L) % (int64_t)s + s) % s;
            if (r != 0 && !find_galois(p, gk, (int32_t)r)) rc = -2;
        }
        if (rc) { free(Cacc); free(Rall); goto done; }
        #pragma omp parallel for schedule(dynamic)
        for (uint32_t t = 0; t < L; t++) {
            const uint32_t g = t / b1s2;
            const int64_t r = (((int64_t)g * b1s2 - (int64_t)(t % Kc) * Hg * L) % (int64_t)s + s) % s;
            uint64_t* Rt = Rall + (size_t)t * w3;
            if (r == 0) memcpy(Rt, W + (size_t)t * w3, sizeof(uint64_t) * w3);
            else orc_rotate(p, W + (size_t)t * w3, l3, (int32_t)r, find_galois(p, gk, (int32_t)r), Rt);
        }
        for (uint32_t t = 0; t < L && !rc; t++) {
            const uint64_t* Rt = Rall + (size_t)t * w3;
            for (uint32_t j = 0; j < nout && !rc; j++) {
                int64_t args[5] = {L, Hg, Kc, t, j};
                if (build_mask(z, s, 0, pred_m3, args))
                    rc = mac_mask(p, Cacc + (size_t)j * w3, Rt, l3, z, pt, prod);
            }
        }
        for (uint32_t j = 0; j < nout && !rc; j++)
            orc_rescale(p, Cacc + (size_t)j * w3, l3, 2, C + (size_t)j * 2 * l3 * N);
        free(Cacc); free(Rall);
    }
done:
    free(z); free(pt); free(prod); free(tmp); free(Bp); free(W);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* CKKS -> MPC masking (Alg. 1, first two steps; Sec. 6.3)                      */
/* ------------------------------------------------------------------------- */
/* The paper's conversion works modulo a single prime q.  The ciphertext is
 * first reduced to level 0 (drop every limb but q_0), then P1 adds a mask
 * r drawn uniformly from Z_{q_0}[X]/(X^N+1) (purpose MASK, keyed by the nonce)
 * to the first polynomial and keeps -r as its share.  P0's share is the
 * decryption of the masked ciphertext; the two shares sum to the message plus
 * noise mod q_0. */
void orc_he2mpc(const orc_params* p, const uint64_t* ct, uint32_t level, uint64_t seed,
                uint32_t nonce, uint64_t* masked, uint64_t* p1_share)
{
    const uint32_t N = p->N, n = level + 1;
    const uint64_t q0 = p->prime[0];
    uint64_t* r = malloc(sizeof(uint64_t) * N);
    orc_sample_uniform(N, q0, seed, nonce, ORC_MASK, 0, r);
    for (uint32_t i = 0; i < N; i++) {
        masked[i] = addmod(ct[i], r[i], q0);
        masked[N + i] = ct[(size_t)n * N + i];
        p1_share[i] = negmod(r[i], q0);
    }
    free(r);
}

/* ------------------------------------------------------------------------- */
/* local parts of the conversions between CKKS and additive shares            */
/* (Alg. 1 steps 3-4, Alg. 2, Sec. 6.3, App. C.3)                              */
/* ------------------------------------------------------------------------- */
/* Shares of the extended ring Z_{2^128} are unsigned 128-bit integers, stored
 * as two words (low, high) per element.  The paper extends the l-bit MPC ring
 * (l = 43, fixed-point scale 2^13, Sec. 7.1) to a larger ring so that every
 * local truncation inside the share FFTs fails with probability below 2^-40
 * (its example width is l + 40).  A truncated product here is the FFT datum
 * (resolution 2^-ORC_FX_P slot units) times a root with ORC_FX_F fraction bits,
 * about 2^87 for slot values up to 2^31, so the ring taken is Z_{2^128}: the
 * failure probability of one truncation of m is |m| / 2^128.
 *
 * The interactive comparisons inside the ring/field extensions (Pi_Ext of
 * SiRNN, as BOLT adapts it) are MPC protocols; here only their ideal
 * functionality is simulated (orc_*_wrap_sim), and everything each party then
 * computes on its own share is written out step by step. */

static u128 ld128(const uint64_t* w, size_t i) { return (u128)w[2 * i] | ((u128)w[2 * i + 1] << 64); }
static void st128(uint64_t* w, size_t i, u128 v)
{
    w[2 * i] = (uint64_t)v;
    w[2 * i + 1] = (uint64_t)(v >> 64);
}

/* Probabilistic truncation by k bits (SecureML, as App. C.3 specifies it: the
 * result is floor(m / 2^k) + u with Pr[u = 1] = (m mod 2^k) / 2^k).  Each party
 * reads its share as a signed 128-bit integer; P0 takes floor(x / 2^k) (an
 * arithmetic shift right), P1 takes ceil(x / 2^k) = -floor(-x / 2^k), SecureML's
 * two local operations.  Shifting both shares alone would subtract one more
 * unit on average, a bias that the FFTs below would accumulate.  The result
 * is wrong (off by about 2^(128-k)) only when the two signed shares overflow
 * when added, with probability |m| / 2^128. */
static u128 trunc_share(u128 x, uint32_t k, uint32_t party)
{
    if (party == 0) return (u128)((__int128)x >> k);
    return (u128)0 - (u128)((__int128)((u128)0 - x) >> k);
}

void orc_share_trunc(uint32_t party, const uint64_t* x, uint64_t n, uint32_t k, uint64_t* out)
{
    for (uint64_t i = 0; i < n; i++) st128(out, i, trunc_share(ld128(x, i), k, party));
}

/* Fixed-point root c zeta^k = (round(2^F c cos(pi k/N)), round(2^F c sin(pi k/N)))
 * from the C library's cos and sin, rounded half to even. */
static void fx_zeta(uint32_t N, uint32_t k, double c, int64_t* re, int64_t* im)
{
    double ang = M_PI * (double)k / (double)N;
    *re = (int64_t)rint(ldexp(cos(ang) * c, ORC_FX_F));
    *im = (int64_t)rint(ldexp(sin(ang) * c, ORC_FX_F));
}

typedef struct { u128 re, im; } cshare;

/* share times a signed integer, mod 2^128 */
static u128 smul(u128 a, int64_t w) { return a * (u128)(__int128)w; }

/* (v.re + i v.im)(wr + i wi) before truncation */
static cshare cmul_share(cshare v, int64_t wr, int64_t wi)
{
    cshare r = {smul(v.re, wr) - smul(v.im, wi), smul(v.re, wi) + smul(v.im, wr)};
    return r;
}

/* Arithmetic shares over Z_{2^128} of the bit w, as the comparison inside
 * Pi_Ext hands them out (ideal functionality): P0 receives rho, the 128-bit
 * Philox draw (i, 0, nonce, WRAP) keyed by seed (word 3 most significant), P1
 * receives w - rho. */
static void share_bit(uint32_t w, uint64_t seed, uint32_t i, uint32_t nonce, uint64_t* w0, uint64_t* w1)
{
    uint32_t d[4];
    draw(seed, i, 0, nonce, ORC_WRAP, d);
    u128 rho = ((u128)d[3] << 96) | ((u128)d[2] << 64) | ((u128)d[1] << 32) | (u128)d[0];
    st128(w0, i, rho);
    st128(w1, i, (u128)w - rho);
}

/* Field to ring, signed form of Pi_Ext^{q, 2^128} (App. C.3): the message m
 * is centered in [-h, h], h = (q-1)/2.  P0 adds h to its share, so the two
 * shares sum (mod q) to m + h in [0, q); the comparison yields the wrap bit
 * w = [(t0 + h mod q) + t1 >= q], shared over Z_{2^128}. */
void orc_f2r_wrap_sim(uint32_t n, uint64_t q, const uint64_t* t0, const uint64_t* t1, uint64_t seed,
                      uint32_t nonce, uint64_t* w0, uint64_t* w1)
{
    const uint64_t h = (q - 1) / 2;
    for (uint32_t i = 0; i < n; i++) {
        uint64_t a = addmod(t0[i], h, q);
        share_bit(a + t1[i] >= q, seed, i, nonce, w0, w1);
    }
}

/* Local step of party b: U_b = t_b' - <w>_b q - [b = 0] h (mod 2^128) with
 * t_0' = t_0 + h mod q and t_1' = t_1, so U_0 + U_1 = (t_0' + t_1 - w q) - h = m. */
void orc_f2r_local(uint32_t party, uint32_t n, uint64_t q, const uint64_t* t, const uint64_t* wsh, uint64_t* U)
{
    const uint64_t h = (q - 1) / 2;
    for (uint32_t i = 0; i < n; i++) {
        u128 tp = party == 0 ? addmod(t[i], h, q) : t[i];
        u128 u = tp - ld128(wsh, i) * (u128)q - (party == 0 ? (u128)h : 0);
        st128(U, i, u);
    }
}

/* Signed extension Pi_Ext^{2^l, 2^128} (SiRNN) with the same offset: P0 adds
 * 2^(l-1) to its share, the comparison yields w = [x0' + x1 >= 2^l]. */
void orc_ext_wrap_sim(uint32_t n, uint32_t l, const uint64_t* x0, const uint64_t* x1, uint64_t seed,
                      uint32_t nonce, uint64_t* w0, uint64_t* w1)
{
    const uint64_t M = 1ull << l, mask = M - 1;
    for (uint32_t i = 0; i < n; i++) {
        uint64_t a = (x0[i] + (M >> 1)) & mask;
        share_bit(a + (x1[i] & mask) >= M, seed, i, nonce, w0, w1);
    }
}

/* X_b = x_b' - <w>_b 2^l - [b = 0] 2^(l-1) (mod 2^128), x_0' = x_0 + 2^(l-1) mod 2^l,
 * x_1' = x_1: X_0 + X_1 is the signed value of x_0 + x_1 mod 2^l. */
void orc_ext_local(uint32_t party, uint32_t n, uint32_t l, const uint64_t* x, const uint64_t* wsh, uint64_t* X)
{
    const uint64_t M = 1ull << l, mask = M - 1;
    for (uint32_t i = 0; i < n; i++) {
        u128 xp = party == 0 ? ((x[i] + (M >> 1)) & mask) : (x[i] & mask);
        u128 v = xp - (ld128(wsh, i) << l) - (party == 0 ? (u128)(M >> 1) : 0);
        st128(X, i, v);
    }
}

/* Ring to field (App. C.3).  The paper's equation takes [m]_0 = M_0 mod q and
 * [m]_1 = M_1 - 2^128 mod q, which is right when M_0 + M_1 = m + 2^128 as
 * integers, i.e. when exactly one of the two shares, read as a signed integer,
 * is negative.  Each party here reads its own share as a signed integer in
 * [-2^127, 2^127) and reduces that mod q_i: the same residues in that case, and
 * also right when both shares have one sign (two zero shares of a coefficient
 * the FFT leaves structurally zero, or two truncated shares that happen to be
 * small); it fails only when the signed shares overflow when added, with
 * probability |m| / 2^128.  Output for every prime q_0..q_level. */
void orc_r2f_local(const orc_params* p, uint32_t party, uint32_t n, const uint64_t* M, uint32_t level,
                   uint64_t* out /* (level+1) x n */)
{
    (void)party;
    for (uint32_t li = 0; li <= level; li++) {
        const uint64_t q = p->prime[li];
        const uint64_t two64 = (uint64_t)(((u128)1 << 64) % q);
        const uint64_t two128 = mulmod(two64, two64, q);
        for (uint32_t i = 0; i < n; i++) {
            u128 v = ld128(M, i);
            uint64_t r = (uint64_t)(v % q);
            out[(size_t)li * n + i] = (v >> 127) ? submod(r, two128, q) : r;
        }
    }
}

/* CKKS -> MPC, what party b computes after masking and decryption (Alg. 1
 * steps 3-4): t is its share of the coefficients of Encode(x) mod q_0 (P0: the
 * decryption of the masked ciphertext, P1: minus the mask), wsh its share of
 * the field-to-ring wrap bits.  Then
 *   1. field to ring: U = shares of the centered coefficients m over Z_{2^128};
 *   2. y_t = U_t / 2^(e-P) (local truncation; a shift left when e < P), where
 *      the scale is Delta = mu 2^e with mu in [1, 2);
 *   3. twist: c_t = (y_t + i y_{t+s}) * round(2^F zeta^t / mu) / 2^F;
 *   4. the s-point DFT of the decoding (see orc_decode) as radix-2
 *      decimation in time on bit-reversed input, every product by a root
 *      round(2^F omega^k) truncated by F before the butterfly's sum and
 *      difference;
 *   5. slot j: the real part at k_j = (5^j - 1)/4, truncated from 2^-P to the
 *      MPC scale 2^-sf and reduced mod 2^l.
 * out receives the N/2 slot shares in Z_{2^l}. */
int orc_c2m_local(const orc_params* p, uint32_t party, const uint64_t* t, const uint64_t* wsh, double scale,
                  uint32_t l, uint32_t sf, uint64_t* out)
{
    const uint32_t N = p->N, s = N / 2, logs = p->logN - 1;
    const uint32_t F = ORC_FX_F, P = ORC_FX_P;
    if (l > 62 || sf > P || l < sf + 2 || !(scale > 0)) return -1;
    int ex;
    const double mu = 2.0 * frexp(scale, &ex); /* scale = mu 2^e, mu in [1, 2) */
    const int e = ex - 1;
    if (e - (int)P >= 64 || (int)P - e >= 64) return -1;
    uint64_t* U = malloc(sizeof(uint64_t) * 2 * N);
    cshare* A = malloc(sizeof(cshare) * s);
    orc_f2r_local(party, N, p->prime[0], t, wsh, U);
    const double c = 1.0 / mu;
    for (uint32_t k = 0; k < s; k++) {
        cshare y = {ld128(U, k), ld128(U, k + s)};
        if (e >= (int)P) {
            y.re = trunc_share(y.re, (uint32_t)(e - (int)P), party);
            y.im = trunc_share(y.im, (uint32_t)(e - (int)P), party);
        } else {
            y.re <<= (uint32_t)((int)P - e);
            y.im <<= (uint32_t)((int)P - e);
        }
        int64_t wr, wi;
        fx_zeta(N, k, c, &wr, &wi);
        cshare v = cmul_share(y, wr, wi);
        A[bitrev(k, logs)] = (cshare){trunc_share(v.re, F, party), trunc_share(v.im, F, party)};
    }
    for (uint32_t len = 2; len <= s; len <<= 1) {
        const uint32_t half = len / 2, step = s / len;
        for (uint32_t i = 0; i < s; i += len) {
            for (uint32_t j = 0; j < half; j++) {
                int64_t wr, wi;
                fx_zeta(N, 4 * j * step, 1.0, &wr, &wi);
                cshare pr = cmul_share(A[i + j + half], wr, wi);
                u128 vr = trunc_share(pr.re, F, party), vi = trunc_share(pr.im, F, party);
                cshare u = A[i + j];
                A[i + j] = (cshare){u.re + vr, u.im + vi};
                A[i + j + half] = (cshare){u.re - vr, u.im - vi};
            }
        }
    }
    const uint64_t mask = (1ull << l) - 1;
    uint64_t g = 1;
    for (uint32_t j = 0; j < s; j++) {
        out[j] = (uint64_t)trunc_share(A[(g - 1) / 4].re, P - sf, party) & mask;
        g = (g * 5) % (2ull * N);
    }
    free(U);
    free(A);
    return 0;
}

/* MPC -> CKKS, what party b computes before encryption (Alg. 2 steps 1-2):
 * x holds its shares of n <= N/2 slot values in Z_{2^l} at the MPC scale
 * 2^-sf, wsh its share of the extension wrap bits.  Then
 *   1. extension to Z_{2^128} (signed), and a shift up to resolution 2^-P;
 *   2. V[k_j] = x_j (slots past n are 0), the inverse of the decoding's DFT
 *      as radix-2 decimation in time on bit-reversed input, each butterfly
 *      halved: (u 2^F +- v conj(omega^k)) / 2^(F+1), one truncation per output;
 *      the result is the inverse DFT divided by s;
 *   3. twist and scale: with Delta = mu 2^e, mu in [0.5, 1),
 *      c_t = A_t round(2^F mu zeta^-t) / 2^(P+F-e) (a shift left when negative),
 *      m_t = Re c_t and m_{t+s} = Im c_t, the shares of Encode(x) = round(Delta pi^-1(x));
 *   4. ring to field for q_0..q_level.
 * out receives (level+1) x N residues in coefficient form. */
int orc_m2c_local(const orc_params* p, uint32_t party, const uint64_t* x, const uint64_t* wsh, uint32_t n,
                  uint32_t level, double scale, uint32_t l, uint32_t sf, uint64_t* out)
{
    const uint32_t N = p->N, s = N / 2, logs = p->logN - 1;
    const uint32_t F = ORC_FX_F, P = ORC_FX_P;
    if (n > s || l > 62 || sf > P || l < sf + 2 || !(scale > 0) || level >= p->nQ) return -1;
    int ex;
    const double mu = frexp(scale, &ex); /* scale = mu 2^ex, mu in [0.5, 1) */
    const int sh = (int)(P + F) - ex;
    if (sh >= 64 || sh <= -64) return -1;
    uint64_t* X = malloc(sizeof(uint64_t) * 2 * (n ? n : 1));
    cshare* V = calloc(s, sizeof(cshare));
    cshare* A = malloc(sizeof(cshare) * s);
    uint64_t* M = malloc(sizeof(uint64_t) * 2 * N);
    orc_ext_local(party, n, l, x, wsh, X);
    uint64_t g = 1;
    for (uint32_t j = 0; j < s; j++) {
        if (j < n) V[(g - 1) / 4].re = ld128(X, j) << (P - sf);
        g = (g * 5) % (2ull * N);
    }
    for (uint32_t k = 0; k < s; k++) A[bitrev(k, logs)] = V[k];
    for (uint32_t len = 2; len <= s; len <<= 1) {
        const uint32_t half = len / 2, step = s / len;
        for (uint32_t i = 0; i < s; i += len) {
            for (uint32_t j = 0; j < half; j++) {
                int64_t wr, wi;
                fx_zeta(N, 4 * j * step, 1.0, &wr, &wi);
                cshare pr = cmul_share(A[i + j + half], wr, -wi);
                u128 ur = A[i + j].re << F, ui = A[i + j].im << F;
                A[i + j] = (cshare){trunc_share(ur + pr.re, F + 1, party), trunc_share(ui + pr.im, F + 1, party)};
                A[i + j + half] = (cshare){trunc_share(ur - pr.re, F + 1, party), trunc_share(ui - pr.im, F + 1, party)};
            }
        }
    }
    for (uint32_t k = 0; k < s; k++) {
        int64_t wr, wi;
        fx_zeta(N, k, mu, &wr, &wi);
        cshare c = cmul_share(A[k], wr, -wi);
        if (sh >= 0) {
            c.re = trunc_share(c.re, (uint32_t)sh, party);
            c.im = trunc_share(c.im, (uint32_t)sh, party);
        } else {
            c.re <<= (uint32_t)(-sh);
            c.im <<= (uint32_t)(-sh);
        }
        st128(M, k, c.re);
        st128(M, k + s, c.im);
    }
    orc_r2f_local(p, party, N, M, level, out);
    free(X);
    free(V);
    free(A);
    free(M);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* rotate-and-sum packing (Sec. 4.2.1) and the LayerNorm head it serves      */
/* ------------------------------------------------------------------------- */
/* Spatial-first packing puts block b (L consecutive slots) of a ciphertext at
 * slots [b L, (b+1) L).  m^0 = m, m^i = m^{i-1} + Rot^{2^{i-1} L}(m^{i-1}) for
 * i = 1..log2 D, with left rotations (dir = 0: sum) or right rotations
 * (dir = 1: broadcast); gk[i-1] is the Galois key of that rotation.  After the
 * last round block b holds the sum of blocks b, b+1, ..., b+D-1 (left) or
 * b, b-1, ..., b-D+1 (right), indices mod N/(2L).  With mask != 0 (the sum) the
 * result is multiplied by the plaintext [1 (L slots), 0, ...] encoded at scale
 * q_level and rescaled, so only block 0 remains and out is at level - 1. */
int orc_rs_packing(const orc_params* p, const uint64_t* ct, uint32_t level, uint32_t L, uint32_t D, int dir,
                   int mask, const uint64_t* const* gk, uint64_t* out)
{
    const uint32_t N = p->N, s = N / 2, n = level + 1;
    if (L == 0 || D == 0 || (D & (D - 1)) || (uint64_t)L * D > s || (mask && (dir || level == 0))) return -1;
    const size_t words = (size_t)2 * n * N;
    uint64_t* m = malloc(sizeof(uint64_t) * words);
    uint64_t* r = malloc(sizeof(uint64_t) * words);
    memcpy(m, ct, sizeof(uint64_t) * words);
    uint32_t i = 0;
    for (uint32_t step = 1; step < D; step <<= 1, i++) {
        int32_t amount = (int32_t)(step * L);
        orc_rotate(p, m, level, dir ? -amount : amount, gk[i], r);
        ct_add_inplace(p, m, r, level, 2);
    }
    if (mask) {
        double* z = calloc(s, sizeof(double));
        uint64_t* pt = malloc(sizeof(uint64_t) * (size_t)n * N);
        for (uint32_t j = 0; j < L; j++) z[j] = 1.0;
        orc_encode(p, z, s, level, (double)p->prime[level], pt);
        orc_mul_plain(p, m, pt, level, r);
        orc_rescale(p, r, level, 2, out);
        free(z);
        free(pt);
    } else {
        memcpy(out, m, sizeof(uint64_t) * words);
    }
    free(m);
    free(r);
    return 0;
}

/* ct * (the constant c in every slot, encoded at scale q_level), rescaled: the
 * scalar multiplications ewmul_cp(., 1/D) of the LayerNorm. */
static void mul_const_rescale(const orc_params* p, const uint64_t* ct, uint32_t level, double c, uint64_t* out)
{
    const uint32_t N = p->N, s = N / 2, n = level + 1;
    double* z = malloc(sizeof(double) * s);
    uint64_t* pt = malloc(sizeof(uint64_t) * (size_t)n * N);
    uint64_t* t = malloc(sizeof(uint64_t) * (size_t)2 * n * N);
    for (uint32_t j = 0; j < s; j++) z[j] = c;
    orc_encode(p, z, s, level, (double)p->prime[level], pt);
    orc_mul_plain(p, ct, pt, level, t);
    orc_rescale(p, t, level, 2, out);
    free(z);
    free(pt);
    free(t);
}

/* ct at level l -> the same ciphertext at level l - 1 (drop the last limb). */
static void drop_limb(const orc_params* p, const uint64_t* ct, uint32_t level, uint64_t* out)
{
    const uint32_t N = p->N, n = level + 1;
    for (uint32_t poly = 0; poly < 2; poly++)
        memcpy(out + (size_t)poly * level * N, ct + (size_t)poly * n * N, sizeof(uint64_t) * (size_t)level * N);
}

/* The HE steps of the secure LayerNorm before rsqrt (Alg. LayerNorm lines 1-6),
 * on X (L rows x D columns) packed spatial-first in nc ciphertexts of k = N/(2L)
 * columns each (k a power of two, nc = ceil(D/k)), at `level`:
 *   X_sum = sum_j X_ij: the nc ciphertexts added, then rotate-and-sum over the
 *           k blocks without the mask (the sum feeds a scalar operator, so every
 *           block keeping the row sum is the broadcast, Sec. 4.2.1);
 *   mu    = ewmul_cp(X_sum, 1/D)                              (level - 1)
 *   X_mu  = sadd_cc(X, -mu): each X_c dropped one level minus mu  (level - 1)
 *   X_mu^2 = ewmul_cc(X_mu, X_mu): tensor, relinearize, rescale  (level - 2)
 *   X_tmp = sum_j X_mu^2 as for X_sum;  var = ewmul_cp(X_tmp, 1/D) (level - 3).
 * Out: X_mu (nc ciphertexts, level - 1) and var (one ciphertext, level - 3,
 * every block holding the row variances); gk[i] is the key of rotation 2^i L. */
int orc_layernorm_head(const orc_params* p, const uint64_t* X, uint32_t nc, uint32_t level, uint32_t L, uint32_t D,
                       const uint64_t* const* gk, const uint64_t* relin_ksk, uint64_t* X_mu, uint64_t* var)
{
    const uint32_t N = p->N, s = N / 2;
    if (L == 0 || s % L || level < 3 || nc == 0) return -1;
    const uint32_t k = s / L;
    if (k & (k - 1)) return -1;
    const size_t w0 = (size_t)2 * (level + 1) * N, w1 = (size_t)2 * level * N, w2 = (size_t)2 * (level - 1) * N;
    uint64_t* acc = malloc(sizeof(uint64_t) * w0);
    uint64_t* tmp = malloc(sizeof(uint64_t) * w0);
    uint64_t* mu = malloc(sizeof(uint64_t) * w1);
    uint64_t* t3 = malloc(sizeof(uint64_t) * 3 * (size_t)level * N);
    uint64_t* sq = malloc(sizeof(uint64_t) * w1);
    uint64_t* acc2 = malloc(sizeof(uint64_t) * w2);
    uint64_t* tmp2 = malloc(sizeof(uint64_t) * w2);
    /* lines 1-2 */
    memcpy(acc, X, sizeof(uint64_t) * w0);
    for (uint32_t c = 1; c < nc; c++) ct_add_inplace(p, acc, X + c * w0, level, 2);
    orc_rs_packing(p, acc, level, L, k, 0, 0, gk, tmp);
    mul_const_rescale(p, tmp, level, 1.0 / (double)D, mu);
    /* lines 3-6 */
    for (uint32_t c = 0; c < nc; c++) {
        uint64_t* xm = X_mu + c * w1;
        drop_limb(p, X + c * w0, level, xm);
        for (uint32_t poly = 0; poly < 2; poly++)
            for (uint32_t l = 0; l < level; l++) {
                const uint64_t q = p->prime[l];
                for (uint32_t i = 0; i < N; i++) {
                    size_t o = ((size_t)poly * level + l) * N + i;
                    xm[o] = submod(xm[o], mu[o], q);
                }
            }
        orc_tensor(p, xm, xm, level - 1, t3);
        orc_relinearize(p, t3, level - 1, relin_ksk, sq);
        if (c == 0)
            orc_rescale(p, sq, level - 1, 2, acc2);
        else {
            orc_rescale(p, sq, level - 1, 2, tmp2);
            ct_add_inplace(p, acc2, tmp2, level - 2, 2);
        }
    }
    orc_rs_packing(p, acc2, level - 2, L, k, 0, 0, gk, tmp2);
    mul_const_rescale(p, tmp2, level - 2, 1.0 / (double)D, var);
    free(acc);
    free(tmp);
    free(mu);
    free(t3);
    free(sq);
    free(acc2);
    free(tmp2);
    return 0;
}
