/*
 * oracle.h -- plain, slow CPU oracle of the RNS-CKKS linear path of BLB
 * (arXiv 2508.19525): ciphertext-plaintext and ciphertext-ciphertext matrix
 * products (Sec. 5), the CKKS primitives beneath them (Sec. 2.4, Eq. 2), the
 * CKKS-to-MPC masking step (Alg. 1, Sec. 6.3) and the local steps of both
 * conversions between CKKS and additive shares (Alg. 1-2, App. C.3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this code; only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no source with the CUDA path: every
 * table, constant and transform here is computed by this file's own code.
 *
 * Representation: every polynomial is stored in COEFFICIENT form, limb-major,
 * as uint64 residues in [0, q).  A ciphertext at level l has l+1 limbs per
 * polynomial (primes q_0..q_l).  Products of polynomials go through this file's
 * own NTT (pinned against schoolbook negacyclic convolution by the tests).
 * Modular products are (unsigned __int128) a*b % q: slow and obviously right.
 */
#ifndef BLB_ORACLE_H
#define BLB_ORACLE_H
#include <stdint.h>

#define ORC_MAX_PRIMES 32

/* Sampling purposes (the fourth Philox counter word). */
enum { ORC_SECRET = 1, ORC_KEY_A = 2, ORC_KEY_E = 3, ORC_ENC_A = 4, ORC_ENC_E = 5, ORC_MASK = 6, ORC_WRAP = 7 };

/* Fixed point of the share FFTs of the conversions: roots carry ORC_FX_F
 * fraction bits, FFT data a resolution of 2^-ORC_FX_P slot units. */
#define ORC_FX_F 30
#define ORC_FX_P 26

typedef struct {
    uint32_t logN, N;
    uint32_t nQ, nP;      /* ciphertext primes q_0..q_{nQ-1}; special primes p_0..p_{nP-1} */
    uint32_t dnum, alpha; /* key-switching digits; alpha = ceil(nQ/dnum) primes per digit */
    uint64_t prime[ORC_MAX_PRIMES]; /* q_0..q_{nQ-1} then p_0..p_{nP-1} */
    uint64_t psi[ORC_MAX_PRIMES];   /* primitive 2N-th root of unity per prime */
} orc_params;

/* ---- arithmetic / parameters ---------------------------------------------- */
int      orc_is_prime(uint64_t n);
int      orc_params_init(orc_params* p, uint32_t logN, uint32_t nQ, uint32_t nP,
                         const uint32_t* q_bits, const uint32_t* p_bits, uint32_t dnum);
uint64_t orc_galois_elt(const orc_params* p, int32_t r);

/* ---- NTT: out[k] = a(psi^(2*bitrev(k)+1)) mod q, k in [N] ----------------- */
void orc_ntt(const orc_params* p, uint32_t prime_idx, uint64_t* a);
void orc_intt(const orc_params* p, uint32_t prime_idx, uint64_t* a);
void orc_negacyclic_mul(const orc_params* p, uint32_t prime_idx, const uint64_t* a,
                        const uint64_t* b, uint64_t* out);

/* ---- sampling (Philox4x32-10, Salmon et al. SC'11) ------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_cdt_table(uint64_t table[19]);
void orc_sample_ternary(uint32_t N, uint64_t seed, uint32_t obj, uint32_t purpose, uint32_t j,
                        int64_t* out);
void orc_sample_gauss(uint32_t N, uint64_t seed, uint32_t obj, uint32_t purpose, uint32_t j,
                      int64_t* out);
void orc_sample_uniform(uint32_t N, uint64_t q, uint64_t seed, uint32_t obj, uint32_t purpose,
                        uint32_t j, uint64_t* out);

/* ---- encode / decode (Eq. 2) ---------------------------------------------- */
int  orc_encode(const orc_params* p, const double* z, uint32_t n, uint32_t level, double scale,
                uint64_t* out /* (level+1) x N */);
int  orc_encode_int(const orc_params* p, const double* z, uint32_t n, double scale,
                    int64_t* out /* N signed coefficients */);
void orc_decode(const orc_params* p, const int64_t* coef, double scale, double* z /* N/2 */);

/* ---- keys ----------------------------------------------------------------- */
/* A key-switching key from s' to s: for digit j < dnum and limb t over all
 * nQ+nP primes, (b_j[t], a_j[t]) in coefficient form.  Layout:
 * [dnum][2][nQ+nP][N] with index 0 = b, 1 = a. */
uint64_t orc_ksk_words(const orc_params* p);
void orc_keygen_secret(const orc_params* p, uint64_t seed, int64_t* s /* N */);
void orc_keygen_ksk(const orc_params* p, uint64_t seed, const int64_t* s, const int64_t* s_prime,
                    uint32_t obj, uint64_t* ksk);
void orc_keygen_relin(const orc_params* p, uint64_t seed, const int64_t* s, uint64_t* ksk);
void orc_keygen_galois(const orc_params* p, uint64_t seed, const int64_t* s, uint64_t g,
                       uint64_t* ksk);

/* ---- ciphertext operations (all coefficient form) -------------------------- */
void orc_encrypt(const orc_params* p, const int64_t* s, const uint64_t* pt, uint32_t level,
                 uint64_t seed, uint32_t nonce, uint64_t* ct /* 2 x (level+1) x N */);
void orc_decrypt(const orc_params* p, const int64_t* s, const uint64_t* ct, uint32_t level,
                 uint32_t npolys, uint64_t* m /* (level+1) x N */);
void orc_automorphism(const orc_params* p, const uint64_t* in, uint32_t nlimbs, uint64_t g,
                      uint64_t* out);
void orc_moddown(const orc_params* p, const uint64_t* acc /* 2 x (level+1+nP) x N */, uint32_t level,
                 uint64_t* out /* 2 x (level+1) x N */);
void orc_modup(const orc_params* p, const uint64_t* d, uint32_t level,
               uint64_t* ext /* beta x (level+1+nP) x N */);
void orc_ks_accumulate(const orc_params* p, const uint64_t* ext, uint32_t level, uint64_t g,
                       const uint64_t* ksk, uint64_t* acc /* 2 x (level+1+nP) x N */);
void orc_keyswitch(const orc_params* p, const uint64_t* d, uint32_t level, const uint64_t* ksk,
                   uint64_t* out /* 2 x (level+1) x N */);
void orc_rotate(const orc_params* p, const uint64_t* ct, uint32_t level, int32_t r,
                const uint64_t* galois_ksk, uint64_t* out);
void orc_rotate_hoisted(const orc_params* p, const uint64_t* ct, uint32_t level, uint32_t k,
                        const int32_t* r, const uint64_t* const* galois_ksk,
                        uint64_t* out /* k x 2 x (level+1) x N */);
void orc_rotate_sum(const orc_params* p, const uint64_t* base /* nullable */, const uint64_t* T,
                    uint32_t level, uint32_t k, const int32_t* r, const uint64_t* const* galois_ksk,
                    uint64_t* out /* 2 x (level+1) x N */);
void orc_rescale(const orc_params* p, const uint64_t* ct, uint32_t level, uint32_t npolys,
                 uint64_t* out /* npolys x level x N */);
void orc_add(const orc_params* p, const uint64_t* a, const uint64_t* b, uint32_t nlimbs,
             uint64_t* out);
void orc_mul_plain(const orc_params* p, const uint64_t* ct, const uint64_t* pt, uint32_t level,
                   uint64_t* out);
void orc_tensor(const orc_params* p, const uint64_t* a, const uint64_t* b, uint32_t level,
                uint64_t* out /* 3 x (level+1) x N */);
void orc_relinearize(const orc_params* p, const uint64_t* ct3, uint32_t level,
                     const uint64_t* relin_ksk, uint64_t* out);

/* ---- protocols ------------------------------------------------------------ */
/* Rotation-key lookup for the protocol drivers: galois[i] is the key for
 * Galois element gal[i]. */
typedef struct {
    uint32_t n;
    const uint64_t* gal;
    const uint64_t* const* ksk;
} orc_galois_set;

uint32_t orc_cp_num_rotations(uint32_t nX, uint32_t nY, uint32_t b1, uint32_t G);
/* The two phases of orc_matmul_cp, for callers that encode the weights once:
 * baby steps baby[c][b] = Rot^{b m}(X_c) (nX x b1 ciphertexts, hoisted); the
 * plaintext diagonals of the outputs out_idx[0..n_out) ([n_out][G][nX][b1]
 * plaintexts at `level`, scale q_level); and the outputs from both (n_out
 * ciphertexts at level - 1, the same limbs as orc_matmul_cp). */
int orc_cp_baby_steps(const orc_params* p, const orc_galois_set* gk, const uint64_t* X, uint32_t nX,
                      uint32_t level, uint32_t m, uint32_t b1, uint64_t* baby);
int orc_cp_encode_diagonals(const orc_params* p, uint32_t level, uint32_t m, uint32_t d, const double* W,
                            uint32_t d_out, uint32_t b1, const uint32_t* out_idx, uint32_t n_out, uint64_t* pts);
int orc_cp_outputs(const orc_params* p, const orc_galois_set* gk, const uint64_t* baby, uint32_t nX,
                   uint32_t level, uint32_t m, uint32_t b1, const uint64_t* pts, uint32_t n_out, uint64_t* Y);
/* One inner sum of the giant steps: T = sum_c sum_b baby[c][b] (.) pts[c][b]
 * (nX x b1 plaintexts at `level`). */
int orc_cp_inner_sum(const orc_params* p, const uint64_t* baby, uint32_t nX, uint32_t level, uint32_t b1,
                     const uint64_t* pts, uint64_t* T);
int orc_matmul_cp(const orc_params* p, const orc_galois_set* gk, const uint64_t* X, uint32_t nX,
                  uint32_t level, uint32_t m, uint32_t d, const double* W, uint32_t d_out,
                  uint32_t b1, const uint32_t* out_idx, uint32_t n_out, uint64_t* Y);
/* Diagonal-input matmul_cp (App. C.2): X holds, per head group g (Hg[g] heads,
 * Kc = s/(L Hg[g])), the Dh/Kc dense-diagonal ciphertexts of Att_h (matmul_cc's
 * outputs j and j + Dh/Kc added; L = 2 Dh); W is (sum Hg) Dh x d_out.  Output
 * as orc_matmul_cp: spatial-first E = Concat_h(Att_h) W, level - 1. */
uint32_t orc_cp_diag_inputs(uint32_t s, uint32_t L, uint32_t n_groups, const uint32_t* Hg, uint32_t Dh);
int orc_matmul_cp_diag(const orc_params* p, const orc_galois_set* gk, const uint64_t* X, uint32_t level, uint32_t L,
                       uint32_t n_groups, const uint32_t* Hg, uint32_t Dh, const double* W, uint32_t d_out,
                       uint32_t b1, const uint32_t* out_idx, uint32_t n_out, uint64_t* Y);
uint32_t orc_cc_num_rotations(uint32_t n_c, uint32_t L, uint32_t Kc, uint32_t b1s1, uint32_t b1s2);
int orc_matmul_cc(const orc_params* p, const orc_galois_set* gk, const uint64_t* relin_ksk, const uint64_t* A,
                  const uint64_t* B, uint32_t n_c, uint32_t level, uint32_t L, uint32_t Hg, uint32_t b1s1,
                  uint32_t b1s2, uint64_t* C /* (L/Kc) x 2 x (level-3) x N */);
void orc_he2mpc(const orc_params* p, const uint64_t* ct, uint32_t level, uint64_t seed,
                uint32_t nonce, uint64_t* masked /* 2 x N */, uint64_t* p1_share /* N */);

/* ---- local parts of the CKKS <-> MPC conversions (Alg. 1 steps 3-4, Alg. 2,
 * App. C.3).  Extended-ring shares are 2 words (low, high) per element. ----- */
void orc_share_trunc(uint32_t party, const uint64_t* x, uint64_t n, uint32_t k, uint64_t* out);
void orc_f2r_wrap_sim(uint32_t n, uint64_t q, const uint64_t* t0, const uint64_t* t1, uint64_t seed,
                      uint32_t nonce, uint64_t* w0, uint64_t* w1);
void orc_f2r_local(uint32_t party, uint32_t n, uint64_t q, const uint64_t* t, const uint64_t* wsh, uint64_t* U);
void orc_ext_wrap_sim(uint32_t n, uint32_t l, const uint64_t* x0, const uint64_t* x1, uint64_t seed,
                      uint32_t nonce, uint64_t* w0, uint64_t* w1);
void orc_ext_local(uint32_t party, uint32_t n, uint32_t l, const uint64_t* x, const uint64_t* wsh, uint64_t* X);
void orc_r2f_local(const orc_params* p, uint32_t party, uint32_t n, const uint64_t* M, uint32_t level,
                   uint64_t* out);
int orc_c2m_local(const orc_params* p, uint32_t party, const uint64_t* t, const uint64_t* wsh, double scale,
                  uint32_t l, uint32_t sf, uint64_t* out /* N/2, mod 2^l */);
/* ---- rotate-and-sum packing (Sec. 4.2.1) and the LayerNorm head ---------- */
int orc_rs_packing(const orc_params* p, const uint64_t* ct, uint32_t level, uint32_t L, uint32_t D, int dir,
                   int mask, const uint64_t* const* gk, uint64_t* out);
int orc_layernorm_head(const orc_params* p, const uint64_t* X, uint32_t nc, uint32_t level, uint32_t L, uint32_t D,
                       const uint64_t* const* gk, const uint64_t* relin_ksk,
                       uint64_t* X_mu /* nc x 2 x level x N */, uint64_t* var /* 2 x (level-2) x N */);
int orc_m2c_local(const orc_params* p, uint32_t party, const uint64_t* x, const uint64_t* wsh, uint32_t n,
                  uint32_t level, double scale, uint32_t l, uint32_t sf, uint64_t* out /* (level+1) x N */);

#endif
