// capi.cu -- C ABI entry points: keys, encoding, encryption, homomorphic
// operations, matmul_cp (BSGS diagonal method) and the CKKS-to-MPC masking step.
//
// Operation scratch layout (rows of N words above the key-switch region):
//   [0, 3 nQ)        per-call temporaries (rotation, relinearization, rescale,
//                    encryption noise, decryption, export)
//   3 nQ             decoding FFT buffer (N/2 complex doubles)
//   3 nQ + 1         decoded slots (N/2 doubles)
//   3 nQ + 2         signed noise coefficients (N int64)
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"

// library-internal helpers (declared in common.cuh)
uint64_t* op_row(blb_ctx* c, size_t r) { return c->op_scratch() + r * c->N; }

bool capturing(blb_ctx* c)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(c->stream, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive;
}

int persist_upload(blb_ctx* c, const void* host, size_t bytes, void** dev)
{
    *dev = nullptr;
    if (!c->upload_stream) BLB_CUDA(cudaStreamCreateWithFlags(&c->upload_stream, cudaStreamNonBlocking));
    BLB_CUDA(cudaMalloc(dev, bytes ? bytes : 16));
    c->graph_keep.push_back({*dev, 0});
    if (bytes) {
        BLB_CUDA(cudaMemcpyAsync(*dev, host, bytes, cudaMemcpyHostToDevice, c->upload_stream));
        BLB_CUDA(cudaStreamSynchronize(c->upload_stream));
    }
    return BLB_OK;
}

void* Scratch::get(size_t bytes)
{
    bytes = std::max<size_t>(bytes, 16);
    void* p = dev_alloc(c, bytes);
    if (p) bufs.push_back({p, bytes});
    return p;
}
Scratch::~Scratch()
{
    for (auto& b : bufs) dev_free(c, b.first, b.second);
}

int host_upload(blb_ctx* c, void* dst, const void* src, size_t bytes)
{
    if (!bytes) return BLB_OK;
    if (!capturing(c)) {
        BLB_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
        return BLB_OK;
    }
    void* kept = nullptr;
    BLB_TRY(persist_upload(c, src, bytes, &kept));
    BLB_CUDA(cudaMemcpyAsync(dst, kept, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return BLB_OK;
}

int refuse_capture(blb_ctx* c, const char* what)
{
    if (!capturing(c)) return BLB_OK;
    return blb_fail(BLB_ERR_ARG, std::string(what) + " cannot run inside a graph capture");
}

int copy_in(blb_ctx* c, void* dst, const void* src, size_t bytes)
{
    const bool dev = is_device_ptr(src);
    if (!dev && capturing(c))
        return blb_fail(BLB_ERR_ARG, "host input buffer during graph capture: pass device memory");
    BLB_CUDA(cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    return BLB_OK;
}

int copy_out(blb_ctx* c, void* dst, const void* src, size_t bytes)
{
    bool dev = is_device_ptr(dst);
    if (!dev && capturing(c))
        return blb_fail(BLB_ERR_ARG, "host output buffer during graph capture: pass device memory");
    BLB_CUDA(cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!dev) BLB_CUDA(cudaStreamSynchronize(c->stream));
    return BLB_OK;
}

int new_ct(blb_ctx* c, uint32_t level, uint32_t npolys, double scale, blb_ct** out)
{
    blb_ct* ct = new blb_ct();
    ct->ctx = c;
    ct->level = level;
    ct->npolys = npolys;
    ct->scale = scale;
    ct->bytes = (size_t)npolys * (level + 1) * c->N * 8;
    ct->d = (uint64_t*)dev_alloc(c, ct->bytes);
    if (!ct->d) {
        delete ct;
        return blb_fail(BLB_ERR_OOM, "ciphertext allocation failed");
    }
    ctx_retain(c);
    *out = ct;
    return BLB_OK;
}

namespace {
constexpr int kT = 256;

bool same_scale(double a, double b) { return std::fabs(a - b) <= 1e-9 * std::max(std::fabs(a), std::fabs(b)); }

// left rotation of a 2-polynomial ciphertext buffer `in` at `level` into `out`
// (both n = level+1 limbs per polynomial); uses operation rows [0, 2n)
int rotate_into(blb_ctx* c, const blb_keys* keys, const uint64_t* in, uint32_t level, int32_t rot, uint64_t* out)
{
    const uint32_t n = level + 1, N = c->N;
    const uint64_t g = galois_element(N, rot);
    if (g == 1) {
        BLB_CUDA(cudaMemcpyAsync(out, in, (size_t)2 * n * N * 8, cudaMemcpyDeviceToDevice, c->stream));
        return BLB_OK;
    }
    const KeyEntry* k = keys->find(g);
    if (!k) return blb_fail(BLB_ERR_NO_KEY, "no Galois key for rotation " + std::to_string(rot));
    uint64_t* perm1 = op_row(c, 0);
    uint64_t* ks0 = op_row(c, n);
    BLB_TRY(launch_automorph_ntt(c, perm1, in + (size_t)n * N, n, g));
    BLB_TRY(keyswitch(c, perm1, level, k->d, ks0, out + (size_t)n * N));
    BLB_TRY(launch_automorph_ntt(c, out, in, n, g));
    BLB_TRY(launch_add_rows(c, out, out, ks0, n, c->qmap(n)));
    return BLB_OK;
}

// acc += rotate(in) (accumulating form used by the giant steps)
int rotate_add(blb_ctx* c, const blb_keys* keys, const uint64_t* in, uint32_t level, int32_t rot, uint64_t* acc)
{
    const uint32_t n = level + 1, N = c->N;
    const uint64_t g = galois_element(N, rot);
    const KeyEntry* k = keys->find(g);
    if (!k) return blb_fail(BLB_ERR_NO_KEY, "no Galois key for rotation " + std::to_string(rot));
    uint64_t* perm1 = op_row(c, 0);
    uint64_t* ks0 = op_row(c, n);
    uint64_t* ks1 = op_row(c, 2 * n);
    BLB_TRY(launch_automorph_ntt(c, perm1, in + (size_t)n * N, n, g));
    BLB_TRY(keyswitch(c, perm1, level, k->d, ks0, ks1));
    BLB_TRY(launch_add_rows(c, acc + (size_t)n * N, acc + (size_t)n * N, ks1, n, c->qmap(n)));
    BLB_TRY(launch_automorph_ntt(c, perm1, in, n, g));
    BLB_TRY(launch_add_rows(c, acc, acc, perm1, n, c->qmap(n)));
    BLB_TRY(launch_add_rows(c, acc, acc, ks0, n, c->qmap(n)));
    return BLB_OK;
}

// matmul_cp inner products for a batch of S sequences sharing one plan:
//   T[s][e][g] = sum_{c, b} baby[s][c][b] (.) pt[e][g][c][b].
// A CTA owns C coefficients of one limb: it stages the baby-step values of every
// sequence and term for those coefficients in shared memory once, then streams
// the plaintexts of every (e, g) through them; each plaintext word is read from
// HBM once and applied to all S sequences.  Lazy 128-bit sums folded every 8
// terms; the 8 plaintext loads of a group are issued together.
}  // namespace

int new_ciphertext(blb_ctx* c, uint32_t level, uint32_t npolys, double scale, blb_ct** out)
{
    return new_ct(c, level, npolys, scale, out);
}

// ===========================================================================
// keys
// ===========================================================================
extern "C" int blb_keygen(blb_ctx* c, uint64_t seed, const int32_t* rot_steps, uint32_t n_rot, int relin,
                          blb_keys** out)
{
    if (!c || !out || (n_rot && !rot_steps)) return blb_fail(BLB_ERR_ARG, "null argument");
    *out = nullptr;
    const uint32_t N = c->N, np = c->np;
    blb_keys* K = new blb_keys();
    K->ctx = c;
    ctx_retain(c);
    K->seed = seed;
    K->bytes = 0;
    const size_t poly_bytes = (size_t)np * N * 8;
    const size_t key_bytes = (size_t)c->dnum * 2 * poly_bytes;
    auto fail = [&](int rc) {
        std::string m = blb_last_error();
        blb_keys_free(K);
        blb_set_error(m);
        return rc;
    };
    K->d_s = (uint64_t*)dev_alloc(c, poly_bytes);
    K->d_s_coef = (int64_t*)dev_alloc(c, (size_t)N * 8);
    uint64_t* sp = (uint64_t*)dev_alloc(c, poly_bytes);
    uint64_t* erow = (uint64_t*)dev_alloc(c, poly_bytes);
    int64_t* ecoef = (int64_t*)dev_alloc(c, (size_t)N * 8);
    uint64_t* tmp = (uint64_t*)dev_alloc(c, poly_bytes);
    if (!K->d_s || !K->d_s_coef || !sp || !erow || !ecoef || !tmp) {
        dev_free(c, sp, poly_bytes);
        dev_free(c, erow, poly_bytes);
        dev_free(c, ecoef, (size_t)N * 8);
        dev_free(c, tmp, poly_bytes);
        blb_fail(BLB_ERR_OOM, "key allocation failed");
        return fail(BLB_ERR_OOM);
    }
    K->bytes += poly_bytes + (size_t)N * 8;
    int rc = BLB_OK;
    const LimbMap all = c->qmap(np);
    do {
        if ((rc = launch_sample_ternary(c, K->d_s_coef, seed, 0, PURPOSE_SECRET, 0))) break;
        if ((rc = launch_signed_to_rows(c, K->d_s, K->d_s_coef, np, all))) break;
        if ((rc = ntt_forward(c, K->d_s, np, all))) break;
        std::vector<uint64_t> gals;
        if (relin) gals.push_back(0);
        for (uint32_t r = 0; r < n_rot; r++) {
            uint64_t g = galois_element(N, rot_steps[r]);
            if (g == 1) continue;
            if (std::find(gals.begin(), gals.end(), g) == gals.end()) gals.push_back(g);
        }
        std::vector<uint32_t> jrow(np);
        for (uint64_t g : gals) {
            uint64_t* kd = (uint64_t*)dev_alloc(c, key_bytes);
            if (!kd) {
                rc = blb_fail(BLB_ERR_OOM, "switching key allocation failed");
                break;
            }
            K->keys.push_back({g, kd});
            K->bytes += key_bytes;
            const uint32_t obj = (uint32_t)g;
            if (g == 0) rc = launch_mul_rows(c, sp, K->d_s, K->d_s, np, all, np);  // s^2
            else rc = launch_automorph_ntt(c, sp, K->d_s, np, g);                   // sigma_g(s)
            if (rc) break;
            for (uint32_t j = 0; j < c->dnum && !rc; j++) {
                uint64_t* B = kd + (size_t)(2 * j) * np * N;
                uint64_t* A = kd + (size_t)(2 * j + 1) * np * N;
                for (uint32_t t = 0; t < np; t++) jrow[t] = 64 * j + t;
                if ((rc = launch_sample_uniform(c, A, np, all, seed, obj, PURPOSE_KEY_A, jrow.data()))) break;
                if ((rc = ntt_forward(c, A, np, all))) break;
                if ((rc = launch_sample_gauss(c, ecoef, seed, obj, PURPOSE_KEY_E, j))) break;
                if ((rc = launch_signed_to_rows(c, erow, ecoef, np, all))) break;
                if ((rc = ntt_forward(c, erow, np, all))) break;
                if ((rc = launch_mul_rows(c, B, A, K->d_s, np, all, np))) break;
                if ((rc = launch_neg_rows(c, B, B, np, all))) break;
                if ((rc = launch_add_rows(c, B, B, erow, np, all))) break;
                const uint32_t lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, c->nQ);
                if (lo < hi) {
                    std::vector<uint64_t> pm(c->P_mod_q.begin() + lo, c->P_mod_q.begin() + hi);
                    LimbMap dm = c->qmap(hi - lo, lo);
                    if ((rc = launch_mul_const_rows(c, tmp, sp + (size_t)lo * N, hi - lo, dm, pm.data()))) break;
                    if ((rc = launch_add_rows(c, B + (size_t)lo * N, B + (size_t)lo * N, tmp, hi - lo, dm))) break;
                }
            }
            if (rc) break;
        }
    } while (0);
    cudaStreamSynchronize(c->stream);
    dev_free(c, sp, poly_bytes);
    dev_free(c, erow, poly_bytes);
    dev_free(c, ecoef, (size_t)N * 8);
    dev_free(c, tmp, poly_bytes);
    if (rc) return fail(rc);
    *out = K;
    return BLB_OK;
}

extern "C" void blb_keys_free(blb_keys* K)
{
    if (!K) return;
    blb_ctx* c = K->ctx;
    const size_t poly_bytes = (size_t)c->np * c->N * 8;
    dev_free(c, K->d_s, poly_bytes);
    dev_free(c, K->d_s_coef, (size_t)c->N * 8);
    for (auto& k : K->keys) dev_free(c, k.d, (size_t)c->dnum * 2 * poly_bytes);
    delete K;
    ctx_release(c);
}

extern "C" int blb_keys_export(blb_ctx* c, const blb_keys* K, int which, int32_t rot, void* host_out)
{
    if (!c || !K || !host_out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (which == 0) return copy_out(c, host_out, K->d_s_coef, (size_t)c->N * 8);
    uint64_t g = which == 1 ? 0 : galois_element(c->N, rot);
    const KeyEntry* k = K->find(g);
    if (!k) return blb_fail(BLB_ERR_NO_KEY, "key not present");
    const size_t rows = (size_t)c->dnum * 2 * c->np, bytes = rows * c->N * 8;
    uint64_t* tmp = (uint64_t*)dev_alloc(c, bytes);
    if (!tmp) return blb_fail(BLB_ERR_OOM, "export buffer allocation failed");
    int rc = BLB_OK;
    if (cudaMemcpyAsync(tmp, k->d, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        rc = blb_fail(BLB_ERR_CUDA, "copy failed");
    if (!rc) rc = ntt_inverse(c, tmp, (uint32_t)rows, c->qmap(c->np));
    if (!rc) rc = copy_out(c, host_out, tmp, bytes);
    cudaStreamSynchronize(c->stream);
    dev_free(c, tmp, bytes);
    return rc;
}

// ===========================================================================
// encode / plaintexts
// ===========================================================================
extern "C" int blb_encode(blb_ctx* c, const double* vals, uint64_t n, uint32_t level, double scale, blb_pt** out)
{
    if (!c || !out || (n && !vals)) return blb_fail(BLB_ERR_ARG, "null argument");
    if (level >= c->nQ) return blb_fail(BLB_ERR_LEVEL, "level out of range");
    if (n > c->N / 2) return blb_fail(BLB_ERR_ARG, "more values than slots");
    if (!(scale > 0)) return blb_fail(BLB_ERR_ARG, "scale must be positive");
    blb_pt* pt = new blb_pt();
    pt->ctx = c;
    ctx_retain(c);
    pt->level = level;
    pt->scale = scale;
    pt->bytes = (size_t)(level + 1) * c->N * 8;
    pt->d = (uint64_t*)dev_alloc(c, pt->bytes);
    double* dz = (double*)op_row(c, 3 * (size_t)c->nQ + 1);
    int rc = pt->d ? BLB_OK : blb_fail(BLB_ERR_OOM, "plaintext allocation failed");
    if (!rc && n) rc = copy_in(c, dz, vals, n * 8);
    if (!rc) rc = encode_slots(c, dz, 1, (uint32_t)n, level, scale, pt->d);
    if (rc) {
        blb_pt_free(pt);
        return rc;
    }
    *out = pt;
    return BLB_OK;
}

extern "C" void blb_pt_free(blb_pt* pt)
{
    if (!pt) return;
    blb_ctx* c = pt->ctx;
    dev_free(c, pt->d, pt->bytes);
    delete pt;
    ctx_release(c);
}

extern "C" int blb_pt_export(blb_ctx* c, const blb_pt* pt, uint64_t* out)
{
    if (!c || !pt || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    const uint32_t n = pt->level + 1;
    uint64_t* tmp = op_row(c, 0);
    BLB_CUDA(cudaMemcpyAsync(tmp, pt->d, pt->bytes, cudaMemcpyDeviceToDevice, c->stream));
    BLB_TRY(ntt_inverse(c, tmp, n, c->qmap(n)));
    return copy_out(c, out, tmp, pt->bytes);
}

extern "C" int blb_pt_import(blb_ctx* c, const uint64_t* coeffs, uint32_t level, double scale, blb_pt** out)
{
    if (!c || !coeffs || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (level >= c->nQ) return blb_fail(BLB_ERR_LEVEL, "level out of range");
    if (!(scale > 0)) return blb_fail(BLB_ERR_ARG, "scale must be positive");
    blb_pt* pt = new blb_pt();
    pt->ctx = c;
    ctx_retain(c);
    pt->level = level;
    pt->scale = scale;
    pt->bytes = (size_t)(level + 1) * c->N * 8;
    pt->d = (uint64_t*)dev_alloc(c, pt->bytes);
    int rc = pt->d ? BLB_OK : blb_fail(BLB_ERR_OOM, "plaintext allocation failed");
    if (!rc) rc = copy_in(c, pt->d, coeffs, pt->bytes);
    if (!rc) rc = ntt_forward(c, pt->d, level + 1, c->qmap(level + 1));
    if (rc) {
        blb_pt_free(pt);
        return rc;
    }
    *out = pt;
    return BLB_OK;
}

// ===========================================================================
// ciphertexts
// ===========================================================================
extern "C" int blb_encrypt(blb_ctx* c, const blb_keys* K, const blb_pt* pt, uint64_t nonce, blb_ct** out)
{
    if (!c || !K || !pt || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    const uint32_t n = pt->level + 1, N = c->N;
    blb_ct* ct;
    BLB_TRY(new_ct(c, pt->level, 2, pt->scale, &ct));
    uint64_t* c0 = ct->d;
    uint64_t* c1 = ct->d + (size_t)n * N;
    uint64_t* erow = op_row(c, 0);
    int64_t* ecoef = (int64_t*)op_row(c, 3 * (size_t)c->nQ + 2);
    const LimbMap qm = c->qmap(n);
    std::vector<uint32_t> jrow(n);
    for (uint32_t i = 0; i < n; i++) jrow[i] = i;
    int rc = BLB_OK;
    do {
        if ((rc = launch_sample_uniform(c, c1, n, qm, K->seed, (uint32_t)nonce, PURPOSE_ENC_A, jrow.data()))) break;
        if ((rc = ntt_forward(c, c1, n, qm))) break;
        if ((rc = launch_sample_gauss(c, ecoef, K->seed, (uint32_t)nonce, PURPOSE_ENC_E, 0))) break;
        if ((rc = launch_signed_to_rows(c, erow, ecoef, n, qm))) break;
        if ((rc = ntt_forward(c, erow, n, qm))) break;
        if ((rc = launch_mul_rows(c, c0, c1, K->d_s, n, qm, c->np))) break;
        if ((rc = launch_neg_rows(c, c0, c0, n, qm))) break;
        if ((rc = launch_add_rows(c, c0, c0, pt->d, n, qm))) break;
        if ((rc = launch_add_rows(c, c0, c0, erow, n, qm))) break;
    } while (0);
    if (rc) {
        blb_ct_free(ct);
        return rc;
    }
    *out = ct;
    return BLB_OK;
}

extern "C" void blb_ct_free(blb_ct* ct)
{
    if (!ct) return;
    blb_ctx* c = ct->ctx;
    dev_free(c, ct->d, ct->bytes);
    delete ct;
    ctx_release(c);
}

extern "C" int blb_ct_info(const blb_ct* ct, uint32_t* level, uint32_t* npolys, double* scale)
{
    if (!ct) return blb_fail(BLB_ERR_ARG, "null ciphertext");
    if (level) *level = ct->level;
    if (npolys) *npolys = ct->npolys;
    if (scale) *scale = ct->scale;
    return BLB_OK;
}

extern "C" int blb_ct_export(blb_ctx* c, const blb_ct* ct, uint64_t* out)
{
    if (!c || !ct || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    const uint32_t n = ct->level + 1;
    uint64_t* tmp = op_row(c, 0);
    BLB_CUDA(cudaMemcpyAsync(tmp, ct->d, ct->bytes, cudaMemcpyDeviceToDevice, c->stream));
    BLB_TRY(ntt_inverse(c, tmp, ct->npolys * n, c->qmap(n)));
    return copy_out(c, out, tmp, ct->bytes);
}

extern "C" int blb_ct_import(blb_ctx* c, const uint64_t* coeffs, uint32_t level, uint32_t npolys, double scale,
                             blb_ct** out)
{
    if (!c || !coeffs || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (level >= c->nQ || npolys < 1 || npolys > 3) return blb_fail(BLB_ERR_ARG, "bad level or polynomial count");
    blb_ct* ct;
    BLB_TRY(new_ct(c, level, npolys, scale, &ct));
    int rc = copy_in(c, ct->d, coeffs, ct->bytes);
    if (!rc) rc = ntt_forward(c, ct->d, npolys * (level + 1), c->qmap(level + 1));
    if (rc) {
        blb_ct_free(ct);
        return rc;
    }
    *out = ct;
    return BLB_OK;
}

extern "C" int blb_decrypt(blb_ctx* c, const blb_keys* K, const blb_ct* ct, uint64_t* coeff_limbs, double* slots)
{
    if (!c || !K || !ct) return blb_fail(BLB_ERR_ARG, "null argument");
    const uint32_t n = ct->level + 1, N = c->N;
    const LimbMap qm = c->qmap(n);
    uint64_t* h = op_row(c, 0);
    // Horner: h = c_{np-1}; h = h s + c_k
    BLB_CUDA(cudaMemcpyAsync(h, ct->d + (size_t)(ct->npolys - 1) * n * N, (size_t)n * N * 8,
                             cudaMemcpyDeviceToDevice, c->stream));
    for (int k = (int)ct->npolys - 2; k >= 0; k--) {
        BLB_TRY(launch_mul_rows(c, h, h, K->d_s, n, qm, c->np));
        BLB_TRY(launch_add_rows(c, h, h, ct->d + (size_t)k * n * N, n, qm));
    }
    BLB_TRY(ntt_inverse(c, h, n, qm));
    if (coeff_limbs) BLB_TRY(copy_out(c, coeff_limbs, h, (size_t)n * N * 8));
    if (slots) {
        double* dz = (double*)op_row(c, 3 * (size_t)c->nQ + 1);
        BLB_TRY(decode_limb0(c, h, ct->scale, dz));
        BLB_TRY(copy_out(c, slots, dz, (size_t)N / 2 * 8));
    }
    return BLB_OK;
}

// ===========================================================================
// homomorphic operations
// ===========================================================================
extern "C" int blb_rotate(blb_ctx* c, const blb_keys* K, const blb_ct* in, int32_t steps, blb_ct** out)
{
    if (!c || !K || !in || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (in->npolys != 2) return blb_fail(BLB_ERR_ARG, "rotate needs a 2-polynomial ciphertext");
    blb_ct* r;
    BLB_TRY(new_ct(c, in->level, 2, in->scale, &r));
    int rc = rotate_into(c, K, in->d, in->level, steps, r->d);
    if (rc) {
        blb_ct_free(r);
        return rc;
    }
    *out = r;
    return BLB_OK;
}

extern "C" int blb_rescale(blb_ctx* c, blb_ct* ct)
{
    if (!c || !ct) return blb_fail(BLB_ERR_ARG, "null argument");
    if (ct->level == 0) return blb_fail(BLB_ERR_LEVEL, "rescale at level 0");
    const size_t bytes = (size_t)ct->npolys * ct->level * c->N * 8;
    uint64_t* o = (uint64_t*)dev_alloc(c, bytes);
    if (!o) return blb_fail(BLB_ERR_OOM, "rescale allocation failed");
    int rc = launch_rescale(c, o, ct->d, ct->level, ct->npolys);
    if (rc) {
        dev_free(c, o, bytes);
        return rc;
    }
    dev_free(c, ct->d, ct->bytes);
    ct->d = o;
    ct->bytes = bytes;
    ct->scale /= (double)c->q[ct->level];
    ct->level -= 1;
    return BLB_OK;
}

extern "C" int blb_ct_copy(blb_ctx* c, blb_ct* dst, const blb_ct* src)
{
    if (!c || !dst || !src) return blb_fail(BLB_ERR_ARG, "null argument");
    if (dst->level != src->level || dst->npolys != src->npolys)
        return blb_fail(BLB_ERR_ARG, "copy needs ciphertexts of one level and size");
    BLB_CUDA(cudaMemcpyAsync(dst->d, src->d, src->bytes, cudaMemcpyDeviceToDevice, c->stream));
    dst->scale = src->scale;
    return BLB_OK;
}

extern "C" int blb_add(blb_ctx* c, const blb_ct* a, const blb_ct* b, blb_ct** out)
{
    if (!c || !a || !b || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (a->level != b->level || a->npolys != b->npolys) return blb_fail(BLB_ERR_ARG, "level or size mismatch");
    if (!same_scale(a->scale, b->scale)) return blb_fail(BLB_ERR_SCALE, "operands have different scales");
    blb_ct* r;
    BLB_TRY(new_ct(c, a->level, a->npolys, a->scale, &r));
    int rc = launch_add_rows(c, r->d, a->d, b->d, a->npolys * (a->level + 1), c->qmap(a->level + 1));
    if (rc) {
        blb_ct_free(r);
        return rc;
    }
    *out = r;
    return BLB_OK;
}

extern "C" int blb_add_plain(blb_ctx* c, const blb_ct* a, const blb_pt* p, blb_ct** out)
{
    if (!c || !a || !p || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (p->level < a->level) return blb_fail(BLB_ERR_LEVEL, "plaintext below the ciphertext's level");
    if (!same_scale(a->scale, p->scale)) return blb_fail(BLB_ERR_SCALE, "operands have different scales");
    const uint32_t n = a->level + 1;
    blb_ct* r;
    BLB_TRY(new_ct(c, a->level, a->npolys, a->scale, &r));
    const size_t poly = (size_t)n * c->N;
    int rc = launch_add_rows(c, r->d, a->d, p->d, n, c->qmap(n));
    if (!rc && a->npolys > 1)
        rc = cudaMemcpyAsync(r->d + poly, a->d + poly, (a->npolys - 1) * poly * 8, cudaMemcpyDeviceToDevice,
                             c->stream) == cudaSuccess
                 ? BLB_OK
                 : blb_fail(BLB_ERR_CUDA, "copy of the remaining polynomials failed");
    if (rc) {
        blb_ct_free(r);
        return rc;
    }
    *out = r;
    return BLB_OK;
}

extern "C" int blb_sub(blb_ctx* c, const blb_ct* a, const blb_ct* b, blb_ct** out)
{
    if (!c || !a || !b || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (a->level != b->level || a->npolys != b->npolys) return blb_fail(BLB_ERR_ARG, "level or size mismatch");
    if (!same_scale(a->scale, b->scale)) return blb_fail(BLB_ERR_SCALE, "operands have different scales");
    blb_ct* r;
    BLB_TRY(new_ct(c, a->level, a->npolys, a->scale, &r));
    int rc = launch_sub_rows(c, r->d, a->d, b->d, a->npolys * (a->level + 1), c->qmap(a->level + 1));
    if (rc) {
        blb_ct_free(r);
        return rc;
    }
    *out = r;
    return BLB_OK;
}

extern "C" int blb_drop_level(blb_ctx* c, const blb_ct* a, uint32_t level, blb_ct** out)
{
    if (!c || !a || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (level > a->level) return blb_fail(BLB_ERR_LEVEL, "cannot raise a ciphertext's level");
    blb_ct* r;
    BLB_TRY(new_ct(c, level, a->npolys, a->scale, &r));
    const size_t N = c->N, n_in = a->level + 1, n_out = level + 1;
    for (uint32_t p = 0; p < a->npolys; p++)
        if (cudaMemcpyAsync(r->d + p * n_out * N, a->d + p * n_in * N, n_out * N * 8, cudaMemcpyDeviceToDevice,
                            c->stream) != cudaSuccess) {
            blb_ct_free(r);
            return blb_fail(BLB_ERR_CUDA, "copy failed");
        }
    *out = r;
    return BLB_OK;
}

extern "C" int blb_mul_const(blb_ctx* c, const blb_ct* a, const double* vals, uint64_t n, double target_scale,
                             blb_ct** out)
{
    if (!c || !a || !out || (n && !vals)) return blb_fail(BLB_ERR_ARG, "null argument");
    if (a->level == 0) return blb_fail(BLB_ERR_LEVEL, "no level left to rescale");
    if (a->npolys != 2) return blb_fail(BLB_ERR_ARG, "mul_const needs a 2-polynomial ciphertext");
    if (n > c->N / 2 || n == 0) return blb_fail(BLB_ERR_ARG, "1 to N/2 values");
    if (!(target_scale > 0)) return blb_fail(BLB_ERR_ARG, "target scale must be positive");
    const uint32_t lv = a->level, nl = lv + 1, N = c->N;
    // the constant's scale makes (scale_a x s_c) / q_level equal the target
    const double s_c = target_scale * (double)c->q[lv] / a->scale;
    Scratch S(c);
    const uint32_t s = N / 2;
    std::vector<double> z(s);
    for (uint32_t j = 0; j < s; j++) z[j] = vals[n == 1 ? 0 : (j < n ? j : 0)] * (n == 1 || j < n ? 1.0 : 0.0);
    double* dz = (double*)S.get((size_t)s * 8);
    uint64_t* pt = (uint64_t*)S.get((size_t)nl * N * 8);
    uint64_t* prod = (uint64_t*)S.get((size_t)2 * nl * N * 8);
    if (!dz || !pt || !prod) return blb_fail(BLB_ERR_OOM, "mul_const buffers");
    BLB_TRY(host_upload(c, dz, z.data(), (size_t)s * 8));
    BLB_TRY(encode_slots(c, dz, 1, s, lv, s_c, pt));
    BLB_TRY(launch_mul_rows(c, prod, a->d, pt, 2 * nl, c->qmap(nl), nl));
    blb_ct* r;
    BLB_TRY(new_ct(c, lv - 1, 2, target_scale, &r));
    int rc = launch_rescale_stack(c, r->d, prod, lv, 2);
    if (!rc) rc = cudaStreamSynchronize(c->stream) == cudaSuccess ? BLB_OK : blb_fail(BLB_ERR_CUDA, "sync failed");
    if (rc) {
        blb_ct_free(r);
        return rc;
    }
    *out = r;
    return BLB_OK;
}

extern "C" int blb_mul_plain(blb_ctx* c, const blb_ct* a, const blb_pt* p, blb_ct** out)
{
    if (!c || !a || !p || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (p->level < a->level) return blb_fail(BLB_ERR_LEVEL, "plaintext below the ciphertext's level");
    const uint32_t n = a->level + 1;
    blb_ct* r;
    BLB_TRY(new_ct(c, a->level, a->npolys, a->scale * p->scale, &r));
    int rc = launch_mul_rows(c, r->d, a->d, p->d, a->npolys * n, c->qmap(n), n);
    if (rc) {
        blb_ct_free(r);
        return rc;
    }
    *out = r;
    return BLB_OK;
}

static int relin_into(blb_ctx* c, const blb_keys* K, const uint64_t* ct3, uint32_t level, uint64_t* out)
{
    const uint32_t n = level + 1, N = c->N;
    const KeyEntry* k = K->find(0);
    if (!k) return blb_fail(BLB_ERR_NO_KEY, "no relinearization key");
    uint64_t* k0 = op_row(c, 0);
    uint64_t* k1 = op_row(c, n);
    BLB_TRY(keyswitch(c, ct3 + (size_t)2 * n * N, level, k->d, k0, k1));
    BLB_TRY(launch_add_rows(c, out, ct3, k0, n, c->qmap(n)));
    BLB_TRY(launch_add_rows(c, out + (size_t)n * N, ct3 + (size_t)n * N, k1, n, c->qmap(n)));
    return BLB_OK;
}

extern "C" int blb_relinearize(blb_ctx* c, const blb_keys* K, const blb_ct* in, blb_ct** out)
{
    if (!c || !K || !in || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (in->npolys != 3) return blb_fail(BLB_ERR_ARG, "relinearize needs a 3-polynomial ciphertext");
    blb_ct* r;
    BLB_TRY(new_ct(c, in->level, 2, in->scale, &r));
    int rc = relin_into(c, K, in->d, in->level, r->d);
    if (rc) {
        blb_ct_free(r);
        return rc;
    }
    *out = r;
    return BLB_OK;
}

extern "C" int blb_mul(blb_ctx* c, const blb_keys* K, const blb_ct* a, const blb_ct* b, int relin, blb_ct** out)
{
    if (!c || !a || !b || !out || (relin && !K)) return blb_fail(BLB_ERR_ARG, "null argument");
    if (a->level != b->level || a->npolys != 2 || b->npolys != 2)
        return blb_fail(BLB_ERR_ARG, "operands must be 2-polynomial ciphertexts at one level");
    blb_ct* t;
    BLB_TRY(new_ct(c, a->level, 3, a->scale * b->scale, &t));
    int rc = launch_tensor(c, t->d, a->d, b->d, a->level);
    if (rc || !relin) {
        if (rc) blb_ct_free(t);
        else *out = t;
        return rc;
    }
    blb_ct* r = nullptr;
    rc = new_ct(c, a->level, 2, t->scale, &r);
    if (!rc) rc = relin_into(c, K, t->d, a->level, r->d);
    blb_ct_free(t);
    if (rc) {
        blb_ct_free(r);
        return rc;
    }
    *out = r;
    return BLB_OK;
}

extern "C" int blb_keyswitch_coeffs(blb_ctx* c, const blb_keys* K, int32_t rot, const uint64_t* d, uint32_t level,
                                    uint64_t* out)
{
    if (!c || !K || !d || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    if (level >= c->nQ) return blb_fail(BLB_ERR_LEVEL, "level out of range");
    const KeyEntry* k = K->find(galois_element(c->N, rot));
    if (!k) return blb_fail(BLB_ERR_NO_KEY, "no Galois key for that rotation");
    const uint32_t n = level + 1, N = c->N;
    uint64_t* dd = op_row(c, 0);
    uint64_t* o = op_row(c, n);
    BLB_TRY(copy_in(c, dd, d, (size_t)n * N * 8));
    BLB_TRY(ntt_forward(c, dd, n, c->qmap(n)));
    BLB_TRY(keyswitch(c, dd, level, k->d, o, o + (size_t)n * N));
    BLB_TRY(ntt_inverse(c, o, 2 * n, c->qmap(n)));
    return copy_out(c, out, o, (size_t)2 * n * N * 8);
}

// ===========================================================================
// matmul_cp
// ===========================================================================
// diag: optional per-input-column (head, diagonal) of a diagonal-packed input
// (head -1 = unused column) and the head dimension; nX then comes from it
struct DiagLayout {
    std::vector<int32_t> head, delta;
    uint32_t Dh, nX;
};

static int cp_plan_build(blb_ctx* c, uint32_t m, uint32_t d, const double* W, uint32_t d_out, uint32_t level,
                         const blb_sched* sched, const DiagLayout* diag, blb_cp_plan** out)
{
    if (!c || !W || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    *out = nullptr;
    const uint32_t s = c->N / 2;
    if (m == 0 || s % m) return blb_fail(BLB_ERR_ARG, "m must divide N/2");
    if (d == 0 || d_out == 0) return blb_fail(BLB_ERR_ARG, "empty matrix");
    if (level < 1 || level >= c->nQ) return blb_fail(BLB_ERR_LEVEL, "matmul_cp needs a level to rescale into");
    const uint32_t k = s / m;
    uint32_t b1 = sched ? sched->b1 : 0;
    if (b1 == 0) {
        b1 = 1;
        while (b1 * b1 < k) b1 <<= 1;
    }
    if (b1 > k || k % b1) return blb_fail(BLB_ERR_ARG, "b1 must divide k = N/2/m");
    blb_cp_plan* P = new blb_cp_plan();
    P->ctx = c;
    ctx_retain(c);
    P->m = m;
    P->d = d;
    P->d_out = d_out;
    P->level = level;
    P->k = k;
    P->nX = diag ? diag->nX : (d + k - 1) / k;
    P->nY = (d_out + k - 1) / k;
    P->b1 = b1;
    P->G = k / b1;
    const uint32_t n = level + 1;
    const uint32_t terms = P->nX * P->b1, neg = P->nY * P->G;
    P->d_ptb = nullptr;
    int lrc = cp_plan_layout(c, P);
    if (lrc) {
        blb_cp_plan_free(P);
        return lrc;
    }
    P->d_ptb = (uint8_t*)dev_alloc(c, P->bytes);
    if (!P->d_ptb) {
        blb_cp_plan_free(P);
        return blb_fail(BLB_ERR_OOM, "plaintext diagonals do not fit");
    }
    const size_t wbytes = (size_t)d * d_out * 8;
    const double* dW = W;
    double* Wcopy = nullptr;
    int rc = BLB_OK;
    if (!is_device_ptr(W)) {
        Wcopy = (double*)dev_alloc(c, wbytes);
        if (!Wcopy) rc = blb_fail(BLB_ERR_OOM, "weight upload buffer");
        else if (cudaMemcpyAsync(Wcopy, W, wbytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            rc = blb_fail(BLB_ERR_CUDA, "weight upload failed");
        dW = Wcopy;
    }
    // one block of 16 outputs (e, g) at a time: encode its plaintexts, then
    // slice them into the byte layout of the tensor-core product
    const uint64_t blk_pts = (uint64_t)16 * terms;
    const size_t blk_bytes = blk_pts * n * c->N * 8;
    int32_t* d_head = nullptr;
    int32_t* d_delta = nullptr;
    const size_t lbytes = diag ? diag->head.size() * 4 : 0;
    if (!rc && diag) {
        d_head = (int32_t*)dev_alloc(c, lbytes);
        d_delta = (int32_t*)dev_alloc(c, lbytes);
        if (!d_head || !d_delta) rc = blb_fail(BLB_ERR_OOM, "diagonal layout");
        else if (cudaMemcpyAsync(d_head, diag->head.data(), lbytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
                 cudaMemcpyAsync(d_delta, diag->delta.data(), lbytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            rc = blb_fail(BLB_ERR_CUDA, "layout upload failed");
    }
    const uint32_t chunk = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(blk_pts, (64ull << 20) / ((uint64_t)s * 8)));
    double* z = rc ? nullptr : (double*)dev_alloc(c, (size_t)chunk * s * 8);
    uint64_t* blk = rc ? nullptr : (uint64_t*)dev_alloc(c, blk_bytes);
    if (!rc && (!z || !blk)) rc = blb_fail(BLB_ERR_OOM, "diagonal buffer");
    for (uint32_t eb = 0; !rc && eb < P->NEB; eb++) {
        const uint64_t first = (uint64_t)eb * blk_pts, npts = (uint64_t)std::min<uint32_t>(16, neg - eb * 16) * terms;
        for (uint64_t f = 0; !rc && f < npts; f += chunk) {
            uint32_t cnt = (uint32_t)std::min<uint64_t>(chunk, npts - f);
            rc = cp_build_diagonals(c, P, dW, (uint32_t)(first + f), cnt, z, d_head, d_delta, diag ? diag->Dh : 0);
            if (!rc) rc = encode_slots(c, z, cnt, s, level, (double)c->q[level], blk + f * n * c->N);
        }
        if (!rc) rc = cp_plan_store_block(c, P, blk, eb);
    }
    cudaStreamSynchronize(c->stream);
    dev_free(c, z, (size_t)chunk * s * 8);
    dev_free(c, blk, blk_bytes);
    dev_free(c, Wcopy, wbytes);
    dev_free(c, d_head, lbytes);
    dev_free(c, d_delta, lbytes);
    if (rc) {
        blb_cp_plan_free(P);
        return rc;
    }
    *out = P;
    return BLB_OK;
}

extern "C" int blb_cp_plan_create(blb_ctx* c, uint32_t m, uint32_t d, const double* W, uint32_t d_out,
                                  uint32_t level, const blb_sched* sched, blb_cp_plan** out)
{
    if (c) BLB_TRY(refuse_capture(c, "plan creation"));
    return cp_plan_build(c, m, d, W, d_out, level, sched, nullptr, out);
}

extern "C" int blb_cp_plan_create_diag(blb_ctx* c, uint32_t L, uint32_t n_groups, const uint32_t* Hg, uint32_t Dh,
                                       const double* W, uint32_t d_out, uint32_t level, const blb_sched* sched,
                                       blb_cp_plan** out)
{
    if (c) BLB_TRY(refuse_capture(c, "plan creation"));
    if (!c || !Hg || !W || !out || n_groups == 0) return blb_fail(BLB_ERR_ARG, "null argument");
    *out = nullptr;
    const uint32_t s = c->N / 2;
    if (L == 0 || s % L || L != 2 * Dh) return blb_fail(BLB_ERR_ARG, "L must divide N/2 and equal 2 Dh");
    const uint32_t k = s / L;
    DiagLayout lay;
    lay.Dh = Dh;
    uint32_t H = 0;
    for (uint32_t g = 0; g < n_groups; g++) {
        if (Hg[g] == 0 || s % (L * Hg[g])) return blb_fail(BLB_ERR_ARG, "L Hg must divide N/2");
        const uint32_t Kc = s / (L * Hg[g]);
        if (Dh % Kc) return blb_fail(BLB_ERR_ARG, "the head dimension must be a multiple of Kc");
        for (uint32_t j = 0; j < Dh / Kc; j++)
            for (uint32_t beta = 0; beta < k; beta++) {
                lay.head.push_back((int32_t)(H + beta % Hg[g]));
                lay.delta.push_back((int32_t)(j * Kc + beta / Hg[g]));
            }
        H += Hg[g];
    }
    lay.nX = (uint32_t)(lay.head.size() / k);
    return cp_plan_build(c, L, H * Dh, W, d_out, level, sched, &lay, out);
}

extern "C" void blb_cp_plan_free(blb_cp_plan* P)
{
    if (!P) return;
    blb_ctx* c = P->ctx;
    dev_free(c, P->d_ptb, P->bytes);
    delete P;
    ctx_release(c);
}

extern "C" int blb_cp_plan_info(const blb_cp_plan* P, uint32_t* nX, uint32_t* nY, uint32_t* b1, uint32_t* G,
                                uint64_t* pt_bytes)
{
    if (!P) return blb_fail(BLB_ERR_ARG, "null plan");
    if (nX) *nX = P->nX;
    if (nY) *nY = P->nY;
    if (b1) *b1 = P->b1;
    if (G) *G = P->G;
    if (pt_bytes) *pt_bytes = P->bytes;
    return BLB_OK;
}

// Y_e = Rescale( sum_g Rot^{g b1 m}( sum_{c,b} Rot^{b m}(X_c) (.) D'_{c,e,g,b} ) ), for S
// sequences at once (X: S x nX handles, sequence-major; Y: S x nY)
static int cp_run(blb_ctx* c, const blb_keys* const* Ks, const blb_cp_plan* P, blb_ct* const* X, uint32_t S,
                  blb_ct** Y)
{
    const uint32_t nX = P->nX, n = P->level + 1, N = c->N;
    for (uint32_t s = 0; s < S; s++)
        if (!Ks[s] || Ks[s]->ctx != c) return blb_fail(BLB_ERR_ARG, "key set missing or from another context");
    for (uint32_t i = 0; i < S * nX; i++) {
        if (!X[i] || X[i]->level != P->level || X[i]->npolys != 2)
            return blb_fail(BLB_ERR_LEVEL, "input ciphertext level does not match the plan");
        if (!same_scale(X[i]->scale, X[0]->scale)) return blb_fail(BLB_ERR_SCALE, "inputs have different scales");
    }
    const size_t ctw = (size_t)2 * n * N;
    const size_t baby_bytes = (size_t)S * nX * P->b1 * ctw * 8, T_bytes = (size_t)S * P->nY * P->G * ctw * 8;
    uint64_t* baby = (uint64_t*)dev_alloc(c, baby_bytes);
    uint64_t* T = (uint64_t*)dev_alloc(c, T_bytes);
    for (uint32_t e = 0; e < S * P->nY; e++) Y[e] = nullptr;
    int rc = (baby && T) ? BLB_OK : blb_fail(BLB_ERR_OOM, "matmul_cp workspace");
    // baby steps: Rot^{b m}(X_c) of every sequence in one pass, hoisted: the
    // decomposition and ModUp of X_c serve all its b1 - 1 rotations
    const uint32_t nb = P->b1 - 1;
    std::vector<uint64_t> gb(nb);
    std::vector<const uint64_t*> kb((size_t)S * nb);  // [sequence][b - 1]
    for (uint32_t b = 1; !rc && b <= nb; b++) {
        gb[b - 1] = galois_element(N, (int32_t)(b * P->m));
        for (uint32_t s = 0; !rc && s < S; s++) {
            const KeyEntry* k = Ks[s]->find(gb[b - 1]);
            if (!k) rc = blb_fail(BLB_ERR_NO_KEY, "no Galois key for rotation " + std::to_string(b * P->m));
            else kb[(size_t)s * nb + b - 1] = k->d;
        }
    }
    {
        std::vector<KsSource> src;
        std::vector<KsProduct> prod;
        std::vector<KsGroup> grp;
        std::vector<KsAdd> adds;
        for (uint32_t ci = 0; !rc && ci < S * nX; ci++) {
            uint64_t* dst0 = baby + (size_t)ci * P->b1 * ctw;
            if (cudaMemcpyAsync(dst0, X[ci]->d, ctw * 8, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                rc = blb_fail(BLB_ERR_CUDA, "copy failed");
            src.push_back(KsSource{X[ci]->d + (size_t)n * N, 1});
            for (uint32_t b = 1; b <= nb; b++) {
                uint64_t* o = dst0 + (size_t)b * ctw;
                grp.push_back(KsGroup{o, o + (size_t)n * N, (uint32_t)prod.size(), (uint32_t)prod.size() + 1,
                                      (uint32_t)adds.size(), (uint32_t)adds.size() + 1});
                prod.push_back(KsProduct{ci, gb[b - 1], kb[(size_t)(ci / nX) * nb + b - 1]});
                adds.push_back(KsAdd{X[ci]->d, gb[b - 1], 0});
            }
        }
        if (!rc && nb)
            rc = ks_run(c, P->level, src.data(), (uint32_t)src.size(), prod.data(), grp.data(), (uint32_t)grp.size(),
                        adds.data(), 0);
    }
    // plaintext products for every (sequence, e, g): at most 8 sequences per
    // launch, and by default at most 4 for plans of several 16-output blocks,
    // where two 4-sequence launches measured faster than one of 8 on the B300
    // (the 8-sequence mma.sync kernel runs out of registers for its warps)
    const uint32_t maxw = (c->batch_mac == 0 && P->NEB > 1) ? 4 : 8;
    for (uint32_t s0 = 0; !rc && s0 < S;) {
        uint32_t chunk = S - s0 >= 8 && maxw >= 8 ? 8 : S - s0 >= 4 ? 4 : S - s0 >= 2 ? 2 : 1;
        rc = launch_cp_mac(c, P, baby + (size_t)s0 * nX * P->b1 * ctw, T + (size_t)s0 * P->nY * P->G * ctw, chunk);
        s0 += chunk;
    }
    // giant steps: T[e][0] + sum_{g >= 1} Rot^{g b1 m}(T[e][g]), the inner
    // products of all g summed over Q_l u P before one ModDown per output
    if (!rc && P->G > 1) {
        std::vector<KsSource> src;
        std::vector<KsProduct> prod;
        std::vector<KsGroup> grp;
        std::vector<KsAdd> adds;
        std::vector<uint64_t> gg(P->G);
        std::vector<const uint64_t*> kg((size_t)S * P->G);  // [sequence][g]
        for (uint32_t g = 1; !rc && g < P->G; g++) {
            gg[g] = galois_element(N, (int32_t)(g * P->b1 * P->m));
            for (uint32_t s = 0; !rc && s < S; s++) {
                const KeyEntry* k = Ks[s]->find(gg[g]);
                if (!k) rc = blb_fail(BLB_ERR_NO_KEY, "no Galois key for rotation " + std::to_string(g * P->b1 * P->m));
                else kg[(size_t)s * P->G + g] = k->d;
            }
        }
        for (uint32_t e = 0; !rc && e < S * P->nY; e++) {
            uint64_t* T0 = T + (size_t)e * P->G * ctw;
            KsGroup G{T0, T0 + (size_t)n * N, (uint32_t)prod.size(), 0, (uint32_t)adds.size(), 0};
            adds.push_back(KsAdd{T0, 1, 0});
            adds.push_back(KsAdd{T0 + (size_t)n * N, 1, 1});
            for (uint32_t g = 1; g < P->G; g++) {
                const uint64_t* Tg = T0 + (size_t)g * ctw;
                prod.push_back(KsProduct{(uint32_t)src.size(), 1, kg[(size_t)(e / P->nY) * P->G + g]});
                src.push_back(KsSource{Tg + (size_t)n * N, gg[g]});
                adds.push_back(KsAdd{Tg, gg[g], 0});
            }
            G.prod1 = (uint32_t)prod.size();
            G.add1 = (uint32_t)adds.size();
            grp.push_back(G);
        }
        if (!rc)
            rc = ks_run(c, P->level, src.data(), (uint32_t)src.size(), prod.data(), grp.data(), (uint32_t)grp.size(),
                        adds.data(), 0);
    }
    // rescale every output in one pass (T[e][0] lie G ciphertexts apart), then
    // hand each its own ciphertext
    const uint32_t ny = S * P->nY;
    const size_t yw = (size_t)2 * P->level * N;
    uint64_t* Ys = rc ? nullptr : (uint64_t*)dev_alloc(c, ny * yw * 8);
    if (!rc && !Ys) rc = blb_fail(BLB_ERR_OOM, "matmul_cp output stack");
    if (!rc) rc = launch_rescale_strided(c, Ys, T, P->level, 2 * ny, 2, (size_t)P->G * ctw);
    for (uint32_t e = 0; !rc && e < ny; e++) {
        blb_ct* y = nullptr;
        rc = new_ct(c, P->level - 1, 2, X[0]->scale, &y);
        if (!rc && cudaMemcpyAsync(y->d, Ys + e * yw, yw * 8, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            rc = blb_fail(BLB_ERR_CUDA, "copy failed");
        Y[e] = y;
    }
    dev_free(c, Ys, ny * yw * 8);
    dev_free(c, baby, baby_bytes);
    dev_free(c, T, T_bytes);
    if (rc) {
        for (uint32_t e = 0; e < S * P->nY; e++) {
            blb_ct_free(Y[e]);
            Y[e] = nullptr;
        }
        return rc;
    }
    return BLB_OK;
}

extern "C" int blb_matmul_cp_plan(blb_ctx* c, const blb_keys* K, const blb_cp_plan* P, blb_ct* const* X,
                                  uint32_t nX, blb_ct** Y)
{
    if (!c || !K || !P || !X || !Y) return blb_fail(BLB_ERR_ARG, "null argument");
    if (nX != P->nX) return blb_fail(BLB_ERR_ARG, "number of input ciphertexts does not match the plan");
    return cp_run(c, &K, P, X, 1, Y);
}

extern "C" int blb_matmul_cp_batch(blb_ctx* c, const blb_keys* K, const blb_cp_plan* P, blb_ct* const* X,
                                   uint32_t n_seq, blb_ct** Y)
{
    if (!c || !K || !P || !X || !Y || n_seq == 0) return blb_fail(BLB_ERR_ARG, "null argument or empty batch");
    std::vector<const blb_keys*> Ks(n_seq, K);
    return cp_run(c, Ks.data(), P, X, n_seq, Y);
}

extern "C" int blb_matmul_cp_multi(blb_ctx* c, const blb_keys* const* keys, const blb_cp_plan* P, blb_ct* const* X,
                                   uint32_t n_seq, blb_ct** Y)
{
    if (!c || !keys || !P || !X || !Y || n_seq == 0) return blb_fail(BLB_ERR_ARG, "null argument or empty batch");
    return cp_run(c, keys, P, X, n_seq, Y);
}

extern "C" int blb_matmul_cp(blb_ctx* c, const blb_keys* K, blb_ct* const* X, uint32_t nX, uint32_t m, uint32_t d,
                             const double* W, uint32_t d_out, const blb_sched* sched, blb_ct** Y)
{
    if (!c || !X || nX == 0 || !X[0]) return blb_fail(BLB_ERR_ARG, "null argument");
    blb_cp_plan* P;
    BLB_TRY(blb_cp_plan_create(c, m, d, W, d_out, X[0]->level, sched, &P));
    int rc = blb_matmul_cp_plan(c, K, P, X, nX, Y);
    blb_cp_plan_free(P);
    return rc;
}

// ===========================================================================
// CKKS -> MPC masking (Alg. 1 steps 1-2)
// ===========================================================================
extern "C" int blb_he2mpc(blb_ctx* c, const blb_keys* K, const blb_ct* ct, uint64_t nonce, blb_ct** masked,
                          uint64_t* p1_share)
{
    if (!c || !K || !ct || !masked || !p1_share) return blb_fail(BLB_ERR_ARG, "null argument");
    if (ct->npolys != 2) return blb_fail(BLB_ERR_ARG, "he2mpc needs a 2-polynomial ciphertext");
    const uint32_t n = ct->level + 1, N = c->N;
    const LimbMap q0 = c->qmap(1);
    uint64_t* r = op_row(c, 0);
    uint64_t* share = op_row(c, 1);
    uint32_t j0 = 0;
    BLB_TRY(launch_sample_uniform(c, r, 1, q0, K->seed, (uint32_t)nonce, PURPOSE_MASK, &j0));
    BLB_TRY(launch_neg_rows(c, share, r, 1, q0));
    BLB_TRY(ntt_forward(c, r, 1, q0));
    blb_ct* o;
    BLB_TRY(new_ct(c, 0, 2, ct->scale, &o));
    int rc = launch_add_rows(c, o->d, ct->d, r, 1, q0);
    if (!rc && cudaMemcpyAsync(o->d + N, ct->d + (size_t)n * N, (size_t)N * 8, cudaMemcpyDeviceToDevice, c->stream))
        rc = blb_fail(BLB_ERR_CUDA, "copy failed");
    if (!rc) rc = copy_out(c, p1_share, share, (size_t)N * 8);
    if (rc) {
        blb_ct_free(o);
        return rc;
    }
    *masked = o;
    return BLB_OK;
}

// ===========================================================================
// low-level transform
// ===========================================================================
extern "C" int blb_ntt(blb_ctx* c, uint64_t* data, uint32_t rows, const uint32_t* prime_idx, int inverse)
{
    if (c && data && !is_device_ptr(data)) BLB_TRY(refuse_capture(c, "blb_ntt on host data"));
    if (!c || !data || !prime_idx) return blb_fail(BLB_ERR_ARG, "null argument");
    for (uint32_t r = 0; r < rows; r++)
        if (prime_idx[r] >= c->np) return blb_fail(BLB_ERR_ARG, "prime index out of range");
    const size_t N = c->N;
    const bool dev = is_device_ptr(data);
    uint64_t* buf = data;
    size_t bytes = rows * N * 8;
    if (!dev) {
        buf = (uint64_t*)dev_alloc(c, bytes);
        if (!buf) return blb_fail(BLB_ERR_OOM, "transform buffer");
        if (cudaMemcpyAsync(buf, data, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            dev_free(c, buf, bytes);
            return blb_fail(BLB_ERR_CUDA, "copy failed");
        }
    }
    int rc = BLB_OK;
    bool same = true;
    for (uint32_t r = 1; r < rows; r++) same &= prime_idx[r] == prime_idx[0];
    if (same && rows) {  // one launch for all rows of one prime
        LimbMap m{};
        m.p[0] = (uint8_t)prime_idx[0];
        m.n = 1;
        rc = inverse ? ntt_inverse(c, buf, rows, m) : ntt_forward(c, buf, rows, m);
    }
    for (uint32_t r0 = 0; !same && !rc && r0 < rows; r0 += BLB_MAXP) {
        uint32_t cnt = std::min<uint32_t>(BLB_MAXP, rows - r0);
        LimbMap m{};
        for (uint32_t r = 0; r < cnt; r++) m.p[r] = (uint8_t)prime_idx[r0 + r];
        m.n = cnt;
        rc = inverse ? ntt_inverse(c, buf + r0 * N, cnt, m) : ntt_forward(c, buf + r0 * N, cnt, m);
    }
    if (!dev) {
        if (!rc && cudaMemcpyAsync(data, buf, bytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            rc = blb_fail(BLB_ERR_CUDA, "copy failed");
        cudaStreamSynchronize(c->stream);
        dev_free(c, buf, bytes);
    }
    return rc;
}
