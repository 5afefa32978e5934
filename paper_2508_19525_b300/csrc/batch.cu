// batch.cu -- encoding, encryption, CKKS -> MPC masking (Alg. 1) and decryption
// of many ciphertexts per call.
//
// Each entry point computes exactly what the single-ciphertext call computes
// for every member of the batch (the same Philox counters, with the caller's
// nonce per ciphertext as the object index, and the same modular arithmetic),
// but runs every step once over a contiguous stack: one sampling launch, one
// NTT over all rows, one combining launch that reads and writes the members
// through pointer tables.  That turns several launches per ciphertext into a
// few per batch, so the per-ciphertext calls no longer leave the GPU idle.
#include "common.cuh"

namespace {
constexpr int kT = 256;

dim3 rows_grid(uint32_t N, uint32_t rows) { return dim3((N + kT - 1) / kT, rows); }

struct RowDraw {
    uint32_t obj, j, prime;
};

// uniform residues: row r draws counter (i, j_r, obj_r, purpose) -> 128 bits mod q
__global__ void k_uniform_rows(uint64_t* __restrict__ out, uint32_t N, const RowDraw* __restrict__ rows,
                               const uint64_t* __restrict__ qs, const uint64_t* __restrict__ bar, uint64_t seed,
                               uint32_t purpose)
{
    const uint32_t r = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const RowDraw d = rows[r];
    const uint4 x = philox_draw(seed, i, d.j, d.obj, purpose);
    const uint64_t lo = (uint64_t)x.x | ((uint64_t)x.y << 32), hi = (uint64_t)x.z | ((uint64_t)x.w << 32);
    out[(size_t)r * N + i] = barrett128(lo, hi, qs[d.prime], bar[2 * d.prime], bar[2 * d.prime + 1]);
}

// discrete Gaussian (CDT), one signed row per object, sub-index 0
__global__ void k_gauss_rows(int64_t* __restrict__ out, uint32_t N, const uint32_t* __restrict__ objs,
                             const uint64_t* __restrict__ cdt, uint64_t seed, uint32_t purpose)
{
    const uint32_t r = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint4 x = philox_draw(seed, i, 0, objs[r], purpose);
    const uint64_t u = (uint64_t)x.x | ((uint64_t)x.y << 32);
    int64_t k = 0;
#pragma unroll
    for (int t = 0; t < 19; t++) k += (u >= cdt[t]);
    out[(size_t)r * N + i] = (x.z & 1u) ? -k : k;
}

// signed row c -> residues of limbs 0..n-1: out[(c n + i) N + k]
__global__ void k_signed_to_limbs(uint64_t* __restrict__ out, const int64_t* __restrict__ in, uint32_t n,
                                  const uint64_t* __restrict__ qs, const uint64_t* __restrict__ bar, uint32_t N)
{
    const uint32_t row = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const uint32_t c = row / n, i = row % n;
    out[(size_t)row * N + k] = signed_mod(in[(size_t)c * N + k], qs[i], bar[2 * i + 1]);
}

// encryption of member c, limb i (row = c n + i):
//   c0 = -(a s) + m + e,  c1 = a   (a = A row, e = E row, NTT domain)
__global__ void k_enc_finish(uint64_t* const* __restrict__ cts, const uint64_t* const* __restrict__ pts,
                             const uint64_t* __restrict__ Arows, const uint64_t* __restrict__ Erows,
                             const uint64_t* __restrict__ s, uint32_t n, const uint64_t* __restrict__ qs,
                             const uint64_t* __restrict__ bar, uint32_t N)
{
    const uint32_t row = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const uint32_t c = row / n, i = row % n;
    const uint64_t q = qs[i];
    const size_t o = (size_t)row * N + k;
    const uint64_t a = Arows[o];
    const uint64_t as = mul_mod(a, s[(size_t)i * N + k], q, bar[2 * i], bar[2 * i + 1]);
    uint64_t c0 = sub_mod(0, as, q);
    c0 = add_mod(c0, pts[c][(size_t)i * N + k], q);
    c0 = add_mod(c0, Erows[o], q);
    cts[c][(size_t)i * N + k] = c0;
    cts[c][((size_t)n + i) * N + k] = a;
}

// masking of member c: (ct.c0 limb 0 + r, ct.c1 limb 0); ins[c] has nl[c] limbs per polynomial
__global__ void k_mask_finish(uint64_t* const* __restrict__ outs, const uint64_t* const* __restrict__ ins,
                              const uint32_t* __restrict__ nl, const uint64_t* __restrict__ Rrows, uint64_t q0,
                              uint32_t N)
{
    const uint32_t c = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const uint64_t* in = ins[c];
    outs[c][k] = add_mod(in[k], Rrows[(size_t)c * N + k], q0);
    outs[c][(size_t)N + k] = in[(size_t)nl[c] * N + k];
}

// decryption of member c, limb i (row = c n + i): Horner over the polynomials,
// h = c_{np-1}; h = h s + c_k
__global__ void k_dec_rows(uint64_t* __restrict__ H, const uint64_t* const* __restrict__ cts, uint32_t n,
                           uint32_t npolys, const uint64_t* __restrict__ s, const uint64_t* __restrict__ qs,
                           const uint64_t* __restrict__ bar, uint32_t N)
{
    const uint32_t row = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const uint32_t c = row / n, i = row % n;
    const uint64_t q = qs[i], r0 = bar[2 * i], r1 = bar[2 * i + 1];
    const uint64_t* ct = cts[c];
    const uint64_t si = s[(size_t)i * N + k];
    uint64_t h = ct[((size_t)(npolys - 1) * n + i) * N + k];
    for (int p = (int)npolys - 2; p >= 0; p--) h = add_mod(mul_mod(h, si, q, r0, r1), ct[((size_t)p * n + i) * N + k], q);
    H[(size_t)row * N + k] = h;
}

// device scratch for one batch call, freed on every return path

}  // namespace

extern "C" int blb_encode_batch(blb_ctx* c, const double* vals, uint64_t n, uint32_t count, uint32_t level,
                                double scale, blb_pt** out)
{
    if (!c || !out || count == 0 || (n && !vals)) return blb_fail(BLB_ERR_ARG, "null argument or empty batch");
    if (level >= c->nQ) return blb_fail(BLB_ERR_LEVEL, "level out of range");
    if (n > c->N / 2) return blb_fail(BLB_ERR_ARG, "more values than slots");
    if (!(scale > 0)) return blb_fail(BLB_ERR_ARG, "scale must be positive");
    for (uint32_t i = 0; i < count; i++) out[i] = nullptr;
    const size_t pw = (size_t)(level + 1) * c->N;
    Scratch S(c);
    double* dz = n ? (double*)S.get((size_t)count * n * 8) : nullptr;
    uint64_t* stack = (uint64_t*)S.get((size_t)count * pw * 8);
    if ((n && !dz) || !stack) return blb_fail(BLB_ERR_OOM, "encoding batch buffers");
    if (n) BLB_TRY(copy_in(c, dz, vals, (size_t)count * n * 8));
    BLB_TRY(encode_slots(c, dz, count, (uint32_t)n, level, scale, stack));
    int rc = BLB_OK;
    for (uint32_t i = 0; !rc && i < count; i++) {
        blb_pt* pt = new blb_pt();
        pt->ctx = c;
        ctx_retain(c);
        pt->level = level;
        pt->scale = scale;
        pt->bytes = pw * 8;
        pt->d = (uint64_t*)dev_alloc(c, pt->bytes);
        out[i] = pt;
        if (!pt->d) rc = blb_fail(BLB_ERR_OOM, "plaintext allocation failed");
        else if (cudaMemcpyAsync(pt->d, stack + i * pw, pt->bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            rc = blb_fail(BLB_ERR_CUDA, "copy failed");
    }
    if (rc)
        for (uint32_t i = 0; i < count; i++) {
            blb_pt_free(out[i]);
            out[i] = nullptr;
        }
    return rc;
}

extern "C" int blb_encrypt_batch(blb_ctx* c, const blb_keys* K, const blb_pt* const* pts, uint32_t count,
                                 const uint64_t* nonces, blb_ct** out)
{
    if (!c || !K || !pts || !nonces || !out || count == 0) return blb_fail(BLB_ERR_ARG, "null argument or empty batch");
    for (uint32_t i = 0; i < count; i++) {
        out[i] = nullptr;
        if (!pts[i]) return blb_fail(BLB_ERR_ARG, "null plaintext");
        if (pts[i]->level != pts[0]->level) return blb_fail(BLB_ERR_LEVEL, "plaintexts of one batch share a level");
    }
    const uint32_t n = pts[0]->level + 1, N = c->N, rows = count * n;
    Scratch S(c);
    uint64_t* A = (uint64_t*)S.get((size_t)rows * N * 8);
    uint64_t* E = (uint64_t*)S.get((size_t)rows * N * 8);
    int64_t* e = (int64_t*)S.get((size_t)count * N * 8);
    std::vector<RowDraw> rd(rows);
    std::vector<uint32_t> objs(count);
    std::vector<const uint64_t*> hp(count);
    for (uint32_t k = 0; k < count; k++) {
        objs[k] = (uint32_t)nonces[k];
        hp[k] = pts[k]->d;
        for (uint32_t i = 0; i < n; i++) rd[k * n + i] = RowDraw{(uint32_t)nonces[k], i, i};
    }
    const RowDraw* d_rd = S.upload(rd);
    const uint32_t* d_objs = S.upload(objs);
    const uint64_t* const* d_pts = S.upload(hp);
    if (!A || !E || !e || !d_rd || !d_objs || !d_pts) return blb_fail(BLB_ERR_OOM, "encryption batch buffers");
    int rc = BLB_OK;
    std::vector<uint64_t*> hc(count);
    for (uint32_t k = 0; !rc && k < count; k++) {
        rc = new_ct(c, n - 1, 2, pts[k]->scale, &out[k]);
        if (!rc) hc[k] = out[k]->d;
    }
    uint64_t* const* d_cts = rc ? nullptr : S.upload(hc);
    if (!rc && !d_cts) rc = blb_fail(BLB_ERR_OOM, "encryption batch table");
    const LimbMap qm = c->qmap(n);
    do {
        if (rc) break;
        k_uniform_rows<<<rows_grid(N, rows), kT, 0, c->stream>>>(A, N, d_rd, c->d_q, c->d_bar, K->seed,
                                                                  PURPOSE_ENC_A);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "sampling launch failed"); break; }
        blb_count_launch();
        if ((rc = ntt_forward(c, A, rows, qm))) break;
        k_gauss_rows<<<rows_grid(N, count), kT, 0, c->stream>>>(e, N, d_objs, c->d_cdt, K->seed, PURPOSE_ENC_E);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "sampling launch failed"); break; }
        blb_count_launch();
        k_signed_to_limbs<<<rows_grid(N, rows), kT, 0, c->stream>>>(E, e, n, c->d_q, c->d_bar, N);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "conversion launch failed"); break; }
        blb_count_launch();
        if ((rc = ntt_forward(c, E, rows, qm))) break;
        k_enc_finish<<<rows_grid(N, rows), kT, 0, c->stream>>>(d_cts, d_pts, A, E, K->d_s, n, c->d_q, c->d_bar, N);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "encryption launch failed"); break; }
        blb_count_launch();
    } while (0);
    if (rc)
        for (uint32_t k = 0; k < count; k++) {
            blb_ct_free(out[k]);
            out[k] = nullptr;
        }
    return rc;
}

extern "C" int blb_he2mpc_batch(blb_ctx* c, const blb_keys* K, const blb_ct* const* cts, uint32_t count,
                                const uint64_t* nonces, blb_ct** masked, uint64_t* p1_shares)
{
    if (!c || !K || !cts || !nonces || !masked || !p1_shares || count == 0)
        return blb_fail(BLB_ERR_ARG, "null argument or empty batch");
    for (uint32_t k = 0; k < count; k++) {
        masked[k] = nullptr;
        if (!cts[k] || cts[k]->npolys != 2) return blb_fail(BLB_ERR_ARG, "he2mpc needs 2-polynomial ciphertexts");
    }
    const uint32_t N = c->N;
    Scratch S(c);
    uint64_t* R = (uint64_t*)S.get((size_t)count * N * 8);
    uint64_t* share = (uint64_t*)S.get((size_t)count * N * 8);
    std::vector<RowDraw> rd(count);
    std::vector<const uint64_t*> hin(count);
    std::vector<uint32_t> nl(count);
    for (uint32_t k = 0; k < count; k++) {
        rd[k] = RowDraw{(uint32_t)nonces[k], 0, 0};
        hin[k] = cts[k]->d;
        nl[k] = cts[k]->level + 1;
    }
    const RowDraw* d_rd = S.upload(rd);
    const uint64_t* const* d_in = S.upload(hin);
    const uint32_t* d_nl = S.upload(nl);
    if (!R || !share || !d_rd || !d_in || !d_nl) return blb_fail(BLB_ERR_OOM, "masking batch buffers");
    int rc = BLB_OK;
    std::vector<uint64_t*> ho(count);
    for (uint32_t k = 0; !rc && k < count; k++) {
        rc = new_ct(c, 0, 2, cts[k]->scale, &masked[k]);
        if (!rc) ho[k] = masked[k]->d;
    }
    uint64_t* const* d_out = rc ? nullptr : S.upload(ho);
    if (!rc && !d_out) rc = blb_fail(BLB_ERR_OOM, "masking batch table");
    const LimbMap q0 = c->qmap(1);
    do {
        if (rc) break;
        k_uniform_rows<<<rows_grid(N, count), kT, 0, c->stream>>>(R, N, d_rd, c->d_q, c->d_bar, K->seed,
                                                                   PURPOSE_MASK);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "sampling launch failed"); break; }
        blb_count_launch();
        if ((rc = launch_neg_rows(c, share, R, count, q0))) break;  // P1's share: -r mod q0
        if ((rc = ntt_forward(c, R, count, q0))) break;
        k_mask_finish<<<rows_grid(N, count), kT, 0, c->stream>>>(d_out, d_in, d_nl, R, c->q[0], N);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "masking launch failed"); break; }
        blb_count_launch();
        rc = copy_out(c, p1_shares, share, (size_t)count * N * 8);
    } while (0);
    if (rc)
        for (uint32_t k = 0; k < count; k++) {
            blb_ct_free(masked[k]);
            masked[k] = nullptr;
        }
    return rc;
}

extern "C" int blb_decrypt_batch(blb_ctx* c, const blb_keys* K, const blb_ct* const* cts, uint32_t count,
                                 uint64_t* coeff_limbs, double* slots)
{
    if (!c || !K || !cts || count == 0) return blb_fail(BLB_ERR_ARG, "null argument or empty batch");
    for (uint32_t k = 0; k < count; k++) {
        if (!cts[k]) return blb_fail(BLB_ERR_ARG, "null ciphertext");
        if (cts[k]->level != cts[0]->level || cts[k]->npolys != cts[0]->npolys)
            return blb_fail(BLB_ERR_LEVEL, "ciphertexts of one batch share a level and a size");
    }
    const uint32_t n = cts[0]->level + 1, N = c->N, rows = count * n;
    Scratch S(c);
    uint64_t* H = (uint64_t*)S.get((size_t)rows * N * 8);
    std::vector<const uint64_t*> hin(count);
    for (uint32_t k = 0; k < count; k++) hin[k] = cts[k]->d;
    const uint64_t* const* d_in = S.upload(hin);
    if (!H || !d_in) return blb_fail(BLB_ERR_OOM, "decryption batch buffers");
    k_dec_rows<<<rows_grid(N, rows), kT, 0, c->stream>>>(H, d_in, n, cts[0]->npolys, K->d_s, c->d_q, c->d_bar, N);
    BLB_LAUNCHED();
    BLB_TRY(ntt_inverse(c, H, rows, c->qmap(n)));
    if (coeff_limbs) BLB_TRY(copy_out(c, coeff_limbs, H, (size_t)rows * N * 8));
    if (slots) {
        double* dz = (double*)S.get((size_t)count * (N / 2) * 8);
        if (!dz) return blb_fail(BLB_ERR_OOM, "decoding batch buffer");
        for (uint32_t k = 0; k < count; k++) BLB_TRY(decode_limb0(c, H + (size_t)k * n * N, cts[k]->scale, dz + (size_t)k * (N / 2)));
        BLB_TRY(copy_out(c, slots, dz, (size_t)count * (N / 2) * 8));
    }
    return BLB_OK;
}
