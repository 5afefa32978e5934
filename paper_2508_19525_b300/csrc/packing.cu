// packing.cu -- rotate-and-sum packing (Sec. 4.2.1) and the HE steps of the
// secure LayerNorm before rsqrt (Alg. LayerNorm lines 1-6), batched over
// independent ciphertexts and sequences.
//
// Spatial-first packing puts block b (L consecutive slots) of a ciphertext at
// slots [b L, (b+1) L).  One round of rotate-and-sum is m <- m + Rot^r(m) with
// r = 2^(i-1) L (left: sum) or -2^(i-1) L (right: broadcast); a round over a
// batch is one key-switching pass (ks_run) whose groups add the rotated c0 and
// the unrotated m to the switched c1, so out = m + Rot^r(m) in one pass.
// Every other step is an existing element-wise kernel, a stacked rescale or a
// batched relinearization, taken in the order the definitions give, so the
// limbs do not depend on the batch.
#include "common.cuh"

namespace {
constexpr int kT = 256;

// out[k] (rows x N) = sum_{c < nc} in[k nc + c] (rows x N), row r mod q_{r % n}
__global__ void k_sum_groups(uint64_t* __restrict__ out, const uint64_t* const* __restrict__ in, uint32_t nc,
                             uint32_t rows, uint32_t n, const uint64_t* __restrict__ qs, uint32_t N)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y, k = blockIdx.z;
    if (i >= N) return;
    const uint64_t q = qs[r % n];
    const size_t o = (size_t)r * N + i;
    uint64_t s = in[(size_t)k * nc][o];
    for (uint32_t c = 1; c < nc; c++) s = add_mod(s, in[(size_t)k * nc + c][o], q);
    out[(size_t)k * rows * N + o] = s;
}

// out[k nc + c] (2 x level rows) = in[k nc + c] with its last limb dropped,
// minus mu[k] (2 x level rows, a contiguous stack)
__global__ void k_drop_sub(uint64_t* const* __restrict__ out, const uint64_t* const* __restrict__ in,
                           const uint64_t* __restrict__ mu, uint32_t nc, uint32_t level,
                           const uint64_t* __restrict__ qs, uint32_t N)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y, j = blockIdx.z;
    if (i >= N) return;
    const uint32_t poly = r / level, l = r % level, k = j / nc;
    const uint64_t q = qs[l];
    const uint64_t x = in[j][((size_t)poly * (level + 1) + l) * N + i];
    const uint64_t m = mu[((size_t)k * 2 * level + r) * N + i];
    out[j][(size_t)r * N + i] = sub_mod(x, m, q);
}

// contiguous stack -> separate ciphertext buffers (rows x N words each)
__global__ void k_unstack(uint64_t* const* __restrict__ out, const uint64_t* __restrict__ in, uint32_t rows, uint32_t N)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y, k = blockIdx.z;
    if (i >= N) return;
    out[k][(size_t)r * N + i] = in[((size_t)k * rows + r) * N + i];
}

int unstack(blb_ctx* c, Scratch& S, blb_ct* const* cts, uint32_t count, const uint64_t* stack)
{
    const uint32_t rows = cts[0]->npolys * (cts[0]->level + 1);
    std::vector<uint64_t*> ptr(count);
    for (uint32_t k = 0; k < count; k++) ptr[k] = cts[k]->d;
    uint64_t* const* d_ptr = S.upload(ptr);
    if (!d_ptr) return blb_fail(BLB_ERR_OOM, "pointer table");
    k_unstack<<<dim3((c->N + kT - 1) / kT, rows, count), kT, 0, c->stream>>>(d_ptr, stack, rows, c->N);
    BLB_LAUNCHED();
    return BLB_OK;
}

// Rounds of rotate-and-sum over `count` ciphertexts stored back to back in
// `buf` (2 x (level+1) x N words each), in place; `tmp` holds one more stack of
// the same size.  Round i reads one of the two stacks and writes the other.
int rs_rounds(blb_ctx* c, const blb_keys* K, uint32_t level, uint64_t* buf, uint64_t* tmp, uint32_t count,
              uint32_t L, uint32_t D, int dir)
{
    const uint32_t N = c->N, n = level + 1;
    const size_t ct_words = (size_t)2 * n * N;
    std::vector<KsSource> src(count);
    std::vector<KsProduct> prod(count);
    std::vector<KsGroup> grp(count);
    std::vector<KsAdd> adds(3 * count);
    uint64_t* cur = buf;
    for (uint32_t step = 1; step < D; step <<= 1) {
        const int32_t r = dir ? -(int32_t)(step * L) : (int32_t)(step * L);
        const uint64_t g = galois_element(N, r);
        const KeyEntry* key = K->find(g);
        if (!key) return blb_fail(BLB_ERR_NO_KEY, "no Galois key for rotation " + std::to_string(r));
        uint64_t* nxt = cur == buf ? tmp : buf;
        for (uint32_t k = 0; k < count; k++) {
            const uint64_t* m = cur + k * ct_words;
            uint64_t* o = nxt + k * ct_words;
            src[k] = KsSource{m + (size_t)n * N, g};
            prod[k] = KsProduct{k, 1, key->d};
            adds[3 * k + 0] = KsAdd{m, g, 0};                  // sigma_g(c0)
            adds[3 * k + 1] = KsAdd{m, 1, 0};                  // + c0
            adds[3 * k + 2] = KsAdd{m + (size_t)n * N, 1, 1};  // + c1
            grp[k] = KsGroup{o, o + (size_t)n * N, k, k + 1, 3 * k, 3 * k + 3};
        }
        BLB_TRY(ks_run(c, level, src.data(), count, prod.data(), grp.data(), count, adds.data(), 0));
        cur = nxt;
    }
    if (cur != buf) BLB_CUDA(cudaMemcpyAsync(buf, cur, count * ct_words * 8, cudaMemcpyDeviceToDevice, c->stream));
    return BLB_OK;
}

// stack (count x 2 x (level+1) rows) times the plaintext of the slot vector z
// (scale q_level), rescaled into out (count x 2 x level rows)
int mul_slots_rescale(blb_ctx* c, Scratch& S, const uint64_t* stack, uint32_t count, uint32_t level,
                      const std::vector<double>& z, uint64_t* out)
{
    const uint32_t N = c->N, n = level + 1;
    double* dz = (double*)S.get(z.size() * 8);
    uint64_t* pt = (uint64_t*)S.get((size_t)n * N * 8);
    uint64_t* prod = (uint64_t*)S.get((size_t)count * 2 * n * N * 8);
    if (!dz || !pt || !prod) return blb_fail(BLB_ERR_OOM, "rotate-and-sum scalar buffers");
    BLB_TRY(host_upload(c, dz, z.data(), z.size() * 8));
    BLB_TRY(encode_slots(c, dz, 1, (uint32_t)z.size(), level, (double)c->q[level], pt));
    BLB_TRY(launch_mul_rows(c, prod, stack, pt, count * 2 * n, c->qmap(n), n));
    BLB_CUDA(cudaStreamSynchronize(c->stream));  // z's host memory is read by the copy above
    return launch_rescale_stack(c, out, prod, level, count * 2);
}

int check_cts(blb_ct* const* in, uint32_t count, uint32_t* level, double* scale)
{
    if (!in || count == 0) return blb_fail(BLB_ERR_ARG, "empty input");
    for (uint32_t k = 0; k < count; k++) {
        if (!in[k] || in[k]->npolys != 2) return blb_fail(BLB_ERR_ARG, "inputs must be 2-polynomial ciphertexts");
        if (in[k]->level != in[0]->level) return blb_fail(BLB_ERR_ARG, "inputs must share one level");
    }
    *level = in[0]->level;
    *scale = in[0]->scale;
    return BLB_OK;
}

void free_all(blb_ct** cts, uint32_t count)
{
    for (uint32_t k = 0; k < count; k++) {
        blb_ct_free(cts[k]);
        cts[k] = nullptr;
    }
}

}  // namespace

extern "C" int blb_rotate_sum_packing(blb_ctx* c, const blb_keys* K, blb_ct* const* in, uint32_t count, uint32_t L,
                                      uint32_t D, int dir, int mask, blb_ct** out)
{
    if (!c || !K || !out) return blb_fail(BLB_ERR_ARG, "null argument");
    uint32_t level;
    double scale;
    BLB_TRY(check_cts(in, count, &level, &scale));
    const uint32_t N = c->N, s = N / 2, n = level + 1;
    if (L == 0 || D == 0 || (D & (D - 1)) || (uint64_t)L * D > s)
        return blb_fail(BLB_ERR_ARG, "need L >= 1, D a power of two and L D <= N/2");
    if (mask && (dir || level == 0)) return blb_fail(BLB_ERR_ARG, "the mask applies to the sum above level 0");
    for (uint32_t k = 0; k < count; k++) out[k] = nullptr;
    const size_t ct_words = (size_t)2 * n * N;
    ProfScope prof(c, "rotsum", (uint64_t)count * ct_words * 8 * 2);
    Scratch S(c);
    uint64_t* a = (uint64_t*)S.get(count * ct_words * 8);
    uint64_t* b = (uint64_t*)S.get(count * ct_words * 8);
    if (!a || !b) return blb_fail(BLB_ERR_OOM, "rotate-and-sum stacks");
    for (uint32_t k = 0; k < count; k++)
        BLB_CUDA(cudaMemcpyAsync(a + k * ct_words, in[k]->d, ct_words * 8, cudaMemcpyDeviceToDevice, c->stream));
    int rc = BLB_OK;
    for (uint32_t k = 0; !rc && k < count; k++) rc = new_ct(c, mask ? level - 1 : level, 2, scale, &out[k]);
    if (!rc) rc = rs_rounds(c, K, level, a, b, count, L, D, dir);
    if (!rc && mask) {
        std::vector<double> z(s, 0.0);
        for (uint32_t j = 0; j < L; j++) z[j] = 1.0;
        rc = mul_slots_rescale(c, S, a, count, level, z, b);
        if (!rc) rc = unstack(c, S, out, count, b);
    } else if (!rc) {
        rc = unstack(c, S, out, count, a);
    }
    if (rc) free_all(out, count);
    return rc;
}

extern "C" int blb_layernorm_head(blb_ctx* c, const blb_keys* K, blb_ct* const* X, uint32_t count, uint32_t nc,
                                  uint32_t L, uint32_t D, blb_ct** X_mu, blb_ct** var)
{
    if (!c || !K || !X_mu || !var || nc == 0) return blb_fail(BLB_ERR_ARG, "null argument");
    uint32_t level;
    double scale;
    BLB_TRY(check_cts(X, count * nc, &level, &scale));
    const uint32_t N = c->N, s = N / 2;
    if (L == 0 || s % L || ((s / L) & (s / L - 1))) return blb_fail(BLB_ERR_ARG, "N/(2L) must be a power of two");
    if (level < 3) return blb_fail(BLB_ERR_LEVEL, "the LayerNorm head needs three levels");
    if (D == 0 || (uint64_t)D > (uint64_t)nc * (s / L)) return blb_fail(BLB_ERR_ARG, "D columns do not fit nc ciphertexts");
    if (!K->find(0)) return blb_fail(BLB_ERR_NO_KEY, "the LayerNorm head needs the relinearization key");
    const uint32_t k = s / L, n0 = level + 1, n1 = level, n2 = level - 1;
    const uint32_t total = count * nc;
    for (uint32_t j = 0; j < total; j++) X_mu[j] = nullptr;
    for (uint32_t j = 0; j < count; j++) var[j] = nullptr;
    ProfScope prof(c, "layernorm", (uint64_t)total * 2 * n0 * N * 8);
    Scratch S(c);
    const size_t w0 = (size_t)2 * n0 * N, w1 = (size_t)2 * n1 * N, w2 = (size_t)2 * n2 * N;
    uint64_t* acc = (uint64_t*)S.get(count * w0 * 8);
    uint64_t* tmp = (uint64_t*)S.get(count * w0 * 8);
    uint64_t* mu = (uint64_t*)S.get(count * w1 * 8);
    uint64_t* t3 = (uint64_t*)S.get((size_t)total * 3 * n1 * N * 8);
    uint64_t* sq2 = (uint64_t*)S.get((size_t)total * w1 * 8);
    uint64_t* sq = (uint64_t*)S.get((size_t)total * w2 * 8);
    uint64_t* acc2 = (uint64_t*)S.get(count * w2 * 8);
    uint64_t* tmp2 = (uint64_t*)S.get(count * w2 * 8);
    if (!acc || !tmp || !mu || !t3 || !sq2 || !sq || !acc2 || !tmp2)
        return blb_fail(BLB_ERR_OOM, "LayerNorm buffers");
    std::vector<const uint64_t*> xin(total);
    for (uint32_t j = 0; j < total; j++) xin[j] = X[j]->d;
    const uint64_t* const* d_xin = S.upload(xin);
    if (!d_xin) return blb_fail(BLB_ERR_OOM, "pointer table");
    int rc = BLB_OK;
    for (uint32_t j = 0; !rc && j < total; j++) rc = new_ct(c, n1 - 1, 2, scale, &X_mu[j]);
    const double sq_scale = scale * scale / (double)c->q[n1 - 1];
    for (uint32_t j = 0; !rc && j < count; j++) rc = new_ct(c, n2 - 2, 2, sq_scale, &var[j]);
    std::vector<double> inv_d(s, 1.0 / (double)D);
    do {
        if (rc) break;
        // lines 1-2: X_sum by rotate-and-sum (no mask: it feeds a scalar operator), mu = X_sum / D
        k_sum_groups<<<dim3((N + kT - 1) / kT, 2 * n0, count), kT, 0, c->stream>>>(acc, d_xin, nc, 2 * n0, n0,
                                                                                   c->d_q, N);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "sum launch failed"); break; }
        blb_count_launch();
        if ((rc = rs_rounds(c, K, level, acc, tmp, count, L, k, 0))) break;
        if ((rc = mul_slots_rescale(c, S, acc, count, level, inv_d, mu))) break;
        // line 3: X_mu = X (one level down) - mu
        std::vector<uint64_t*> xo(total);
        for (uint32_t j = 0; j < total; j++) xo[j] = X_mu[j]->d;
        uint64_t* const* d_xo = S.upload(xo);
        if (!d_xo) { rc = blb_fail(BLB_ERR_OOM, "pointer table"); break; }
        k_drop_sub<<<dim3((N + kT - 1) / kT, 2 * n1, total), kT, 0, c->stream>>>(d_xo, d_xin, mu, nc, n1, c->d_q, N);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "subtraction launch failed"); break; }
        blb_count_launch();
        // line 4: X_mu^2, relinearized and rescaled
        for (uint32_t j = 0; !rc && j < total; j++)
            rc = launch_tensor(c, t3 + (size_t)j * 3 * n1 * N, X_mu[j]->d, X_mu[j]->d, n1 - 1);
        if (rc) break;
        const KeyEntry* rk = K->find(0);
        std::vector<KsItem> items(total);
        for (uint32_t j = 0; j < total; j++) {
            const uint64_t* t = t3 + (size_t)j * 3 * n1 * N;
            uint64_t* o = sq2 + (size_t)j * w1;
            items[j] = KsItem{t, t + (size_t)2 * n1 * N, t + (size_t)n1 * N, rk->d, o, o + (size_t)n1 * N, 1};
        }
        if ((rc = keyswitch_batch(c, n1 - 1, items.data(), total, 0))) break;
        if ((rc = launch_rescale_stack(c, sq, sq2, n1 - 1, 2 * total))) break;
        // lines 5-6: the row sums of X_mu^2, divided by D
        std::vector<const uint64_t*> sqp(total);
        for (uint32_t j = 0; j < total; j++) sqp[j] = sq + (size_t)j * w2;
        const uint64_t* const* d_sqp = S.upload(sqp);
        if (!d_sqp) { rc = blb_fail(BLB_ERR_OOM, "pointer table"); break; }
        k_sum_groups<<<dim3((N + kT - 1) / kT, 2 * n2, count), kT, 0, c->stream>>>(acc2, d_sqp, nc, 2 * n2, n2,
                                                                                   c->d_q, N);
        if (cudaGetLastError() != cudaSuccess) { rc = blb_fail(BLB_ERR_CUDA, "sum launch failed"); break; }
        blb_count_launch();
        if ((rc = rs_rounds(c, K, n2 - 1, acc2, tmp2, count, L, k, 0))) break;
        uint64_t* vstack = tmp2;  // count x 2 x (n2 - 1) rows, free again after the rounds
        if ((rc = mul_slots_rescale(c, S, acc2, count, n2 - 1, inv_d, vstack))) break;
        rc = unstack(c, S, var, count, vstack);
    } while (0);
    if (rc) {
        free_all(X_mu, total);
        free_all(var, count);
    }
    return rc;
}
