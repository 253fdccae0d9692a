// Surrogate MLP: forward, backward and AdamW on the GPU.
//
// The paper screens candidate designs with a Gaussian-process model inside its
// efficient global optimisation (Sec. II.A); the surrogate here is a small
// multilayer perceptron, x -> [W x + b -> GELU] x depth -> W x + b (logits of the
// target-switch and adjacent-flip probabilities), trained with the sigmoid
// binary cross-entropy and AdamW (decoupled weight decay on the weight
// matrices).  Every contraction runs on the tcgen05 GEMM with BF16 operands and
// FP32 accumulation; FP32 master weights and Adam moments live on the device.
//
// Layer l multiplies activations [batch][in_pad] by W_l [out_pad][in_pad]:
//   forward      Z = H W^T + b, H' = GELU(Z)       (epilogue keeps Z and both layouts of H')
//   weight grad  dW = dZ^T H                        (K = batch: operands dZ^T, H^T)
//   input grad   dH = dZ W, dZ_prev = dH GELU'(Z)   (epilogue, plus per-block bias sums)
// in_pad = out_pad of the previous layer; feature widths are padded to 128 so
// that every GEMM dimension meets the tile sizes, and the pads stay zero.
#include <cmath>
#include <cstdio>

#include "bpm_internal.cuh"

namespace bpm {

namespace {

int rup(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

struct Mlp {
    int n_in = 0, width = 0, depth = 0, n_out = 0, L = 0;
    std::vector<int> in_real, out_real, in_pad, out_pad;
    std::vector<size_t> w_off, b_off;
    size_t P = 0;
    float *params = nullptr, *mom1 = nullptr, *mom2 = nullptr, *grad = nullptr;
    std::vector<__nv_bfloat16*> W, WT;
    long long t = 0;
    // workspace for up to ws_rows batch rows
    int ws_rows = 0;
    std::vector<__nv_bfloat16*> H, HT;   // H[l]: input of layer l ([rows][in_pad[l]]), HT its transpose
    std::vector<float*> Z;               // Z[l]: pre-activation of hidden layer l
    float *logits = nullptr, *Y = nullptr, *colsum = nullptr, *loss = nullptr;
    __nv_bfloat16 *dZa = nullptr, *dZaT = nullptr, *dZb = nullptr, *dZbT = nullptr;
    int* err = nullptr;
    int max_pad = 0;
};

namespace {

void free_ws(Mlp* m) {
    for (auto p : m->H) cudaFree(p);
    for (auto p : m->HT) cudaFree(p);
    for (auto p : m->Z) cudaFree(p);
    m->H.clear();
    m->HT.clear();
    m->Z.clear();
    cudaFree(m->logits);
    cudaFree(m->Y);
    cudaFree(m->colsum);
    cudaFree(m->dZa);
    cudaFree(m->dZaT);
    cudaFree(m->dZb);
    cudaFree(m->dZbT);
    m->logits = m->Y = m->colsum = nullptr;
    m->dZa = m->dZaT = m->dZb = m->dZbT = nullptr;
    m->ws_rows = 0;
}

template <class T>
int zalloc(T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) e = cudaMemset(*p, 0, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        set_error("device allocation of %zu bytes: %s", n * sizeof(T), cudaGetErrorString(e));
        return BPM_ERR_OOM;
    }
    return BPM_OK;
}

int ensure_ws(Mlp* m, int rows) {
    if (rows <= m->ws_rows) return BPM_OK;
    free_ws(m);
    m->H.assign(m->L, nullptr);
    m->HT.assign(m->L, nullptr);
    m->Z.assign(m->L, nullptr);
    for (int l = 0; l < m->L; ++l) {
        BPM_TRY(zalloc(&m->H[l], (size_t)rows * m->in_pad[l]));
        BPM_TRY(zalloc(&m->HT[l], (size_t)rows * m->in_pad[l]));
        if (l < m->L - 1) BPM_TRY(zalloc(&m->Z[l], (size_t)rows * m->out_pad[l]));
    }
    BPM_TRY(zalloc(&m->logits, (size_t)rows * m->n_out));
    BPM_TRY(zalloc(&m->Y, (size_t)rows * m->n_out));
    BPM_TRY(zalloc(&m->colsum, (size_t)(rows / 32) * m->max_pad));
    BPM_TRY(zalloc(&m->dZa, (size_t)rows * m->max_pad));
    BPM_TRY(zalloc(&m->dZaT, (size_t)rows * m->max_pad));
    BPM_TRY(zalloc(&m->dZb, (size_t)rows * m->max_pad));
    BPM_TRY(zalloc(&m->dZbT, (size_t)rows * m->max_pad));
    m->ws_rows = rows;
    return BPM_OK;
}

// rows [0, nb) of X (fp32 [*][n_in]) -> bf16 [rows][in_pad] and its transpose; pads zero
// the input batch as BF16 [rows][in_pad] (zero padded): one thread per 8 columns of a row, so
// that a warp writes consecutive 16-byte chunks
__global__ void k_load_x(int nb, int rows, int n_in, int in_pad, const float* __restrict__ X,
                         __nv_bfloat16* __restrict__ H0) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int chunks = in_pad / 8;
    if (q >= (long long)rows * chunks) return;
    const int r = (int)(q / chunks), c0 = (int)(q % chunks) * 8;
    uint32_t pk[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = c0 + 2 * u;
        const float a = (r < nb && c < n_in) ? X[(size_t)r * n_in + c] : 0.f;
        const float b = (r < nb && c + 1 < n_in) ? X[(size_t)r * n_in + c + 1] : 0.f;
        const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        pk[u] = *reinterpret_cast<const uint32_t*>(&v);
    }
    *reinterpret_cast<uint4*>(H0 + (size_t)r * in_pad + c0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
}

// its transpose [in_pad][rows] for the weight gradient of the first layer (training only)
__global__ void k_load_xt(int nb, int rows, int n_in, int in_pad, const float* __restrict__ X,
                          __nv_bfloat16* __restrict__ H0T) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)rows * in_pad) return;
    const int c = (int)(q / rows), r = (int)(q % rows);
    const float v = (r < nb && c < n_in) ? X[(size_t)r * n_in + c] : 0.f;
    H0T[q] = __float2bfloat16_rn(v);
}

// loss head (one CTA): mean sigmoid-BCE over nb x n_out, dz = (sigmoid(z) - y) / (nb n_out)
// into dZ [rows][out_pad] and dZ^T [out_pad][rows], bias gradient and loss in fixed order
__global__ void k_loss_head(int nb, int n_out, int out_pad, int rows, const float* __restrict__ logits,
                            const float* __restrict__ Y, __nv_bfloat16* __restrict__ dZ,
                            __nv_bfloat16* __restrict__ dZT, float* __restrict__ db, float* __restrict__ loss_out) {
    __shared__ float red[32];
    const float inv = 1.f / ((float)nb * (float)n_out);
    float lsum = 0.f;
    for (int r = threadIdx.x; r < nb; r += blockDim.x)
        for (int o = 0; o < n_out; ++o) {
            float z = logits[(size_t)r * n_out + o], y = Y[(size_t)r * n_out + o];
            lsum += fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - y * z;
            float g = (1.f / (1.f + expf(-z)) - y) * inv;
            __nv_bfloat16 b = __float2bfloat16_rn(g);
            dZ[(size_t)r * out_pad + o] = b;
            dZT[(size_t)o * rows + r] = b;
        }
    auto bsum = [&](float v) {
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        return s;
    };
    float L = bsum(lsum);
    if (threadIdx.x == 0 && loss_out) *loss_out = L * inv;
    for (int o = 0; o < n_out; ++o) {
        float g = 0.f;
        for (int r = threadIdx.x; r < nb; r += blockDim.x) {
            float z = logits[(size_t)r * n_out + o], y = Y[(size_t)r * n_out + o];
            g += (1.f / (1.f + expf(-z)) - y) * inv;
        }
        float s = bsum(g);
        if (threadIdx.x == 0) db[o] = s;
    }
}

// bias gradient from the per-(32-row block) partial column sums, fixed order
__global__ void k_colsum_reduce(int nblk, int ncol, int ld, const float* __restrict__ part, float* __restrict__ db) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    float s = 0.f;
    for (int k = 0; k < nblk; ++k) s += part[(size_t)k * ld + c];
    db[c] = s;
}

struct LayerTable {
    int L;
    long long w_off[8], b_off[8];
    int in_real[8], out_real[8], in_pad[8], out_pad[8];
};

// AdamW on the flat FP32 parameters, then the BF16 copies W [out_pad][in_pad] and W^T [in_pad][out_pad]
__global__ void k_adamw(long long P, LayerTable T, float* __restrict__ p, float* __restrict__ m1,
                        float* __restrict__ m2, const float* __restrict__ g, float lr, float wd, float b1, float b2,
                        float eps, float c1, float c2, __nv_bfloat16* const* __restrict__ W,
                        __nv_bfloat16* const* __restrict__ WT) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    int l = 0;
    while (l + 1 < T.L && k >= T.w_off[l + 1]) ++l;
    const bool is_w = k < T.b_off[l];
    float gv = g[k];
    float a = b1 * m1[k] + (1.f - b1) * gv;
    float v = b2 * m2[k] + (1.f - b2) * gv * gv;
    m1[k] = a;
    m2[k] = v;
    float pv = p[k];
    pv -= lr * ((a / c1) / (sqrtf(v / c2) + eps) + (is_w ? wd * pv : 0.f));
    p[k] = pv;
    if (is_w) {
        long long e = k - T.w_off[l];
        int o = (int)(e / T.in_real[l]), i = (int)(e % T.in_real[l]);
        __nv_bfloat16 b = __float2bfloat16_rn(pv);
        W[l][(size_t)o * T.in_pad[l] + i] = b;
        WT[l][(size_t)i * T.out_pad[l] + o] = b;
    }
}

// BF16 copies of the current weights (after creation or load)
__global__ void k_publish(long long P, LayerTable T, const float* __restrict__ p, __nv_bfloat16* const* __restrict__ W,
                          __nv_bfloat16* const* __restrict__ WT) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    int l = 0;
    while (l + 1 < T.L && k >= T.w_off[l + 1]) ++l;
    if (k >= T.b_off[l]) return;
    long long e = k - T.w_off[l];
    int o = (int)(e / T.in_real[l]), i = (int)(e % T.in_real[l]);
    __nv_bfloat16 b = __float2bfloat16_rn(p[k]);
    W[l][(size_t)o * T.in_pad[l] + i] = b;
    WT[l][(size_t)i * T.out_pad[l] + o] = b;
}

LayerTable table(const Mlp* m) {
    LayerTable T{};
    T.L = m->L;
    for (int l = 0; l < m->L; ++l) {
        T.w_off[l] = (long long)m->w_off[l];
        T.b_off[l] = (long long)m->b_off[l];
        T.in_real[l] = m->in_real[l];
        T.out_real[l] = m->out_real[l];
        T.in_pad[l] = m->in_pad[l];
        T.out_pad[l] = m->out_pad[l];
    }
    return T;
}

__nv_bfloat16** device_ptr_table(const std::vector<__nv_bfloat16*>& v, int* err) {
    __nv_bfloat16** d = nullptr;
    if (cudaMalloc(&d, v.size() * sizeof(void*)) != cudaSuccess ||
        cudaMemcpy(d, v.data(), v.size() * sizeof(void*), cudaMemcpyHostToDevice) != cudaSuccess) {
        *err = 1;
        return nullptr;
    }
    return d;
}

// forward over `rows` (multiple of 128) batch rows, nb of them valid, input already in H[0]/HT[0]
// infer: skip the pre-activations and transposes kept for the backward pass;
// sigmoid: probabilities instead of logits in m->logits
int forward(Mlp* m, cudaStream_t s, int rows, int nb, bool infer, bool sigmoid) {
    for (int l = 0; l < m->L; ++l) {
        TcEpilogue e{};
        e.bias = m->params + m->b_off[l];
        e.rows_valid = nb;
        e.cols_valid = m->out_real[l];
        if (l < m->L - 1) {
            // the pre-activation z and the transposed activations serve the backward pass only
            e.C = infer ? nullptr : m->Z[l];
            e.ldc = m->out_pad[l];
            e.H = m->H[l + 1];
            e.ldh = m->in_pad[l + 1];
            e.HT = infer ? nullptr : m->HT[l + 1];
            e.ldht = rows;
            BPM_TRY(gemm_tc(s, TC_EPI_BIAS_GELU, rows, m->out_pad[l], m->in_pad[l], m->H[l], m->W[l], e, m->err));
        } else {
            e.C = m->logits;
            e.ldc = m->n_out;
            e.sigmoid = sigmoid ? 1 : 0;
            BPM_TRY(gemm_tc(s, TC_EPI_BIAS_OUT, rows, m->out_pad[l], m->in_pad[l], m->H[l], m->W[l], e, m->err));
        }
    }
    return BPM_OK;
}

// backward for the batch in the workspace: gradients into m->grad, loss into loss_slot
int backward(Mlp* m, cudaStream_t s, int rows, int nb, float* loss_slot) {
    const int Lm = m->L - 1;
    BPM_CK(cudaMemsetAsync(m->dZa, 0, sizeof(__nv_bfloat16) * (size_t)rows * m->max_pad, s));
    BPM_CK(cudaMemsetAsync(m->dZaT, 0, sizeof(__nv_bfloat16) * (size_t)rows * m->max_pad, s));
    k_loss_head<<<1, 1024, 0, s>>>(nb, m->n_out, m->out_pad[Lm], rows, m->logits, m->Y, m->dZa, m->dZaT,
                                   m->grad + m->b_off[Lm], loss_slot);
    BPM_CK(cudaGetLastError());
    __nv_bfloat16 *dz = m->dZa, *dzT = m->dZaT, *dzn = m->dZb, *dznT = m->dZbT;
    for (int l = Lm; l >= 0; --l) {
        // dW_l = dZ_l^T H_l
        TcEpilogue g{};
        g.C = m->grad + m->w_off[l];
        g.ldc = m->in_real[l];
        g.rows_valid = m->out_real[l];
        g.cols_valid = m->in_real[l];
        BPM_TRY(gemm_tc(s, TC_EPI_STORE, m->out_pad[l], m->in_pad[l], rows, dzT, m->HT[l], g, m->err));
        if (l == 0) break;
        // dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1}), bias gradient of layer l-1
        TcEpilogue e{};
        e.Zin = m->Z[l - 1];
        e.ldz = m->out_pad[l - 1];
        e.H = dzn;
        e.ldh = m->out_pad[l - 1];
        e.HT = dznT;
        e.ldht = rows;
        e.colsum = m->colsum;
        e.ldcs = m->in_pad[l];
        e.rows_valid = nb;
        e.cols_valid = m->out_real[l - 1];
        BPM_TRY(gemm_tc(s, TC_EPI_GELU_BWD, rows, m->in_pad[l], m->out_pad[l], dz, m->WT[l], e, m->err));
        k_colsum_reduce<<<(m->out_real[l - 1] + 127) / 128, 128, 0, s>>>(rows / 32, m->out_real[l - 1], m->in_pad[l],
                                                                         m->colsum, m->grad + m->b_off[l - 1]);
        BPM_CK(cudaGetLastError());
        std::swap(dz, dzn);
        std::swap(dzT, dznT);
    }
    return BPM_OK;
}

// Screened error rates (Sec. II.C), one chunk of rows [r0, r0 + nb) of the
// design-major sample list: one warp per (design, output) that has samples in
// the chunk adds its share to acc[d][k] in FP64, lanes strided over the
// samples and a fixed shuffle tree, so the sums do not depend on scheduling.
// Output 0 counts the target island not switching, sigmoid(-z); the others
// their own event, sigmoid(z).  Both tails keep full relative precision.
__global__ void k_screen_accum(const float* __restrict__ z, long long r0, int nb, int J, int n_out, long long d_lo,
                               int n_d, double* __restrict__ acc) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n_d * n_out) return;
    const long long d = d_lo + warp / n_out;
    const int k = warp % n_out;
    const long long lo = max(d * J, r0), hi = min((d + 1) * J, r0 + nb);
    double sum = 0.0;
    for (long long r = lo + lane; r < hi; r += 32) {
        double x = (double)z[(r - r0) * n_out + k];
        if (k == 0) x = -x;
        const double e = exp(-fabs(x));
        sum += x >= 0.0 ? 1.0 / (1.0 + e) : e / (1.0 + e);
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) acc[d * n_out + k] += sum;
}

__global__ void k_screen_mean(double* acc, long long n, int J) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[i] /= (double)J;
}

int check_err(Mlp* m, cudaStream_t s) {
    int e = 0;
    BPM_CK(cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BPM_CK(cudaStreamSynchronize(s));
    if (e) {
        set_error("a bounded wait in the tensor-core GEMM gave up (code %d)", e);
        return BPM_ERR_TIMEOUT;
    }
    return BPM_OK;
}

}  // namespace

void free_mlp(Mlp* m) {
    if (!m) return;
    free_ws(m);
    for (auto p : m->W) cudaFree(p);
    for (auto p : m->WT) cudaFree(p);
    cudaFree(m->params);
    cudaFree(m->mom1);
    cudaFree(m->mom2);
    cudaFree(m->grad);
    cudaFree(m->loss);
    cudaFree(m->err);
    delete m;
}

static Mlp* get_mlp(bpm_ctx* ctx, int sid) {
    if (!ctx || sid < 0 || sid >= (int)ctx->mlps.size() || !ctx->mlps[sid]) {
        set_error("unknown surrogate id %d", sid);
        return nullptr;
    }
    return ctx->mlps[sid];
}

}  // namespace bpm

using namespace bpm;

extern "C" {

int bpm_surrogate_create(bpm_ctx* ctx, const bpm_mlp_cfg* cfg, const float* params, int32_t* sid) {
    if (!ctx || !cfg || !params || !sid || cfg->n_in < 1 || cfg->width < 1 || cfg->depth < 1 || cfg->depth > 6 ||
        cfg->n_out < 1 || cfg->n_in > 4096 || cfg->width > 4096 || cfg->n_out > 128) {
        set_error("bad surrogate configuration (depth 1..6, widths <= 4096, n_out <= 128)");
        return BPM_ERR_ARG;
    }
    BPM_CK(cudaSetDevice(ctx->device));
    Mlp* m = new Mlp();
    m->n_in = cfg->n_in;
    m->width = cfg->width;
    m->depth = cfg->depth;
    m->n_out = cfg->n_out;
    m->L = cfg->depth + 1;
    size_t off = 0;
    for (int l = 0; l < m->L; ++l) {
        int in = l == 0 ? m->n_in : m->width;
        int out = l == m->L - 1 ? m->n_out : m->width;
        m->in_real.push_back(in);
        m->out_real.push_back(out);
        m->out_pad.push_back(rup(out, 128));
        m->in_pad.push_back(l == 0 ? rup(in, 64) : m->out_pad[l - 1]);
        m->w_off.push_back(off);
        off += (size_t)out * in;
        m->b_off.push_back(off);
        off += out;
    }
    m->P = off;
    for (int l = 0; l < m->L; ++l) m->max_pad = std::max(m->max_pad, std::max(m->in_pad[l], m->out_pad[l]));
    int r = BPM_OK;
    auto chk = [&](int rr) {
        if (r == BPM_OK) r = rr;
    };
    chk(zalloc(&m->params, m->P));
    chk(zalloc(&m->mom1, m->P));
    chk(zalloc(&m->mom2, m->P));
    chk(zalloc(&m->grad, m->P));
    chk(zalloc(&m->loss, 1));
    chk(zalloc(&m->err, 1));
    m->W.assign(m->L, nullptr);
    m->WT.assign(m->L, nullptr);
    for (int l = 0; l < m->L && r == BPM_OK; ++l) {
        chk(zalloc(&m->W[l], (size_t)m->out_pad[l] * m->in_pad[l]));
        chk(zalloc(&m->WT[l], (size_t)m->out_pad[l] * m->in_pad[l]));
    }
    if (r == BPM_OK) {
        cudaError_t e = cudaMemcpy(m->params, params, m->P * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            set_error("parameter upload: %s", cudaGetErrorString(e));
            r = BPM_ERR_CUDA;
        }
    }
    if (r == BPM_OK) {
        int terr = 0;
        __nv_bfloat16** dW = device_ptr_table(m->W, &terr);
        __nv_bfloat16** dWT = device_ptr_table(m->WT, &terr);
        if (!terr) {
            k_publish<<<(unsigned)((m->P + 255) / 256), 256, 0, ctx->stream>>>((long long)m->P, table(m), m->params, dW,
                                                                               dWT);
            cudaStreamSynchronize(ctx->stream);
        }
        cudaFree(dW);
        cudaFree(dWT);
        if (terr || cudaGetLastError() != cudaSuccess) {
            set_error("surrogate weight publish failed");
            r = BPM_ERR_CUDA;
        }
    }
    if (r != BPM_OK) {
        free_mlp(m);
        return r;
    }
    ctx->mlps.push_back(m);
    *sid = (int32_t)ctx->mlps.size() - 1;
    return BPM_OK;
}

int bpm_surrogate_param_count(bpm_ctx* ctx, int32_t sid, int64_t* count) {
    Mlp* m = get_mlp(ctx, sid);
    if (!m || !count) return BPM_ERR_ARG;
    *count = (int64_t)m->P;
    return BPM_OK;
}

int bpm_surrogate_get_params(bpm_ctx* ctx, int32_t sid, float* out) {
    Mlp* m = get_mlp(ctx, sid);
    if (!m || !out) return BPM_ERR_ARG;
    BPM_CK(cudaSetDevice(ctx->device));
    BPM_CK(cudaStreamSynchronize(ctx->stream));
    BPM_CK(cudaMemcpy(out, m->params, m->P * sizeof(float), cudaMemcpyDeviceToHost));
    return BPM_OK;
}

static int load_batch(bpm_ctx* ctx, Mlp* m, const float* Xd, const float* Yd, int nb, int rows) {
    cudaStream_t s = ctx->stream;
    BPM_TRY(ensure_ws(m, rows));
    const long long cx = (long long)rows * (m->in_pad[0] / 8), ct = (long long)rows * m->in_pad[0];
    k_load_x<<<(unsigned)((cx + 255) / 256), 256, 0, s>>>(nb, rows, m->n_in, m->in_pad[0], Xd, m->H[0]);
    if (Yd) k_load_xt<<<(unsigned)((ct + 255) / 256), 256, 0, s>>>(nb, rows, m->n_in, m->in_pad[0], Xd, m->HT[0]);
    BPM_CK(cudaGetLastError());
    if (Yd) {
        BPM_CK(cudaMemsetAsync(m->Y, 0, sizeof(float) * (size_t)rows * m->n_out, s));
        BPM_CK(cudaMemcpyAsync(m->Y, Yd, sizeof(float) * (size_t)nb * m->n_out, cudaMemcpyDeviceToDevice, s));
    }
    return BPM_OK;
}

int bpm_surrogate_grad(bpm_ctx* ctx, int32_t sid, const float* X, const float* Y, int32_t N, float* grad,
                       float* loss) {
    Mlp* m = get_mlp(ctx, sid);
    if (!m || !X || !Y || !grad || N < 1 || N > (1 << 20)) {
        set_error("bad surrogate gradient arguments");
        return BPM_ERR_ARG;
    }
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    float *Xd = nullptr, *Yd = nullptr;
    BPM_CK(cudaMallocAsync(&Xd, sizeof(float) * (size_t)N * m->n_in, s));
    BPM_CK(cudaMallocAsync(&Yd, sizeof(float) * (size_t)N * m->n_out, s));
    BPM_CK(cudaMemcpyAsync(Xd, X, sizeof(float) * (size_t)N * m->n_in, cudaMemcpyHostToDevice, s));
    BPM_CK(cudaMemcpyAsync(Yd, Y, sizeof(float) * (size_t)N * m->n_out, cudaMemcpyHostToDevice, s));
    const int rows = rup(N, 128);
    int r = load_batch(ctx, m, Xd, Yd, N, rows);
    if (r == BPM_OK) r = forward(m, s, rows, N, false, false);
    if (r == BPM_OK) r = backward(m, s, rows, N, m->loss);
    cudaFreeAsync(Xd, s);
    cudaFreeAsync(Yd, s);
    if (r != BPM_OK) return r;
    BPM_TRY(check_err(m, s));
    BPM_CK(cudaMemcpy(grad, m->grad, m->P * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss) BPM_CK(cudaMemcpy(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return BPM_OK;
}

int bpm_surrogate_train(bpm_ctx* ctx, int32_t sid, const float* X, const float* Y, int64_t N,
                        const bpm_train_cfg* cfg, float* loss_curve) {
    Mlp* m = get_mlp(ctx, sid);
    if (!m || !X || !Y || !cfg || N < 1 || cfg->epochs < 1 || cfg->batch < 1 || cfg->batch > (1 << 16)) {
        set_error("bad surrogate training arguments");
        return BPM_ERR_ARG;
    }
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const long long steps_per_epoch = (N + cfg->batch - 1) / cfg->batch;
    const long long steps = steps_per_epoch * cfg->epochs;
    float *Xd = nullptr, *Yd = nullptr, *curve = nullptr;
    BPM_CK(cudaMallocAsync(&Xd, sizeof(float) * (size_t)N * m->n_in, s));
    BPM_CK(cudaMallocAsync(&Yd, sizeof(float) * (size_t)N * m->n_out, s));
    BPM_CK(cudaMallocAsync(&curve, sizeof(float) * (size_t)steps, s));
    BPM_CK(cudaMemcpyAsync(Xd, X, sizeof(float) * (size_t)N * m->n_in, cudaMemcpyHostToDevice, s));
    BPM_CK(cudaMemcpyAsync(Yd, Y, sizeof(float) * (size_t)N * m->n_out, cudaMemcpyHostToDevice, s));
    int r = ensure_ws(m, rup(cfg->batch, 128));
    int terr = 0;
    __nv_bfloat16** dW = device_ptr_table(m->W, &terr);
    __nv_bfloat16** dWT = device_ptr_table(m->WT, &terr);
    if (terr && r == BPM_OK) {
        set_error("pointer table upload failed");
        r = BPM_ERR_CUDA;
    }
    const LayerTable T = table(m);
    long long step = 0;
    for (int ep = 0; ep < cfg->epochs && r == BPM_OK; ++ep) {
        for (long long s0 = 0; s0 < N && r == BPM_OK; s0 += cfg->batch, ++step) {
            const int nb = (int)std::min<long long>(cfg->batch, N - s0);
            const int rows = rup(nb, 128);
            r = load_batch(ctx, m, Xd + s0 * m->n_in, Yd + s0 * m->n_out, nb, rows);
            if (r == BPM_OK) r = forward(m, s, rows, nb, false, false);
            if (r == BPM_OK) r = backward(m, s, rows, nb, curve + step);
            if (r != BPM_OK) break;
            m->t += 1;
            const double c1 = 1.0 - std::pow((double)cfg->beta1, (double)m->t);
            const double c2 = 1.0 - std::pow((double)cfg->beta2, (double)m->t);
            k_adamw<<<(unsigned)((m->P + 255) / 256), 256, 0, s>>>((long long)m->P, T, m->params, m->mom1, m->mom2,
                                                                  m->grad, cfg->lr, cfg->weight_decay, cfg->beta1,
                                                                  cfg->beta2, cfg->eps, (float)c1, (float)c2, dW, dWT);
            if (cudaGetLastError() != cudaSuccess) {
                set_error("AdamW launch failed");
                r = BPM_ERR_CUDA;
            }
        }
    }
    if (r == BPM_OK) r = check_err(m, s);
    if (r == BPM_OK && loss_curve) {
        cudaError_t e = cudaMemcpy(loss_curve, curve, sizeof(float) * (size_t)steps, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error("loss curve copy: %s", cudaGetErrorString(e));
            r = BPM_ERR_CUDA;
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(dW);
    cudaFree(dWT);
    cudaFreeAsync(Xd, s);
    cudaFreeAsync(Yd, s);
    cudaFreeAsync(curve, s);
    return r;
}

int bpm_surrogate_infer(bpm_ctx* ctx, int32_t sid, const float* X, int64_t N, float* P, int on_device) {
    Mlp* m = get_mlp(ctx, sid);
    if (!m || !X || !P || N < 1) {
        set_error("bad surrogate inference arguments");
        return BPM_ERR_ARG;
    }
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const int chunk = 65536;   // 512 row tiles per layer GEMM: enough CTAs for every SM
    const float* Xd = X;
    float* Xtmp = nullptr;
    if (!on_device) {
        BPM_CK(cudaMallocAsync(&Xtmp, sizeof(float) * (size_t)N * m->n_in, s));
        BPM_CK(cudaMemcpyAsync(Xtmp, X, sizeof(float) * (size_t)N * m->n_in, cudaMemcpyHostToDevice, s));
        Xd = Xtmp;
    }
    int r = BPM_OK;
    for (long long s0 = 0; s0 < N && r == BPM_OK; s0 += chunk) {
        const int nb = (int)std::min<long long>(chunk, N - s0);
        const int rows = rup(nb, 128);
        r = load_batch(ctx, m, Xd + s0 * m->n_in, nullptr, nb, std::max(rows, std::min(rup(chunk, 128), rows)));
        if (r == BPM_OK) r = forward(m, s, rows, nb, true, true);
        if (r == BPM_OK) {
            cudaError_t e = cudaMemcpyAsync(P + s0 * m->n_out, m->logits, sizeof(float) * (size_t)nb * m->n_out,
                                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) {
                set_error("inference copy: %s", cudaGetErrorString(e));
                r = BPM_ERR_CUDA;
            }
        }
    }
    if (Xtmp) cudaFreeAsync(Xtmp, s);
    if (r != BPM_OK) return r;
    if (!on_device) return check_err(m, s);
    return BPM_OK;
}

int bpm_surrogate_screen(bpm_ctx* ctx, int32_t sid, const float* X, int64_t n_designs, int32_t n_jitter,
                         double* rates, int on_device) {
    Mlp* m = get_mlp(ctx, sid);
    if (!m || !X || !rates || n_designs < 1 || n_jitter < 1) {
        set_error("bad surrogate screening arguments");
        return BPM_ERR_ARG;
    }
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const long long N = (long long)n_designs * n_jitter;
    const int chunk = 65536;
    const float* Xd = X;
    float* Xtmp = nullptr;
    double* acc = nullptr;
    const size_t out_bytes = sizeof(double) * (size_t)n_designs * m->n_out;
    if (!on_device) {
        BPM_CK(cudaMallocAsync(&Xtmp, sizeof(float) * (size_t)N * m->n_in, s));
        BPM_CK(cudaMemcpyAsync(Xtmp, X, sizeof(float) * (size_t)N * m->n_in, cudaMemcpyHostToDevice, s));
        Xd = Xtmp;
        BPM_CK(cudaMallocAsync(&acc, out_bytes, s));
    } else {
        acc = rates;
    }
    BPM_CK(cudaMemsetAsync(acc, 0, out_bytes, s));
    int r = BPM_OK;
    for (long long s0 = 0; s0 < N && r == BPM_OK; s0 += chunk) {
        const int nb = (int)std::min<long long>(chunk, N - s0);
        const int rows = rup(nb, 128);
        r = load_batch(ctx, m, Xd + s0 * m->n_in, nullptr, nb, std::max(rows, std::min(rup(chunk, 128), rows)));
        if (r == BPM_OK) r = forward(m, s, rows, nb, true, false);
        if (r == BPM_OK) {
            const long long d_lo = s0 / n_jitter, d_hi = (s0 + nb - 1) / n_jitter;
            const int n_d = (int)(d_hi - d_lo + 1);
            const long long threads = 32LL * n_d * m->n_out;
            k_screen_accum<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(m->logits, s0, nb, n_jitter, m->n_out,
                                                                            d_lo, n_d, acc);
            if (cudaGetLastError() != cudaSuccess) {
                set_error("screening kernel launch failed");
                r = BPM_ERR_CUDA;
            }
        }
    }
    if (r == BPM_OK) {
        const long long n = (long long)n_designs * m->n_out;
        k_screen_mean<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(acc, n, n_jitter);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(rates, acc, out_bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
            set_error("screening: %s", cudaGetErrorString(e));
            r = BPM_ERR_CUDA;
        }
    }
    if (Xtmp) cudaFreeAsync(Xtmp, s);
    if (!on_device && acc) cudaFreeAsync(acc, s);
    if (r != BPM_OK) return r;
    if (!on_device) return check_err(m, s);
    return BPM_OK;
}

int bpm_surrogate_save(bpm_ctx* ctx, int32_t sid, const char* path) {
    Mlp* m = get_mlp(ctx, sid);
    if (!m || !path) return BPM_ERR_ARG;
    BPM_CK(cudaSetDevice(ctx->device));
    BPM_CK(cudaStreamSynchronize(ctx->stream));
    std::vector<float> buf(3 * m->P);
    BPM_CK(cudaMemcpy(buf.data(), m->params, m->P * sizeof(float), cudaMemcpyDeviceToHost));
    BPM_CK(cudaMemcpy(buf.data() + m->P, m->mom1, m->P * sizeof(float), cudaMemcpyDeviceToHost));
    BPM_CK(cudaMemcpy(buf.data() + 2 * m->P, m->mom2, m->P * sizeof(float), cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    if (!f) {
        set_error("cannot open %s for writing", path);
        return BPM_ERR_ARG;
    }
    const int32_t hdr[6] = {0x424d4c50, 1, m->n_in, m->width, m->depth, m->n_out};
    long long t = m->t;
    bool ok = fwrite(hdr, sizeof(hdr), 1, f) == 1 && fwrite(&t, sizeof(t), 1, f) == 1 &&
              fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("write to %s failed", path);
        return BPM_ERR_ARG;
    }
    return BPM_OK;
}

int bpm_surrogate_load(bpm_ctx* ctx, int32_t sid, const char* path) {
    Mlp* m = get_mlp(ctx, sid);
    if (!m || !path) return BPM_ERR_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) {
        set_error("cannot open %s", path);
        return BPM_ERR_ARG;
    }
    int32_t hdr[6];
    long long t = 0;
    std::vector<float> buf(3 * m->P);
    bool ok = fread(hdr, sizeof(hdr), 1, f) == 1 && fread(&t, sizeof(t), 1, f) == 1 &&
              fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok || hdr[0] != 0x424d4c50 || hdr[2] != m->n_in || hdr[3] != m->width || hdr[4] != m->depth ||
        hdr[5] != m->n_out) {
        set_error("%s is not a surrogate of this shape", path);
        return BPM_ERR_ARG;
    }
    BPM_CK(cudaSetDevice(ctx->device));
    BPM_CK(cudaStreamSynchronize(ctx->stream));
    BPM_CK(cudaMemcpy(m->params, buf.data(), m->P * sizeof(float), cudaMemcpyHostToDevice));
    BPM_CK(cudaMemcpy(m->mom1, buf.data() + m->P, m->P * sizeof(float), cudaMemcpyHostToDevice));
    BPM_CK(cudaMemcpy(m->mom2, buf.data() + 2 * m->P, m->P * sizeof(float), cudaMemcpyHostToDevice));
    m->t = t;
    int terr = 0;
    __nv_bfloat16** dW = device_ptr_table(m->W, &terr);
    __nv_bfloat16** dWT = device_ptr_table(m->WT, &terr);
    if (!terr) {
        k_publish<<<(unsigned)((m->P + 255) / 256), 256, 0, ctx->stream>>>((long long)m->P, table(m), m->params, dW, dWT);
        cudaStreamSynchronize(ctx->stream);
    }
    cudaFree(dW);
    cudaFree(dWT);
    if (terr || cudaGetLastError() != cudaSuccess) {
        set_error("surrogate weight publish failed");
        return BPM_ERR_CUDA;
    }
    return BPM_OK;
}

int bpm_surrogate_destroy(bpm_ctx* ctx, int32_t sid) {
    Mlp* m = get_mlp(ctx, sid);
    if (!m) return BPM_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_mlp(m);
    ctx->mlps[sid] = nullptr;
    return BPM_OK;
}

}  // extern "C"
