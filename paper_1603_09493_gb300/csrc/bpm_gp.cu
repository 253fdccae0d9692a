// Efficient global optimisation (Sec. II.A; Jones, Schonlau, Welch 1998) on the
// GPU: maximin choice among random Latin hypercubes, the concentrated kriging
// likelihood for a batch of correlation-length vectors, the kriging fit, and
// the predictor, its mean squared error and the expected improvement over
// large candidate sets.  FP64 throughout: the kriging systems are small
// (n <= 2048 training designs) and nearly singular for long correlation
// lengths, where lower precision loses the variance.
//
//   R_ij = exp(-sum_k theta_k (x_ik - x_jk)^2) + nugget [i == j]
//   mu = 1'R^-1 y / 1'R^-1 1,  sigma2 = (y - mu)'R^-1(y - mu) / n,
//   nll = n ln sigma2 + ln det R
//   yhat(x) = mu + r'R^-1(y - mu),  s2 = sigma2 [1 - r'R^-1 r + (1 - 1'R^-1 r)^2 / 1'R^-1 1]
//   EI = (f_min - yhat) Phi(z) + s phi(z),  z = (f_min - yhat) / s
#include <algorithm>
#include <cmath>
#include <vector>

#include "bpm_internal.cuh"

namespace bpm {

struct Gp {
    int n = 0, d = 0;
    double mu = 0, sigma2 = 0, one_Ri_1 = 0;
    double* X = nullptr;      // [n][d]
    double* theta = nullptr;  // [d]
    double* Linv = nullptr;   // [n][n] inverse of the Cholesky factor (lower)
    double* a = nullptr;      // [n] R^-1 (y - mu)
    double* c = nullptr;      // [n] Linv 1
};

void free_gp(Gp* g) {
    if (!g) return;
    cudaFree(g->X);
    cudaFree(g->theta);
    cudaFree(g->Linv);
    cudaFree(g->a);
    cudaFree(g->c);
    delete g;
}

namespace {

constexpr int kGpThreads = 256;
constexpr int kGpMaxN = 2048, kGpMaxD = 64;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// fixed-order CTA sum, result in every thread
__device__ double cta_sum(double v, double* red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// smallest squared distance between two points of each candidate design
__global__ void __launch_bounds__(kGpThreads) k_lhs_min_d2(const double* __restrict__ C, int n, int d,
                                                           double* __restrict__ out) {
    __shared__ double red[kGpThreads / 32];
    const double* X = C + (size_t)blockIdx.x * n * d;
    double m = INFINITY;
    for (int i = 0; i < n - 1; ++i)
        for (int j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) {
                const double t = X[i * d + k] - X[j * d + k];
                s += t * t;
            }
            m = fmin(m, s);
        }
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = INFINITY;
        for (int w = 0; w < kGpThreads / 32; ++w) r = fmin(r, red[w]);
        out[blockIdx.x] = r;
    }
}

// Cholesky factor of the correlation matrix of one theta vector per CTA, in place
// in A (lower triangle, row-major [n][n]), then z = L^-1 y, w = L^-1 1 and
// nll = n ln sigma2 + ln det R.  A non-positive pivot gives nll = +inf.
__global__ void __launch_bounds__(kGpThreads) k_gp_factor(const double* __restrict__ X,
                                                          const double* __restrict__ y, int n, int d,
                                                          const double* __restrict__ theta, double nugget,
                                                          double* __restrict__ Aall, double* __restrict__ zall,
                                                          double* __restrict__ wall, double* __restrict__ nll,
                                                          double* __restrict__ stats) {
    __shared__ double red[kGpThreads / 32];
    __shared__ double th[kGpMaxD];
    __shared__ int s_fail;
    const int t = blockIdx.x;
    double* A = Aall + (size_t)t * n * n;
    double* z = zall + (size_t)t * n;
    double* w = wall + (size_t)t * n;
    for (int k = threadIdx.x; k < d; k += blockDim.x) th[k] = theta[(size_t)t * d + k];
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    // lower triangle of R
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) {
        const int i = (int)(q / n), j = (int)(q % n);
        if (j > i) continue;
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            const double u = X[i * d + k] - X[j * d + k];
            s += th[k] * u * u;
        }
        A[q] = exp(-s) + (i == j ? nugget : 0.0);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int k = 0; k < n; ++k) {
        __syncthreads();
        const double piv = A[(size_t)k * n + k];
        if (!(piv > 0.0)) {
            if (threadIdx.x == 0) s_fail = 1;
            break;
        }
        const double lkk = sqrt(piv);
        __syncthreads();                       // every thread has read the pivot
        if (threadIdx.x == 0) A[(size_t)k * n + k] = lkk;
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + k] /= lkk;
        __syncthreads();
        for (int i = k + 1 + warp; i < n; i += nwarps) {
            const double lik = A[(size_t)i * n + k];
            for (int j = k + 1 + lane; j <= i; j += 32) A[(size_t)i * n + j] -= lik * A[(size_t)j * n + k];
        }
    }
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) nll[t] = INFINITY;
        return;
    }
    // forward substitution for y and 1 together: z_i = (y_i - sum_j<i L_ij z_j) / L_ii
    for (int i = 0; i < n; ++i) {
        double sz = 0.0, sw = 0.0;
        for (int j = threadIdx.x; j < i; j += blockDim.x) {
            const double l = A[(size_t)i * n + j];
            sz += l * z[j];
            sw += l * w[j];
        }
        sz = cta_sum(sz, red);
        sw = cta_sum(sw, red);
        if (threadIdx.x == 0) {
            const double l = A[(size_t)i * n + i];
            z[i] = (y[i] - sz) / l;
            w[i] = (1.0 - sw) / l;
        }
        __syncthreads();
    }
    double ww = 0.0, wz = 0.0, ld = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        ww += w[i] * w[i];
        wz += w[i] * z[i];
        ld += log(A[(size_t)i * n + i]);
    }
    ww = cta_sum(ww, red);
    wz = cta_sum(wz, red);
    ld = cta_sum(ld, red);
    const double mu = wz / ww;
    double rr = 0.0;                           // |L^-1 (y - mu 1)|^2 = (y - mu)'R^-1(y - mu)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = z[i] - mu * w[i];
        rr += r * r;
    }
    rr = cta_sum(rr, red);
    if (threadIdx.x == 0) {
        const double sigma2 = rr / n;
        nll[t] = sigma2 > 0.0 ? n * log(sigma2) + 2.0 * ld : INFINITY;
        if (stats) {
            stats[3 * t] = mu;
            stats[3 * t + 1] = sigma2;
            stats[3 * t + 2] = ww;        // 1'R^-1 1
        }
    }
}

// column j of Linv = L^-1 by forward substitution (one thread per column)
__global__ void k_gp_linv(const double* __restrict__ L, int n, double* __restrict__ Linv) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int i = 0; i < j; ++i) Linv[(size_t)i * n + j] = 0.0;
    Linv[(size_t)j * n + j] = 1.0 / L[(size_t)j * n + j];
    for (int i = j + 1; i < n; ++i) {
        double s = 0.0;
        for (int k = j; k < i; ++k) s += L[(size_t)i * n + k] * Linv[(size_t)k * n + j];
        Linv[(size_t)i * n + j] = -s / L[(size_t)i * n + i];
    }
}

// u = Linv (y - mu 1) and c = Linv 1 (one thread per row)
__global__ void k_gp_rows(const double* __restrict__ Linv, const double* __restrict__ y, double mu, int n,
                          double* __restrict__ u, double* __restrict__ c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double su = 0.0, sc = 0.0;
    for (int j = 0; j <= i; ++j) {
        const double l = Linv[(size_t)i * n + j];
        su += l * (y[j] - mu);
        sc += l;
    }
    u[i] = su;
    c[i] = sc;
}

// a = Linv' u = R^-1 (y - mu 1) (one thread per column)
__global__ void k_gp_cols(const double* __restrict__ Linv, const double* __restrict__ u, int n,
                          double* __restrict__ a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int i = j; i < n; ++i) s += Linv[(size_t)i * n + j] * u[i];
    a[j] = s;
}

// Rc[c][i] = exp(-sum_k theta_k (C_ck - X_ik)^2)
__global__ void k_gp_corr(const double* __restrict__ C, const double* __restrict__ X,
                          const double* __restrict__ theta, int N, int n, int d, double* __restrict__ Rc) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)N * n) return;
    const int c = (int)(q / n), i = (int)(q % n);
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = C[(size_t)c * d + k] - X[(size_t)i * d + k];
        s += theta[k] * t * t;
    }
    Rc[q] = exp(-s);
}

// V[N][n] = Rc[N][n] * Linv[n][n]^T, FP64, 64 x 64 tiles, 4 x 4 outputs per thread.  B lower
// triangular: row r of B is zero past column r, so output columns n0 .. n0 + 63 need K only up
// to n0 + 64 (the skipped products are exact zeros; the sums are unchanged)
constexpr int kTM = 64, kTN = 64, kTK = 16;
__global__ void __launch_bounds__(256) k_gp_gemm_nt(const double* __restrict__ A, const double* __restrict__ B,
                                                    int M, int N, int K, double* __restrict__ Cout) {
    __shared__ double As[kTK][kTM + 1];
    __shared__ double Bs[kTK][kTN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    double acc[4][4] = {};
    const int kend = min(K, n0 + kTN);
    for (int k0 = 0; k0 < kend; k0 += kTK) {
        for (int e = threadIdx.x; e < kTM * kTK; e += 256) {
            const int r = e / kTK, kk = e % kTK;
            As[kk][r] = (m0 + r < M && k0 + kk < K) ? A[(size_t)(m0 + r) * K + k0 + kk] : 0.0;
            Bs[kk][r] = (n0 + r < N && k0 + kk < K) ? B[(size_t)(n0 + r) * K + k0 + kk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                av[q] = As[kk][ty + 16 * q];
                bv[q] = Bs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = m0 + ty + 16 * p, col = n0 + tx + 16 * q;
            if (r < M && col < N) Cout[(size_t)r * N + col] = acc[p][q];
        }
}

// predictor, MSE and expected improvement (one warp per candidate)
__global__ void k_gp_ei(const double* __restrict__ Rc, const double* __restrict__ V, const double* __restrict__ a,
                        const double* __restrict__ cvec, int N, int n, double mu, double sigma2, double one_Ri_1,
                        double f_min, double* __restrict__ yhat, double* __restrict__ s_out,
                        double* __restrict__ ei) {
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (c >= N) return;
    double sy = 0.0, q = 0.0, p = 0.0;
    for (int i = lane; i < n; i += 32) {
        const double v = V[(size_t)c * n + i];
        sy += Rc[(size_t)c * n + i] * a[i];
        q += v * v;
        p += cvec[i] * v;
    }
    sy = warp_sum(sy);
    q = warp_sum(q);
    p = warp_sum(p);
    if (lane == 0) {
        const double yh = mu + sy;
        const double s2 = sigma2 * (1.0 - q + (1.0 - p) * (1.0 - p) / one_Ri_1);
        const double s = s2 > 0.0 ? sqrt(s2) : 0.0;
        double e;
        if (s > 0.0) {
            const double z = (f_min - yh) / s;
            e = (f_min - yh) * 0.5 * (1.0 + erf(z * 0.70710678118654752)) +
                s * exp(-0.5 * z * z) * 0.39894228040143268;
        } else {
            e = fmax(f_min - yh, 0.0);
        }
        if (yhat) yhat[c] = yh;
        if (s_out) s_out[c] = s;
        if (ei) ei[c] = e;
    }
}

}  // namespace
}  // namespace bpm

using namespace bpm;

namespace {

// device buffers of one call, freed on every exit path
struct GpScratch {
    std::vector<void*> ptrs;
    template <typename T>
    int alloc(T** p, size_t count) {
        cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T));
        if (e != cudaSuccess) {
            set_error("optimiser buffers: %s", cudaGetErrorString(e));
            return BPM_ERR_OOM;
        }
        ptrs.push_back(*p);
        return BPM_OK;
    }
    template <typename T>
    int upload(T** p, const T* h, size_t count, cudaStream_t s) {
        BPM_TRY(alloc(p, count));
        BPM_CK(cudaMemcpyAsync(*p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
        return BPM_OK;
    }
    ~GpScratch() {
        for (void* p : ptrs) cudaFree(p);
    }
};

int check_design(const double* X, const double* y, int n, int d) {
    if (!X || !y || n < 2 || n > kGpMaxN || d < 1 || d > kGpMaxD) {
        set_error("kriging data: 2 <= n <= %d training designs, 1 <= d <= %d parameters", kGpMaxN, kGpMaxD);
        return BPM_ERR_ARG;
    }
    return BPM_OK;
}

int gp_of(bpm_ctx* ctx, int id, Gp** out) {
    if (!ctx || id < 0 || id >= (int)ctx->gps.size() || !ctx->gps[id]) {
        set_error("unknown kriging model %d", id);
        return BPM_ERR_ARG;
    }
    *out = ctx->gps[id];
    return BPM_OK;
}

}  // namespace

extern "C" int bpm_lhs_maximin(bpm_ctx* ctx, const double* cands, int32_t T, int32_t n, int32_t d, int32_t* best,
                               double* min_d2) {
    if (!ctx || !cands || !best || T < 1 || n < 2 || d < 1) {
        set_error("bad Latin hypercube arguments");
        return BPM_ERR_ARG;
    }
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    GpScratch sc;
    double *dC = nullptr, *dD = nullptr;
    BPM_TRY(sc.upload(&dC, cands, (size_t)T * n * d, s));
    BPM_TRY(sc.alloc(&dD, T));
    k_lhs_min_d2<<<T, kGpThreads, 0, s>>>(dC, n, d, dD);
    BPM_CK(cudaGetLastError());
    std::vector<double> h(T);
    BPM_CK(cudaMemcpyAsync(h.data(), dD, T * sizeof(double), cudaMemcpyDeviceToHost, s));
    BPM_CK(cudaStreamSynchronize(s));
    int b = 0;
    for (int t = 1; t < T; ++t)
        if (h[t] > h[b]) b = t;
    *best = b;
    if (min_d2) std::copy(h.begin(), h.end(), min_d2);
    return BPM_OK;
}

extern "C" int bpm_gp_nll(bpm_ctx* ctx, const double* X, const double* y, int32_t n, int32_t d,
                          const double* theta, int32_t T, double nugget, double* nll) {
    if (!ctx || !theta || !nll || T < 1 || !(nugget >= 0)) {
        set_error("bad likelihood arguments");
        return BPM_ERR_ARG;
    }
    BPM_TRY(check_design(X, y, n, d));
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    // theta vectors per launch: their factors together stay under 1 GiB
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(T, (size_t(1) << 30) / (8 * (size_t)n * n)));
    GpScratch sc;
    double *dX = nullptr, *dy = nullptr, *dth = nullptr, *A = nullptr, *z = nullptr, *w = nullptr, *dn = nullptr;
    BPM_TRY(sc.upload(&dX, X, (size_t)n * d, s));
    BPM_TRY(sc.upload(&dy, y, n, s));
    BPM_TRY(sc.upload(&dth, theta, (size_t)T * d, s));
    BPM_TRY(sc.alloc(&A, (size_t)chunk * n * n));
    BPM_TRY(sc.alloc(&z, (size_t)chunk * n));
    BPM_TRY(sc.alloc(&w, (size_t)chunk * n));
    BPM_TRY(sc.alloc(&dn, T));
    for (int t0 = 0; t0 < T; t0 += chunk) {
        const int m = std::min(chunk, T - t0);
        k_gp_factor<<<m, kGpThreads, 0, s>>>(dX, dy, n, d, dth + (size_t)t0 * d, nugget, A, z, w, dn + t0, nullptr);
        BPM_CK(cudaGetLastError());
    }
    BPM_CK(cudaMemcpyAsync(nll, dn, T * sizeof(double), cudaMemcpyDeviceToHost, s));
    BPM_CK(cudaStreamSynchronize(s));
    return BPM_OK;
}

extern "C" int bpm_gp_create(bpm_ctx* ctx, const double* X, const double* y, int32_t n, int32_t d,
                             const double* theta, double nugget, int32_t* gp_id, double* mu_sigma2) {
    if (!ctx || !theta || !gp_id || !(nugget >= 0)) {
        set_error("bad kriging fit arguments");
        return BPM_ERR_ARG;
    }
    BPM_TRY(check_design(X, y, n, d));
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    GpScratch sc;
    double *dy = nullptr, *A = nullptr, *z = nullptr, *w = nullptr, *dn = nullptr, *st = nullptr, *u = nullptr;
    Gp* g = new Gp();
    g->n = n;
    g->d = d;
    auto fail = [&](int r) {
        free_gp(g);
        return r;
    };
    int r = BPM_OK;
    if ((r = sc.upload(&dy, y, n, s)) || (r = sc.alloc(&A, (size_t)n * n)) || (r = sc.alloc(&z, n)) ||
        (r = sc.alloc(&w, n)) || (r = sc.alloc(&dn, 1)) || (r = sc.alloc(&st, 3)) || (r = sc.alloc(&u, n)))
        return fail(r);
    cudaError_t e = cudaMalloc(&g->X, (size_t)n * d * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&g->theta, d * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&g->Linv, (size_t)n * n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&g->a, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&g->c, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->X, X, (size_t)n * d * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->theta, theta, d * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        set_error("kriging model buffers: %s", cudaGetErrorString(e));
        return fail(BPM_ERR_OOM);
    }
    k_gp_factor<<<1, kGpThreads, 0, s>>>(g->X, dy, n, d, g->theta, nugget, A, z, w, dn, st);
    double hst[3] = {0, 0, 0}, hn = 0;
    e = cudaMemcpyAsync(hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hn, dn, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("kriging factor: %s", cudaGetErrorString(e));
        return fail(BPM_ERR_CUDA);
    }
    if (!std::isfinite(hn)) {
        set_error("correlation matrix is not positive definite at this theta and nugget");
        return fail(BPM_ERR_NONFINITE);
    }
    g->mu = hst[0];
    g->sigma2 = hst[1];
    g->one_Ri_1 = hst[2];
    const int nb = (n + 127) / 128;
    k_gp_linv<<<nb, 128, 0, s>>>(A, n, g->Linv);
    k_gp_rows<<<nb, 128, 0, s>>>(g->Linv, dy, g->mu, n, u, g->c);
    k_gp_cols<<<nb, 128, 0, s>>>(g->Linv, u, n, g->a);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("kriging fit: %s", cudaGetErrorString(e));
        return fail(BPM_ERR_CUDA);
    }
    ctx->gps.push_back(g);
    *gp_id = (int32_t)ctx->gps.size() - 1;
    if (mu_sigma2) {
        mu_sigma2[0] = g->mu;
        mu_sigma2[1] = g->sigma2;
    }
    return BPM_OK;
}

extern "C" int bpm_gp_predict(bpm_ctx* ctx, int32_t gp_id, const double* C, int64_t N, double f_min, double* yhat,
                              double* s_out, double* ei) {
    Gp* g = nullptr;
    BPM_TRY(gp_of(ctx, gp_id, &g));
    if (!C || N < 0) {
        set_error("bad prediction arguments");
        return BPM_ERR_ARG;
    }
    if (N == 0) return BPM_OK;
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const int n = g->n, d = g->d;
    const int chunk = (int)std::min<int64_t>(N, 32768);
    GpScratch sc;
    double *dC = nullptr, *Rc = nullptr, *V = nullptr, *dy = nullptr, *ds = nullptr, *de = nullptr;
    BPM_TRY(sc.alloc(&dC, (size_t)chunk * d));
    BPM_TRY(sc.alloc(&Rc, (size_t)chunk * n));
    BPM_TRY(sc.alloc(&V, (size_t)chunk * n));
    BPM_TRY(sc.alloc(&dy, chunk));
    BPM_TRY(sc.alloc(&ds, chunk));
    BPM_TRY(sc.alloc(&de, chunk));
    for (int64_t c0 = 0; c0 < N; c0 += chunk) {
        const int m = (int)std::min<int64_t>(chunk, N - c0);
        BPM_CK(cudaMemcpyAsync(dC, C + c0 * d, (size_t)m * d * sizeof(double), cudaMemcpyHostToDevice, s));
        const long long cells = (long long)m * n;
        k_gp_corr<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(dC, g->X, g->theta, m, n, d, Rc);
        k_gp_gemm_nt<<<dim3((n + kTN - 1) / kTN, (m + kTM - 1) / kTM), 256, 0, s>>>(Rc, g->Linv, m, n, n, V);
        k_gp_ei<<<(m + 7) / 8, 256, 0, s>>>(Rc, V, g->a, g->c, m, n, g->mu, g->sigma2, g->one_Ri_1, f_min, dy, ds,
                                             de);
        BPM_CK(cudaGetLastError());
        if (yhat) BPM_CK(cudaMemcpyAsync(yhat + c0, dy, m * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (s_out) BPM_CK(cudaMemcpyAsync(s_out + c0, ds, m * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (ei) BPM_CK(cudaMemcpyAsync(ei + c0, de, m * sizeof(double), cudaMemcpyDeviceToHost, s));
        BPM_CK(cudaStreamSynchronize(s));
    }
    return BPM_OK;
}

extern "C" int bpm_gp_destroy(bpm_ctx* ctx, int32_t gp_id) {
    Gp* g = nullptr;
    BPM_TRY(gp_of(ctx, gp_id, &g));
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_gp(g);
    ctx->gps[gp_id] = nullptr;
    return BPM_OK;
}
