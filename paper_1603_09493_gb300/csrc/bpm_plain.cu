// The plain, one-island-per-launch form of the recording simulation: every
// island is integrated on its own, with an FP32 matrix-vector demag product
// (the dense operator streamed from HBM once per Heun stage) and single-island
// stage kernels -- the straightforward GPU port of the paper's per-island runs
// (Sec. II.C runs each recording simulation as its own job).  It is the
// baseline that the batched tensor-core path is measured against, and it
// shares the stage kernels, so both forms give the same outcomes.  Its FP64
// twin (bpm_run_plain_f64) computes every step in FP64 from the assembly's FP64
// operators: the GPU form of the oracle's arithmetic, one island per launch.
#include <cstring>

#include "bpm_step.cuh"

namespace bpm {

namespace {

// y[o] = sum_k W[o][k] x[k]: one warp per output row, 16-byte loads
__global__ void k_gemv_f32(int K, const float* __restrict__ W, const float* __restrict__ x, float* __restrict__ y) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= K) return;
    const float4* w4 = reinterpret_cast<const float4*>(W + (size_t)row * K);
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float s = 0.f;
    for (int q = lane; q < K / 4; q += 32) {
        float4 w = __ldg(w4 + q), v = __ldg(x4 + q);
        s += w.x * v.x + w.y * v.y + w.z * v.z + w.w * v.w;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
}

__global__ void k_plus_z(int n, int n_pad, float* m) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    m[i] = 0.f;
    m[n_pad + i] = 0.f;
    m[2 * n_pad + i] = 1.f;
}

// ---------------------------------------------------------------------------
// FP64 plain form: the same per-island recording simulation with every field
// term, the demag product, the Heun stages and the switch detector in FP64
// (the demag operator is the assembly's FP64 N, kept with BPM_MESH_KEEP_F64).
// State arrays are component-planar [3][n] (c n + i).

struct Plain64 {
    int n, k;
    unsigned mask;
    const int* rowptr;
    const int* col;
    const double* c;          // exchange, difference form: B_ex,i = (1/Ms_s) sum_e c_e (m_col - m_i)
    const NodeF64* node;      // x, y, z (nm), V_i / sum V
    const double2* mat;       // 2 Ku_i / Ms_i (T), Ms_i (A/m)
    const float4* map;        // head map voxels [nz][ny][nx], or nullptr
    int mx, my, mz;
    double mh, mox, moy, moz;
    double inv_ms, kr, ms_s;  // 1 / Ms_scale, Ku_scale / Ms_scale, Ms_scale
    double u[3], pos[2], hext[3], uni[3];
    double t0, h, alpha, gp, rise, v_nm_ps, x0;
    double *m, *ms, *k1, *M, *Bd;   // state, predictor, slope, demag source Ms m (A/m), demag field (T)
    double* det;              // mz_prev, t_sw
    int* idet;                // crossed, status
};

// y[r] = scale * sum_q W[r][q] x[q], W [R][R] row-major: one warp per row
__global__ void k_gemv_f64(int R, const double* __restrict__ W, const double* __restrict__ x, double scale,
                           double* __restrict__ y) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= R) return;
    const double* w = W + (size_t)row * R;
    double s = 0.0;
    for (int q = lane; q < R; q += 32) s += __ldg(w + q) * __ldg(x + q);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = scale * s;
}

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3(double x, double y, double z) { return D3{x, y, z}; }
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return d3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ D3 operator*(double s, D3 a) { return d3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
    return d3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ D3 unit(D3 v) {
    const double r = sqrt(dot(v, v));
    return d3(v.x / r, v.y / r, v.z / r);
}
__device__ __forceinline__ D3 load3(const double* v, int n, int i) { return d3(v[i], v[n + i], v[2 * n + i]); }
__device__ __forceinline__ void store3(double* v, int n, int i, D3 a) {
    v[i] = a.x;
    v[n + i] = a.y;
    v[2 * n + i] = a.z;
}

// trilinear interpolation of the map at (px, py, pz) nm, clamped to the grid box, in FP64
__device__ D3 trilinear64(const Plain64& a, double px, double py, double pz) {
    const double p[3] = {px, py, pz}, org[3] = {a.mox, a.moy, a.moz};
    const int dims[3] = {a.mx, a.my, a.mz};
    int i0[3];
    double w[3];
    for (int c = 0; c < 3; ++c) {
        double f = (p[c] - org[c]) / a.mh;
        f = fmin(fmax(f, 0.0), (double)(dims[c] - 1));
        const double fl = fmin(floor(f), (double)(dims[c] - 2));
        i0[c] = (int)fl;
        w[c] = f - fl;
    }
    D3 acc = d3(0, 0, 0);
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const double ww = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
                const float4 v = a.map[((size_t)(i0[2] + dz) * a.my + (i0[1] + dy)) * a.mx + (i0[0] + dx)];
                acc = acc + ww * d3(v.x, v.y, v.z);
            }
    return acc;
}

// effective field (T) at node i of the state src, with the terms in the order the
// equation lists them: exchange, anisotropy, demag, ramped head and uniform fields, H_ext
__device__ D3 field64(const Plain64& a, const double* src, int i, D3 mi, double ramp, double xh) {
    D3 B = d3(0, 0, 0);
    if (a.mask & BPM_TERM_EXCHANGE) {
        D3 s = d3(0, 0, 0);
        for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) s = s + a.c[e] * (load3(src, a.n, a.col[e]) - mi);
        B = B + a.inv_ms * s;
    }
    if (a.mask & BPM_TERM_ANISOTROPY) {
        const D3 u = d3(a.u[0], a.u[1], a.u[2]);
        B = B + ((a.mat[i].x * a.kr) * dot(mi, u)) * u;
    }
    if (a.mask & BPM_TERM_DEMAG) B = B + load3(a.Bd, a.n, i);
    if ((a.mask & BPM_TERM_HEAD) && a.map) {
        const NodeF64 q = a.node[i];
        B = B + ramp * trilinear64(a, q.x + a.pos[0] - xh, q.y + a.pos[1], q.z);
    }
    if (a.mask & BPM_TERM_UNIFORM) {
        B = B + ramp * d3(a.uni[0], a.uni[1], a.uni[2]);
        B = B + d3(a.hext[0], a.hext[1], a.hext[2]);
    }
    return B;
}

__device__ __forceinline__ D3 rhs64(const Plain64& a, D3 m, D3 B) {
    const D3 mxB = cross(m, B);
    return (-a.gp) * (mxB + a.alpha * cross(m, mxB));
}

__device__ __forceinline__ double ramp_at(const Plain64& a, double t) {
    return a.rise > 0.0 ? fmin(1.0, t / a.rise) : 1.0;
}

// FP64 sum over the CTA in a fixed order (warp shuffles, then the warps in order)
__device__ double cta_sum64(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

constexpr int kPlain64Threads = 1024;

// demag source of m and the detector's start state
__global__ void __launch_bounds__(kPlain64Threads) k_plain64_init(Plain64 a) {
    __shared__ double red[kPlain64Threads / 32];
    double mzp = 0.0;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        const D3 v = load3(a.m, a.n, i);
        store3(a.M, a.n, i, (a.mat[i].y * a.ms_s) * v);
        mzp += a.node[i].w * v.z;
    }
    const double mz = cta_sum64(mzp, red);
    if (threadIdx.x == 0) {
        a.det[0] = mz;
        a.det[1] = mz <= 0.0 ? a.t0 : -1.0;
        a.idet[0] = mz <= 0.0;
        a.idet[1] = isfinite(mz) ? 0 : BPM_ISLAND_NONFINITE;
    }
}

// predictor of integrator step `step` (t_n = t0 + step h): k1 = f(m, t_n), m* = N(m + h k1)
__global__ void __launch_bounds__(kPlain64Threads) k_plain64_stage1(Plain64 a, long long step) {
    const double tn = a.t0 + (double)step * a.h;
    const double ramp = ramp_at(a, tn), xh = a.x0 + a.v_nm_ps * tn;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        const D3 mi = load3(a.m, a.n, i);
        const D3 f = rhs64(a, mi, field64(a, a.m, i, mi, ramp, xh));
        const D3 v = unit(mi + a.h * f);
        store3(a.k1, a.n, i, f);
        store3(a.ms, a.n, i, v);
        store3(a.M, a.n, i, (a.mat[i].y * a.ms_s) * v);
    }
}

// corrector and detector: k2 = f(m*, t_n + h), m = N(m + h/2 (k1 + k2)), <m_z>, first crossing
__global__ void __launch_bounds__(kPlain64Threads) k_plain64_stage2(Plain64 a, long long step) {
    __shared__ double red[kPlain64Threads / 32];
    const double tn = a.t0 + (double)step * a.h, t = tn + a.h;
    const double ramp = ramp_at(a, t), xh = a.x0 + a.v_nm_ps * t;
    // every thread reads m* of its neighbours: all of m* is written by the predictor launch
    double mzp = 0.0;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        const D3 mi = load3(a.ms, a.n, i);
        const D3 f2 = rhs64(a, mi, field64(a, a.ms, i, mi, ramp, xh));
        const D3 v = unit(load3(a.m, a.n, i) + (0.5 * a.h) * (load3(a.k1, a.n, i) + f2));
        store3(a.m, a.n, i, v);
        store3(a.M, a.n, i, (a.mat[i].y * a.ms_s) * v);
        mzp += a.node[i].w * v.z;
    }
    const double mz = cta_sum64(mzp, red);
    if (threadIdx.x == 0) {
        const double prev = a.det[0];
        if (!a.idet[0] && mz <= 0.0) {
            a.det[1] = tn + a.h * (prev / (prev - mz));
            a.idet[0] = 1;
        }
        a.det[0] = mz;
        if (!isfinite(mz)) a.idet[1] |= BPM_ISLAND_NONFINITE;
    }
}

__global__ void k_plus_z64(int n, double* m) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    m[i] = 0.0;
    m[n + i] = 0.0;
    m[2 * n + i] = 1.0;
}

}  // namespace

}  // namespace bpm

using namespace bpm;

extern "C" int bpm_run_plain(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p,
                             int32_t n_intervals, float* m_final, int32_t ld, uint8_t* switched, float* t_sw_ps,
                             int32_t* status, double* device_ms) {
    if (!ctx || !isl || !p || B < 1 || n_intervals < 0 || p->substeps < 0 || !(p->dt_ps > 0)) {
        set_error("bad arguments to the plain run");
        return BPM_ERR_ARG;
    }
    int k_steps = 0;
    BPM_TRY(run_substeps(ctx, isl, B, p, &k_steps));
    const HeadMap* H = nullptr;
    if (p->map_id >= 0) {
        if (p->map_id >= (int)ctx->maps.size() || !ctx->maps[p->map_id]) {
            set_error("unknown head map id %d", p->map_id);
            return BPM_ERR_ARG;
        }
        H = ctx->maps[p->map_id];
    }
    for (int b = 0; b < B; ++b) {
        const int mid = isl[b].mesh_id;
        if (mid < 0 || mid >= (int)ctx->meshes.size() || !ctx->meshes[mid]) {
            set_error("island %d: unknown mesh id %d", b, mid);
            return BPM_ERR_ARG;
        }
        if (m_final && ld < ctx->meshes[mid]->n) {
            set_error("ld %d < n_nodes %d", ld, ctx->meshes[mid]->n);
            return BPM_ERR_ARG;
        }
        if (!(isl[b].Ms_scale > 0) || !(isl[b].Ku_scale >= 0)) {
            set_error("island %d: Ms_scale must be > 0 and Ku_scale >= 0", b);
            return BPM_ERR_ARG;
        }
    }
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    // one region per buffer, each large enough for a state [3][n_pad] and a GEMM row [k_pad]
    int kmax = 0;
    for (int b = 0; b < B; ++b) kmax = std::max(kmax, ctx->meshes[isl[b].mesh_id]->K());
    const size_t S = (size_t)kmax;
    float *buf = nullptr, *scal = nullptr;
    int *iscal = nullptr;
    long long* interval = nullptr;
    float4* d_isl = nullptr;
    BPM_CK(cudaMalloc(&buf, 4 * S * sizeof(float)));
    BPM_CK(cudaMalloc(&scal, 2 * sizeof(float)));
    BPM_CK(cudaMalloc(&iscal, 2 * sizeof(int)));
    BPM_CK(cudaMalloc(&interval, sizeof(long long)));
    BPM_CK(cudaMalloc(&d_isl, 3 * sizeof(float4)));
    cudaEvent_t e0, e1;
    BPM_CK(cudaEventCreate(&e0));
    BPM_CK(cudaEventCreate(&e1));
    int r = BPM_OK;
    double total_ms = 0;
    for (int b = 0; b < B && r == BPM_OK; ++b) {
        const bpm_island& I = isl[b];
        const Mesh* M = ctx->meshes[I.mesh_id];
        const int n = M->n, np = M->n_pad, K = M->K();
        float4 ip[3] = {make_float4(1.f / I.Ms_scale, I.Ku_scale / I.Ms_scale, I.Ms_scale, 0.f),
                        make_float4(I.u[0], I.u[1], I.u[2], I.pos_nm[0]),
                        make_float4(I.pos_nm[1], I.Hext_T[0], I.Hext_T[1], I.Hext_T[2])};
        cudaMemcpyAsync(d_isl, ip, sizeof(ip), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(buf, 0, 4 * S * sizeof(float), s);
        cudaMemsetAsync(interval, 0, sizeof(long long), s);
        StepArgs a{};
        a.B = 1;
        a.n = n;
        a.n_pad = np;
        a.kp = K;
        a.node_pos = M->node_pos;
        a.node_mat = M->node_mat;
        a.sell_off = M->sell_off;
        a.sell_ent = M->sell_ent;
        a.sell_il = M->sell_il;
        a.isl = d_isl;
        a.map = H ? H->B : nullptr;
        a.tex = H ? H->tex : 0;
        a.mx = H ? H->nx : 2;
        a.my = H ? H->ny : 2;
        a.mz = H ? H->nz : 2;
        a.mh = H ? H->h : 1.f;
        a.mox = H ? H->origin[0] : 0.f;
        a.moy = H ? H->origin[1] : 0.f;
        a.moz = H ? H->origin[2] : 0.f;
        a.m = buf;
        a.k1 = buf + S;
        float* hd = buf + 2 * S;
        a.Hd = hd;
        a.A32 = buf + 3 * S;
        a.prec = BPM_PREC_FP32;
        a.mz_prev = scal;
        a.t_sw = scal + 1;
        a.crossed = iscal;
        a.status = iscal + 1;
        a.interval = interval;
        a.t0 = p->t0_ps;
        a.k = k_steps;
        a.h = p->dt_ps / k_steps;
        a.alpha = (float)p->alpha;
        a.gp = (float)(kGammaPs / (1.0 + p->alpha * p->alpha));
        a.rise = (float)p->rise_ps;
        a.v_nm_ps = (float)(p->v_m_per_s * 1e-3);
        a.x0 = (float)p->x0_nm;
        for (int c = 0; c < 3; ++c) a.uni[c] = p->uniform_T[c];
        a.mask = p->term_mask;
        k_plus_z<<<(n + 255) / 256, 256, 0, s>>>(n, np, buf);
        launch_init(a, s);
        const int gblocks = (K * 32 + 255) / 256;
        cudaEventRecord(e0, s);
        for (int it = 0; it < n_intervals; ++it) {
            for (int j = 0; j < k_steps; ++j) {
                k_gemv_f32<<<gblocks, 256, 0, s>>>(K, M->N32, a.A32, hd);
                launch_stage1(a, j, s);
                k_gemv_f32<<<gblocks, 256, 0, s>>>(K, M->N32, a.A32, hd);
                launch_stage2(a, j, s);
            }
            launch_interval_tick(interval, s);
        }
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            set_error("plain run: %s", cudaGetErrorString(e));
            r = BPM_ERR_CUDA;
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        total_ms += ms;
        float sc[2];
        int is[2];
        cudaMemcpy(sc, scal, sizeof(sc), cudaMemcpyDeviceToHost);
        cudaMemcpy(is, iscal, sizeof(is), cudaMemcpyDeviceToHost);
        if (switched) switched[b] = sc[0] <= 0.f ? 1 : 0;
        if (t_sw_ps) t_sw_ps[b] = sc[1];
        if (status) status[b] = is[1];
        if (m_final)
            for (int c = 0; c < 3; ++c)
                cudaMemcpy(m_final + ((size_t)b * 3 + c) * ld, buf + (size_t)c * np, n * sizeof(float),
                           cudaMemcpyDeviceToHost);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("plain run copy failed");
            r = BPM_ERR_CUDA;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(scal);
    cudaFree(iscal);
    cudaFree(interval);
    cudaFree(d_isl);
    if (device_ms) *device_ms = total_ms;
    return r;
}

extern "C" int bpm_run_plain_f64(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p,
                                 int32_t n_intervals, double* m_final, int32_t ld, uint8_t* switched,
                                 double* t_sw_ps, int32_t* status, double* device_ms) {
    if (!ctx || !isl || !p || B < 1 || n_intervals < 0 || p->substeps < 0 || !(p->dt_ps > 0)) {
        set_error("bad arguments to the plain FP64 run");
        return BPM_ERR_ARG;
    }
    int k_steps = 0;
    BPM_TRY(run_substeps(ctx, isl, B, p, &k_steps));
    const HeadMap* H = nullptr;
    if (p->map_id >= 0) {
        if (p->map_id >= (int)ctx->maps.size() || !ctx->maps[p->map_id]) {
            set_error("unknown head map id %d", p->map_id);
            return BPM_ERR_ARG;
        }
        H = ctx->maps[p->map_id];
    }
    int nmax = 0;
    for (int b = 0; b < B; ++b) {
        const int mid = isl[b].mesh_id;
        if (mid < 0 || mid >= (int)ctx->meshes.size() || !ctx->meshes[mid]) {
            set_error("island %d: unknown mesh id %d", b, mid);
            return BPM_ERR_ARG;
        }
        const Mesh* M = ctx->meshes[mid];
        if (!M->N64) {
            set_error("mesh %d: the FP64 demag operator was not kept (upload with BPM_MESH_KEEP_F64)", mid);
            return BPM_ERR_STATE;
        }
        if (m_final && ld < M->n) {
            set_error("ld %d < n_nodes %d", ld, M->n);
            return BPM_ERR_ARG;
        }
        if (!(isl[b].Ms_scale > 0) || !(isl[b].Ku_scale >= 0)) {
            set_error("island %d: Ms_scale must be > 0 and Ku_scale >= 0", b);
            return BPM_ERR_ARG;
        }
        nmax = std::max(nmax, M->n);
    }
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const size_t S = 3 * (size_t)nmax;
    double *buf = nullptr, *det = nullptr;
    int* idet = nullptr;
    BPM_CK(cudaMalloc(&buf, 5 * S * sizeof(double)));
    BPM_CK(cudaMalloc(&det, 2 * sizeof(double)));
    BPM_CK(cudaMalloc(&idet, 2 * sizeof(int)));
    cudaEvent_t e0, e1;
    BPM_CK(cudaEventCreate(&e0));
    BPM_CK(cudaEventCreate(&e1));
    int r = BPM_OK;
    double total_ms = 0;
    std::vector<double> mh(S);
    for (int b = 0; b < B && r == BPM_OK; ++b) {
        const bpm_island& I = isl[b];
        const Mesh* M = ctx->meshes[I.mesh_id];
        const int n = M->n, R = 3 * n;
        Plain64 a{};
        a.n = n;
        a.k = k_steps;
        a.mask = p->term_mask;
        a.rowptr = M->csr_rowptr;
        a.col = M->csr_col;
        a.c = M->csr_c64;
        a.node = M->node64;
        a.mat = M->mat64;
        a.map = H ? H->B : nullptr;
        a.mx = H ? H->nx : 2;
        a.my = H ? H->ny : 2;
        a.mz = H ? H->nz : 2;
        a.mh = H ? H->h : 1.0;
        a.mox = H ? H->origin[0] : 0.0;
        a.moy = H ? H->origin[1] : 0.0;
        a.moz = H ? H->origin[2] : 0.0;
        a.ms_s = I.Ms_scale;
        a.inv_ms = 1.0 / (double)I.Ms_scale;
        a.kr = (double)I.Ku_scale / (double)I.Ms_scale;
        for (int c = 0; c < 3; ++c) {
            a.u[c] = I.u[c];
            a.hext[c] = I.Hext_T[c];
            a.uni[c] = p->uniform_T[c];
        }
        a.pos[0] = I.pos_nm[0];
        a.pos[1] = I.pos_nm[1];
        a.t0 = p->t0_ps;
        a.h = p->dt_ps / k_steps;
        a.alpha = p->alpha;
        a.gp = kGammaPs / (1.0 + p->alpha * p->alpha);
        a.rise = p->rise_ps;
        a.v_nm_ps = p->v_m_per_s * 1e-3;
        a.x0 = p->x0_nm;
        a.m = buf;
        a.ms = buf + S;
        a.k1 = buf + 2 * S;
        a.M = buf + 3 * S;
        a.Bd = buf + 4 * S;
        a.det = det;
        a.idet = idet;
        cudaMemsetAsync(buf, 0, 5 * S * sizeof(double), s);
        k_plus_z64<<<(n + 255) / 256, 256, 0, s>>>(n, a.m);
        k_plain64_init<<<1, kPlain64Threads, 0, s>>>(a);
        const int gblocks = (R * 32 + 255) / 256;
        const double demag = (p->term_mask & BPM_TERM_DEMAG) ? -kMu0 : 0.0;
        cudaEventRecord(e0, s);
        for (int it = 0; it < n_intervals; ++it)
            for (int j = 0; j < k_steps; ++j) {
                const long long step = (long long)it * k_steps + j;
                if (demag != 0.0) k_gemv_f64<<<gblocks, 256, 0, s>>>(R, M->N64, a.M, demag, a.Bd);
                k_plain64_stage1<<<1, kPlain64Threads, 0, s>>>(a, step);
                if (demag != 0.0) k_gemv_f64<<<gblocks, 256, 0, s>>>(R, M->N64, a.M, demag, a.Bd);
                k_plain64_stage2<<<1, kPlain64Threads, 0, s>>>(a, step);
            }
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("plain FP64 run: %s", cudaGetErrorString(e));
            r = BPM_ERR_CUDA;
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        total_ms += ms;
        double dh[2];
        int ih[2];
        e = cudaMemcpy(dh, det, sizeof(dh), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(ih, idet, sizeof(ih), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && m_final) e = cudaMemcpy(mh.data(), a.m, R * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error("plain FP64 run copy: %s", cudaGetErrorString(e));
            r = BPM_ERR_CUDA;
            break;
        }
        if (switched) switched[b] = dh[0] <= 0.0 ? 1 : 0;
        if (t_sw_ps) t_sw_ps[b] = dh[1];
        if (status) status[b] = ih[1];
        if (m_final)
            for (int c = 0; c < 3; ++c)
                std::memcpy(m_final + ((size_t)b * 3 + c) * ld, mh.data() + (size_t)c * n, n * sizeof(double));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(det);
    cudaFree(idet);
    if (device_ms) *device_ms = total_ms;
    return r;
}
