// The plain, one-island-per-launch form of the recording simulation: every
// island is integrated on its own, with an FP32 matrix-vector demag product
// (the dense operator streamed from HBM once per Heun stage) and single-island
// stage kernels -- the straightforward GPU port of the paper's per-island runs
// (Sec. II.C runs each recording simulation as its own job).  It is the
// baseline that the batched tensor-core path is measured against, and it
// shares the stage kernels, so both forms give the same outcomes.
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

}  // namespace

}  // namespace bpm

using namespace bpm;

extern "C" int bpm_run_plain(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p,
                             int32_t n_intervals, float* m_final, int32_t ld, uint8_t* switched, float* t_sw_ps,
                             int32_t* status, double* device_ms) {
    if (!ctx || !isl || !p || B < 1 || n_intervals < 0 || p->substeps < 1 || !(p->dt_ps > 0)) {
        set_error("bad arguments to the plain run");
        return BPM_ERR_ARG;
    }
    const HeadMap* H = nullptr;
    if (p->map_id >= 0) {
        if (p->map_id >= (int)ctx->maps.size()) {
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
    BPM_CK(cudaMalloc(&buf, 5 * S * sizeof(float)));
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
        cudaMemsetAsync(buf, 0, 5 * S * sizeof(float), s);
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
        a.ms = buf + S;
        a.k1 = buf + 2 * S;
        float* hd = buf + 3 * S;
        a.Hd = hd;
        a.A32 = buf + 4 * S;
        a.prec = BPM_PREC_FP32;
        a.mz_prev = scal;
        a.t_sw = scal + 1;
        a.crossed = iscal;
        a.status = iscal + 1;
        a.interval = interval;
        a.t0 = p->t0_ps;
        a.k = p->substeps;
        a.h = p->dt_ps / p->substeps;
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
            for (int j = 0; j < p->substeps; ++j) {
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
