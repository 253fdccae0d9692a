// Allocation-free LLG advance.
//
// Some callers cannot allocate device memory at the point where they need to
// step islands: a host application whose own pool allocator has reserved the
// device memory (a cudaMalloc from here would fail or fragment its pool), or a
// time-critical loop that must not stall on cudaMalloc/cudaFree, which can
// synchronise the device.  For them this file provides one entry point that
// runs the FP32 batch advance with all of its scratch (island table, Heun
// stages, demag operand and field, detector state, step counter) in a
// file-scope device array of fixed size.  The caller passes its state in and
// gets it back in place; the mesh operators are the ones uploaded earlier.
//
// The array is a static __device__ symbol: every GPU that loads the library
// holds it until the process exits.  Host code cannot use the symbol's name as
// a device address (it names a host-side stand-in), so the address is looked
// up once per device with cudaGetSymbolAddress while that device is current.
#include <mutex>

#include "bpm_step.cuh"

namespace bpm {

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[BPM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// device address of the scratch array on the current device (looked up once per device)
int scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) {
        set_error("device index %d out of range for the allocation-free scratch table", device);
        return BPM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the allocation-free scratch failed: %s", cudaGetErrorString(e));
            return BPM_ERR_CUDA;
        }
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return BPM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

}  // namespace bpm

using namespace bpm;

extern "C" int bpm_llg_advance_noalloc(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p,
                                       int32_t n_intervals, float* m, int32_t ld, float* mz) {
    if (!ctx || !isl || !p || !m || B < 1 || n_intervals < 0) {
        set_error("bad arguments to the allocation-free advance");
        return BPM_ERR_ARG;
    }
    const int mid = isl[0].mesh_id;
    if (mid < 0 || mid >= (int)ctx->meshes.size() || !ctx->meshes[mid]) {
        set_error("unknown mesh id %d", mid);
        return BPM_ERR_ARG;
    }
    for (int b = 1; b < B; ++b)
        if (isl[b].mesh_id != mid) {
            set_error("all islands must share one mesh (island %d)", b);
            return BPM_ERR_ARG;
        }
    if (p->precision != BPM_PREC_FP32) {
        set_error("the allocation-free advance computes the demag product in FP32 only (precision %d given)",
                  p->precision);
        return BPM_ERR_ARG;
    }
    if (p->substeps < 0 || !(p->dt_ps > 0)) {
        set_error("bad run parameters (substeps >= 0, dt > 0)");
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
    const Mesh* M = ctx->meshes[mid];
    const int n = M->n, np = M->n_pad, K = M->K();
    if (ld < n) {
        set_error("ld %d < n_nodes %d", ld, n);
        return BPM_ERR_ARG;
    }
    // scratch layout
    const size_t state = (size_t)B * K * sizeof(float);
    size_t off = 0;
    const size_t o_isl = off;
    off = align256(off + 3 * (size_t)B * sizeof(float4));
    const size_t o_m = off;
    off = align256(off + state);
    const size_t o_k1 = off;
    off = align256(off + state);
    const size_t o_hd = off;
    off = align256(off + state);
    const size_t o_a = off;
    off = align256(off + state);
    const size_t o_mzp = off;
    off = align256(off + B * sizeof(float));
    const size_t o_tsw = off;
    off = align256(off + B * sizeof(float));
    const size_t o_cr = off;
    off = align256(off + B * sizeof(int));
    const size_t o_st = off;
    off = align256(off + B * sizeof(int));
    const size_t o_it = off;
    off = align256(off + sizeof(long long));
    if (off > (size_t)BPM_NOALLOC_SCRATCH_BYTES) {
        set_error("allocation-free advance: %d islands of a %d-node mesh need %zu bytes of scratch, more than the "
                  "%d-byte maximum (use fewer islands per call)",
                  B, n, off, (int)BPM_NOALLOC_SCRATCH_BYTES);
        return BPM_ERR_ARG;
    }
    std::vector<float4> ip(3 * (size_t)B);
    for (int b = 0; b < B; ++b) {
        const bpm_island& I = isl[b];
        if (!(I.Ms_scale > 0) || !(I.Ku_scale >= 0)) {
            set_error("island %d: Ms_scale must be > 0 and Ku_scale >= 0", b);
            return BPM_ERR_ARG;
        }
        ip[3 * b] = make_float4(1.f / I.Ms_scale, I.Ku_scale / I.Ms_scale, I.Ms_scale, 0.f);
        ip[3 * b + 1] = make_float4(I.u[0], I.u[1], I.u[2], I.pos_nm[0]);
        ip[3 * b + 2] = make_float4(I.pos_nm[1], I.Hext_T[0], I.Hext_T[1], I.Hext_T[2]);
    }
    BPM_CK(cudaSetDevice(ctx->device));
    void* base = nullptr;
    BPM_TRY(scratch_address(ctx->device, &base));
    unsigned char* s8 = static_cast<unsigned char*>(base);
    cudaStream_t s = ctx->stream;
    // the array keeps the previous call's contents: clear the whole region this call uses
    BPM_CK(cudaMemsetAsync(s8, 0, off, s));
    BPM_CK(cudaMemcpyAsync(s8 + o_isl, ip.data(), ip.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    float* m_in = reinterpret_cast<float*>(s8 + o_m);
    BPM_CK(cudaMemcpy2DAsync(m_in, np * sizeof(float), m, ld * sizeof(float), n * sizeof(float), 3 * (size_t)B,
                             cudaMemcpyDeviceToDevice, s));
    StepArgs a{};
    a.B = B;
    a.n = n;
    a.n_pad = np;
    a.kp = K;
    a.node_pos = M->node_pos;
    a.node_mat = M->node_mat;
    a.sell_off = M->sell_off;
    a.sell_ent = M->sell_ent;
    a.sell_il = M->sell_il;
    a.isl = reinterpret_cast<const float4*>(s8 + o_isl);
    a.map = H ? H->B : nullptr;
    a.tex = H ? H->tex : 0;
    a.mx = H ? H->nx : 2;
    a.my = H ? H->ny : 2;
    a.mz = H ? H->nz : 2;
    a.mh = H ? H->h : 1.f;
    a.mox = H ? H->origin[0] : 0.f;
    a.moy = H ? H->origin[1] : 0.f;
    a.moz = H ? H->origin[2] : 0.f;
    a.m = m_in;
    a.k1 = reinterpret_cast<float*>(s8 + o_k1);
    float* hd = reinterpret_cast<float*>(s8 + o_hd);
    a.Hd = hd;
    a.A32 = reinterpret_cast<float*>(s8 + o_a);
    a.prec = BPM_PREC_FP32;
    a.mz_prev = reinterpret_cast<float*>(s8 + o_mzp);
    a.t_sw = reinterpret_cast<float*>(s8 + o_tsw);
    a.crossed = reinterpret_cast<int*>(s8 + o_cr);
    a.status = reinterpret_cast<int*>(s8 + o_st);
    long long* interval = reinterpret_cast<long long*>(s8 + o_it);
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
    launch_init(a, s);
    for (int it = 0; it < n_intervals; ++it) {
        for (int j = 0; j < k_steps; ++j) {
            BPM_TRY(gemm_f32_nt(s, B, K, K, a.A32, K, M->N32, K, hd, K));
            launch_stage1(a, j, s);
            BPM_TRY(gemm_f32_nt(s, B, K, K, a.A32, K, M->N32, K, hd, K));
            launch_stage2(a, j, s);
        }
        launch_interval_tick(interval, s);
    }
    BPM_CK(cudaGetLastError());
    BPM_CK(cudaMemcpy2DAsync(m, ld * sizeof(float), m_in, np * sizeof(float), n * sizeof(float), 3 * (size_t)B,
                             cudaMemcpyDeviceToDevice, s));
    if (mz) BPM_CK(cudaMemcpyAsync(mz, a.mz_prev, B * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return BPM_OK;
}
