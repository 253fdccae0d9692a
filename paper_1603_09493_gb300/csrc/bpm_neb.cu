// Energy barriers of islands in the head's fringing field by the nudged elastic
// band (Sec. II.C, adjacent-track erasure; BER_adj follows from Eq. 3).
//
// The images of every band are rows of one batch: per iteration one demag GEMM
// over all images (tensor cores for the BF16 precisions), one energy/field
// kernel and one band-update kernel, each with one CTA per image.  The band
// update is a Jacobi step (neighbours from the previous iterate), so the images
// are independent rows within an iteration.
#include <algorithm>
#include <cstring>
#include <vector>

#include "bpm_step.cuh"

namespace bpm {
namespace {

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// device buffers of one band run, freed on every exit path
struct NebBuffers {
    std::vector<void*> ptrs;
    template <typename T>
    int alloc(T** p, size_t count) {
        cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T));
        if (e != cudaSuccess) {
            set_error("band buffers: %s", cudaGetErrorString(e));
            return BPM_ERR_OOM;
        }
        ptrs.push_back(*p);
        e = cudaMemset(*p, 0, std::max<size_t>(1, count) * sizeof(T));
        if (e != cudaSuccess) {
            set_error("band buffers: %s", cudaGetErrorString(e));
            return BPM_ERR_CUDA;
        }
        return BPM_OK;
    }
    ~NebBuffers() {
        for (void* p : ptrs) cudaFree(p);
    }
};

}  // namespace
}  // namespace bpm

using namespace bpm;

extern "C" int bpm_neb_run(bpm_ctx* ctx, const bpm_island* isl, int32_t D, const bpm_neb_params* p,
                           const float* m_init, int32_t ld, double* E_path, double* E_barrier, float* m_path,
                           int32_t* iters_done, double* max_force) {
    if (!ctx || !isl || !p || D < 1 || p->n_images < 3 || p->max_iters < 0 || !(p->step > 0) ||
        !(p->spring >= 0) || !(p->force_tol >= 0)) {
        set_error("bad band arguments (D >= 1, n_images >= 3, max_iters >= 0, step > 0, spring >= 0)");
        return BPM_ERR_ARG;
    }
    const int prec = p->precision;
    if (prec != BPM_PREC_FP32 && prec != BPM_PREC_BF16X3 && prec != BPM_PREC_BF16 && prec != BPM_PREC_BF16X3_REF) {
        set_error("unknown precision %d", prec);
        return BPM_ERR_ARG;
    }
    const int mid = isl[0].mesh_id;
    if (mid < 0 || mid >= (int)ctx->meshes.size() || !ctx->meshes[mid]) {
        set_error("unknown mesh id %d", mid);
        return BPM_ERR_ARG;
    }
    for (int d = 0; d < D; ++d) {
        if (isl[d].mesh_id != mid) {
            set_error("band %d: every island of one call must share a mesh (%d != %d)", d, isl[d].mesh_id, mid);
            return BPM_ERR_ARG;
        }
        if (!(isl[d].Ms_scale > 0) || !(isl[d].Ku_scale >= 0)) {
            set_error("island %d: Ms_scale must be > 0 and Ku_scale >= 0", d);
            return BPM_ERR_ARG;
        }
    }
    const HeadMap* H = nullptr;
    if (p->map_id >= 0) {
        if (p->map_id >= (int)ctx->maps.size() || !ctx->maps[p->map_id]) {
            set_error("unknown head map id %d", p->map_id);
            return BPM_ERR_ARG;
        }
        H = ctx->maps[p->map_id];
    }
    const Mesh* M = ctx->meshes[mid];
    const int n = M->n, np = M->n_pad, K = M->K(), P = p->n_images;
    if ((m_init || m_path) && ld < n) {
        set_error("ld %d < n_nodes %d", ld, n);
        return BPM_ERR_ARG;
    }
    const int R = D * P, Rp = round_up(R, kIslandPad);
    BPM_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;

    NebBuffers buf;
    float4* d_isl = nullptr;
    float *m0 = nullptr, *m1 = nullptr, *Bt = nullptr, *Hd = nullptr, *A32 = nullptr, *fmax = nullptr;
    __nv_bfloat16 *Ahi = nullptr, *Alo = nullptr;
    double* E = nullptr;
    int* err = nullptr;
    const size_t S = (size_t)Rp * 3 * np, G = (size_t)Rp * K;
    BPM_TRY(buf.alloc(&d_isl, 3 * (size_t)R));
    BPM_TRY(buf.alloc(&m0, S));
    BPM_TRY(buf.alloc(&m1, S));
    BPM_TRY(buf.alloc(&Bt, S));
    BPM_TRY(buf.alloc(&Hd, G));
    if (prec == BPM_PREC_FP32) {
        BPM_TRY(buf.alloc(&A32, G));
    } else {
        BPM_TRY(buf.alloc(&Ahi, G));
        BPM_TRY(buf.alloc(&Alo, G));
    }
    BPM_TRY(buf.alloc(&E, R));
    BPM_TRY(buf.alloc(&fmax, R));
    BPM_TRY(buf.alloc(&err, 1));

    // island parameters, the same for every image of a band
    std::vector<float4> ip(3 * (size_t)R);
    for (int d = 0; d < D; ++d)
        for (int k = 0; k < P; ++k) {
            const bpm_island& I = isl[d];
            const size_t r = (size_t)d * P + k;
            ip[3 * r] = make_float4(1.f / I.Ms_scale, I.Ku_scale / I.Ms_scale, I.Ms_scale, 0.f);
            ip[3 * r + 1] = make_float4(I.u[0], I.u[1], I.u[2], I.pos_nm[0]);
            ip[3 * r + 2] = make_float4(I.pos_nm[1], I.Hext_T[0], I.Hext_T[1], I.Hext_T[2]);
        }
    BPM_CK(cudaMemcpyAsync(d_isl, ip.data(), ip.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    if (m_init) {
        for (int r = 0; r < R; ++r)
            BPM_CK(cudaMemcpy2DAsync(m0 + (size_t)r * 3 * np, np * sizeof(float), m_init + (size_t)r * 3 * ld,
                                     ld * sizeof(float), n * sizeof(float), 3, cudaMemcpyHostToDevice, s));
    }

    StepArgs a{};
    a.B = R;
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
    a.m = m0;
    a.Hd = Hd;
    a.A32 = A32;
    a.Ahi = Ahi;
    a.Alo = Alo;
    a.prec = prec;
    a.x0 = (float)p->head_x_nm;
    for (int c = 0; c < 3; ++c) a.uni[c] = (float)p->uniform_T[c];
    a.mask = p->term_mask;
    a.threads = 256;
    a.ipb = 1;

    GroupedGemm gg;
    const bool tc = prec == BPM_PREC_BF16X3 || prec == BPM_PREC_BF16;
    if (tc) {
        std::vector<GemmOperands> ops{GemmOperands{Ahi, Alo, M->Nhi, M->Nlo, Hd, Rp, K, K}};
        int r = grouped_gemm_setup(&gg, ops, 256, prec == BPM_PREC_BF16X3 ? 3 : 1, BPM_RASTER_AUTO, 32,
                                   ctx->l2_bytes);
        if (r != BPM_OK) {
            grouped_gemm_free(&gg);
            return r;
        }
    }
    auto demag = [&]() -> int {
        if (!(p->term_mask & BPM_TERM_DEMAG)) return BPM_OK;
        if (tc) return grouped_gemm_launch(s, gg, ctx->sm_count, err);
        if (prec == BPM_PREC_FP32) return gemm_f32_nt(s, Rp, K, K, A32, K, M->N32, K, Hd, K);
        return gemm_bf16x3_simt(s, Rp, K, K, Ahi, Alo, M->Nhi, M->Nlo, Hd, 3);
    };

    const double vol_scale = M->info.volume_nm3 * 1e-21;
    launch_neb_init(a, P, m_init ? 0 : 1, s);
    float* cur = m0;
    float* nxt = m1;
    int r = BPM_OK, it = 0;
    std::vector<float> fm(R);
    double fmax_last = 0.0;
    const int check = p->check_every > 0 ? p->check_every : 50;
    for (; it < p->max_iters && r == BPM_OK; ++it) {
        a.m = cur;
        r = demag();
        if (r != BPM_OK) break;
        launch_neb_energy(a, Bt, E, vol_scale, s);
        NebArgs nb{P, (p->climb_after >= 0 && it >= p->climb_after) ? 1 : 0, (float)p->step, (float)p->spring,
                   E, Bt, cur, nxt, fmax};
        launch_neb_step(a, nb, s);
        std::swap(cur, nxt);
        if ((it + 1) % check == 0 || it + 1 == p->max_iters) {
            cudaError_t e = cudaMemcpyAsync(fm.data(), fmax, R * sizeof(float), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                set_error("band iteration: %s", cudaGetErrorString(e));
                r = BPM_ERR_CUDA;
                break;
            }
            fmax_last = *std::max_element(fm.begin(), fm.end());
            if (p->force_tol > 0 && fmax_last < p->force_tol) {
                ++it;
                break;
            }
        }
    }
    // energies of the final band
    if (r == BPM_OK) {
        a.m = cur;
        r = demag();
    }
    if (r == BPM_OK) launch_neb_energy(a, Bt, E, vol_scale, s);
    if (tc) grouped_gemm_free(&gg);
    if (r != BPM_OK) return r;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("band run: %s", cudaGetErrorString(e));
        return BPM_ERR_CUDA;
    }
    int herr = 0;
    BPM_CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        set_error("tensor-core GEMM wait timed out (code %d)", herr);
        return BPM_ERR_TIMEOUT;
    }
    std::vector<double> Eh(R);
    BPM_CK(cudaMemcpy(Eh.data(), E, R * sizeof(double), cudaMemcpyDeviceToHost));
    if (E_path) std::memcpy(E_path, Eh.data(), R * sizeof(double));
    if (E_barrier)
        for (int d = 0; d < D; ++d) {
            double emax = Eh[(size_t)d * P + 1];
            for (int k = 2; k < P - 1; ++k) emax = std::max(emax, Eh[(size_t)d * P + k]);
            E_barrier[d] = emax - Eh[(size_t)d * P];
        }
    if (m_path)
        for (int rr = 0; rr < R; ++rr)
            BPM_CK(cudaMemcpy2D(m_path + (size_t)rr * 3 * ld, ld * sizeof(float), cur + (size_t)rr * 3 * np,
                                np * sizeof(float), n * sizeof(float), 3, cudaMemcpyDeviceToHost));
    if (iters_done) *iters_done = it;
    if (max_force) *max_force = fmax_last;
    return BPM_OK;
}
