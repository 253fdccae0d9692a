// C ABI of libbpmllg.so: contexts, mesh and head-map upload, batched LLG runs.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "bpm_step.cuh"

namespace bpm {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Heun's explicit step is stable on the fastest precession mode when
// gamma/(1+alpha^2) |B| h <= 1/2; k is the smallest step count per output
// interval that keeps h = dt/k there for the largest field the run can see.
static int substeps_for_bound(double bound_T, double dt_ps, double alpha) {
    const double gp = kGammaPs / (1.0 + alpha * alpha);
    const double k = std::ceil(gp * bound_T * dt_ps / 0.5);
    return k < 1.0 ? 1 : (int)k;
}

int stable_substeps(bpm_ctx* ctx, const bpm_island* isl, int B, const bpm_run_params* p, int* k, double* bound) {
    if (!ctx || !isl || !p || B < 1 || !(p->dt_ps > 0) || !(p->alpha >= 0)) {
        set_error("bad step-count arguments (B >= 1, dt > 0, alpha >= 0)");
        return BPM_ERR_ARG;
    }
    const HeadMap* H = nullptr;
    if (p->map_id >= 0) {
        if (p->map_id >= (int)ctx->maps.size() || !ctx->maps[p->map_id]) {
            set_error("unknown head map id %d", p->map_id);
            return BPM_ERR_ARG;
        }
        H = ctx->maps[p->map_id];
    }
    const double uni = std::sqrt((double)p->uniform_T[0] * p->uniform_T[0] + (double)p->uniform_T[1] * p->uniform_T[1] +
                                 (double)p->uniform_T[2] * p->uniform_T[2]);
    // the bound of each mesh over its own islands; the run's bound is the largest
    struct Ext {
        int mesh;
        double ms_min, ms_max, kr_max, hext_max;
    };
    std::vector<Ext> ext;
    for (int b = 0; b < B; ++b) {
        const bpm_island& I = isl[b];
        const int mid = I.mesh_id;
        if (mid < 0 || mid >= (int)ctx->meshes.size() || !ctx->meshes[mid]) {
            set_error("island %d: unknown mesh id %d", b, mid);
            return BPM_ERR_ARG;
        }
        if (!(I.Ms_scale > 0) || !(I.Ku_scale >= 0)) {
            set_error("island %d: Ms_scale must be > 0 and Ku_scale >= 0", b);
            return BPM_ERR_ARG;
        }
        const double ms = I.Ms_scale, kr = (double)I.Ku_scale / (double)I.Ms_scale;
        const double he = std::sqrt((double)I.Hext_T[0] * I.Hext_T[0] + (double)I.Hext_T[1] * I.Hext_T[1] +
                                    (double)I.Hext_T[2] * I.Hext_T[2]);
        size_t g = 0;
        while (g < ext.size() && ext[g].mesh != mid) ++g;
        if (g == ext.size()) {
            ext.push_back(Ext{mid, ms, ms, kr, he});
            continue;
        }
        Ext& e = ext[g];
        e.ms_min = std::min(e.ms_min, ms);
        e.ms_max = std::max(e.ms_max, ms);
        e.kr_max = std::max(e.kr_max, kr);
        e.hext_max = std::max(e.hext_max, he);
    }
    double best = 0;
    for (const Ext& e : ext) {
        const Mesh* M = ctx->meshes[e.mesh];
        double b = M->info.exchange_lambda_max_T / e.ms_min;   // exchange: lambda_max of S, divided by the Ms factor
        b += M->an_max * e.kr_max;                             // anisotropy 2 Ku/Ms x Ku_s/Ms_s
        b += kMu0 * M->ms_max * e.ms_max;                      // demag: |mu0 H_d| <= mu0 Ms
        if (H) b += H->max_norm;                               // head map
        b += uni + e.hext_max;                                 // uniform and per-island constant fields
        best = std::max(best, b);
    }
    *k = substeps_for_bound(best, p->dt_ps, p->alpha);
    if (bound) *bound = best;
    return BPM_OK;
}

int run_substeps(bpm_ctx* ctx, const bpm_island* isl, int B, const bpm_run_params* p, int* k) {
    if (p->substeps < 0) {
        set_error("substeps %d < 0 (0 picks the stable count)", p->substeps);
        return BPM_ERR_ARG;
    }
    if (p->substeps > 0) {
        *k = p->substeps;
        return BPM_OK;
    }
    return stable_substeps(ctx, isl, B, p, k, nullptr);
}

}  // namespace bpm

using namespace bpm;

// One mesh's share of a batch: its islands, state and demag buffers.
struct Group {
    Mesh* mesh = nullptr;
    int B = 0, Bp = 0;
    std::vector<int> user_idx;    // batch island index of each group row
    int* d_idx = nullptr;
    float4* isl = nullptr;
    float *m = nullptr, *k1 = nullptr, *Hd = nullptr, *A32 = nullptr;
    __nv_bfloat16 *Ahi = nullptr, *Alo = nullptr;
    float *mz_prev = nullptr, *t_sw = nullptr;
    int *crossed = nullptr, *status = nullptr;
    StepArgs args{};
};

struct bpm_batch {
    bpm_ctx* ctx = nullptr;
    HeadMap* map = nullptr;
    int B = 0, n_max = 0;
    bpm_run_params p{};
    std::vector<Group> groups;
    int* gemm_err = nullptr;
    long long* interval = nullptr;
    long long intervals_done = 0;
    double t0 = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaStream_t> side;   // fork streams for the groups of a multi-mesh batch
    std::vector<cudaEvent_t> ev;
    int tile_n = 256;                 // demag GEMM output columns per CTA
    int raster = BPM_RASTER_AUTO;     // demag GEMM tile order
    int k_block = 32;                 // demag GEMM K depth per pipeline stage
    int pair = 0;                     // demag GEMM on CTA pairs (256 x 256 tiles)
    GroupedGemm gg;                   // tensor-core demag GEMM over all groups (BF16 precisions)
    // multi-stream intervals (tuning streams = 2 .. 4): consecutive chunks of `chunk` islands
    // (the last one shorter) of the one group run as `chains` chains, chain c > 0 on
    // chain_stream[c - 1]; chains = 0 when the mode is off
    int streams = 2;
    int chains = 0, chunk = 0;
    GroupedGemm gg_chain[kMaxChains];
    StepArgs chain_args[kMaxChains]{};          // chunk views of the one group
    std::vector<int> chain_groups[kMaxChains];  // the groups of each chain of a multi-mesh batch
    cudaStream_t chain_stream[kMaxChains - 1] = {};
    cudaEvent_t chain_ev[kMaxChains] = {};
};

namespace {

std::vector<bpm_batch*>& live_batches(bpm_ctx* ctx) {
    static std::vector<std::pair<bpm_ctx*, std::vector<bpm_batch*>>> all;
    for (auto& e : all)
        if (e.first == ctx) return e.second;
    all.push_back({ctx, {}});
    return all.back().second;
}

int ensure_device(bpm_ctx* ctx) {
    BPM_CK(cudaSetDevice(ctx->device));
    return BPM_OK;
}

Mesh* get_mesh(bpm_ctx* ctx, int id) {
    if (!ctx || id < 0 || id >= (int)ctx->meshes.size() || !ctx->meshes[id]) {
        set_error("unknown mesh id %d", id);
        return nullptr;
    }
    return ctx->meshes[id];
}

bool tensor_core_precision(const bpm_batch* bt) {
    return bt->p.precision == BPM_PREC_BF16X3 || bt->p.precision == BPM_PREC_BF16;
}

// (re)encode the grouped tensor-core GEMM of the batch for its current tile width
int setup_grouped_gemm(bpm_batch* bt) {
    std::vector<GemmOperands> ops;
    for (auto& g : bt->groups) {
        const int K = g.mesh->K();
        ops.push_back(GemmOperands{g.Ahi, g.Alo, g.mesh->Nhi, g.mesh->Nlo, g.Hd, g.Bp, K, K});
    }
    return grouped_gemm_setup(&bt->gg, ops, bt->tile_n, bt->p.precision == BPM_PREC_BF16X3 ? 3 : 1, bt->raster,
                              bt->k_block, bt->ctx->l2_bytes, bt->pair);
}

// The chains of a multi-stream batch: the one group's islands cut into `streams` chunks of a
// multiple of 128 islands (the GEMM's M tile; the last chunk takes the rest), each with its own
// GEMM over its operand rows and its own view of the stage arguments.  chains stays 0 where the
// mode does not apply (another precision, several meshes, fewer than two chunks).
int setup_chains(bpm_batch* bt) {
    for (auto& h : bt->gg_chain) grouped_gemm_free(&h);
    bt->chains = 0;
    for (auto& v : bt->chain_groups) v.clear();
    if (bt->streams < 2 || !tensor_core_precision(bt)) return BPM_OK;
    const int ng = (int)bt->groups.size();
    const int chunk = ng > 1 ? 0 : kIslandPad * ((bt->groups[0].B + bt->streams * kIslandPad - 1) /
                                                 (bt->streams * kIslandPad));
    const int chains = ng > 1 ? std::min(bt->streams, ng) : (bt->groups[0].B + chunk - 1) / chunk;
    if (chains < 2) return BPM_OK;
    for (int c = 0; c < kMaxChains - 1; ++c)
        if (!bt->chain_stream[c] && cudaStreamCreateWithFlags(&bt->chain_stream[c], cudaStreamNonBlocking) !=
                                        cudaSuccess) {
            set_error("stream creation failed");
            return BPM_ERR_CUDA;
        }
    for (auto& e : bt->chain_ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            set_error("event creation failed");
            return BPM_ERR_CUDA;
        }
    const int products = bt->p.precision == BPM_PREC_BF16X3 ? 3 : 1;
    if (ng > 1) {
        // a multi-mesh batch: its groups dealt to the chains, largest GEMM first, each to the chain
        // with the least GEMM work so far (rows x K^2)
        std::vector<int> order(ng);
        for (int i = 0; i < ng; ++i) order[i] = i;
        auto work = [&](int i) { return (double)bt->groups[i].Bp * bt->groups[i].mesh->K() * bt->groups[i].mesh->K(); };
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
        std::vector<double> load(chains, 0.0);
        for (int i : order) {
            const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            bt->chain_groups[c].push_back(i);
            load[c] += work(i);
        }
        for (int c = 0; c < chains; ++c) {
            std::vector<GemmOperands> ops;
            for (int i : bt->chain_groups[c]) {
                const Group& q = bt->groups[i];
                const int K = q.mesh->K();
                ops.push_back(GemmOperands{q.Ahi, q.Alo, q.mesh->Nhi, q.mesh->Nlo, q.Hd, q.Bp, K, K});
            }
            BPM_TRY(grouped_gemm_setup(&bt->gg_chain[c], ops, bt->tile_n, products, bt->raster, bt->k_block,
                                       bt->ctx->l2_bytes, bt->pair));
        }
        bt->chains = chains;
        return BPM_OK;
    }
    Group& g = bt->groups[0];
    const int K = g.mesh->K();
    for (int c = 0; c < chains; ++c) {
        const int b0 = c * chunk;
        const int rows = c + 1 < chains ? chunk : g.Bp - b0;   // the last chunk's GEMM covers the padding
        const size_t off = (size_t)b0 * K, S = (size_t)b0 * 3 * g.mesh->n_pad;
        std::vector<GemmOperands> ops{GemmOperands{g.Ahi + off, g.Alo + off, g.mesh->Nhi, g.mesh->Nlo, g.Hd + off,
                                                   rows, K, K}};
        BPM_TRY(grouped_gemm_setup(&bt->gg_chain[c], ops, bt->tile_n, products, bt->raster, bt->k_block,
                                   bt->ctx->l2_bytes, bt->pair));
        StepArgs a = g.args;
        a.B = std::min(chunk, g.B - b0);
        a.isl += 3 * (size_t)b0;
        a.m += S;
        a.k1 += S;
        a.Hd += off;
        if (a.A32) a.A32 += off;
        if (a.Ahi) a.Ahi += off;
        if (a.Alo) a.Alo += off;
        a.mz_prev += b0;
        a.t_sw += b0;
        a.crossed += b0;
        a.status += b0;
        bt->chain_args[c] = a;
    }
    bt->chains = chains;
    bt->chunk = chunk;
    return BPM_OK;
}

// demag GEMM of every group's current operand A -> Hd: one persistent launch
// on the tensor cores, or one CUDA-core launch per group
int run_demag_all(bpm_batch* bt, cudaStream_t s);

// demag GEMM of a group's current operand A -> Hd (CUDA-core precisions)
int run_demag_gemm(bpm_batch* bt, Group& g, cudaStream_t s) {
    Mesh* M = g.mesh;
    const int K = M->K();
    switch (bt->p.precision) {
        case BPM_PREC_FP32:
            return gemm_f32_nt(s, g.Bp, K, K, g.A32, K, M->N32, K, g.Hd, K);
        case BPM_PREC_BF16X3_REF:
            return gemm_bf16x3_simt(s, g.Bp, K, K, g.Ahi, g.Alo, M->Nhi, M->Nlo, g.Hd, 3);
        default:
            set_error("unknown precision %d", bt->p.precision);
            return BPM_ERR_ARG;
    }
}

int run_demag_all(bpm_batch* bt, cudaStream_t s) {
    if (tensor_core_precision(bt)) return grouped_gemm_launch(s, bt->gg, bt->ctx->sm_count, bt->gemm_err);
    for (auto& g : bt->groups) BPM_TRY(run_demag_gemm(bt, g, s));
    return BPM_OK;
}

int enqueue_group_interval(bpm_batch* bt, Group& g, cudaStream_t s) {
    for (int j = 0; j < bt->p.substeps; ++j) {
        BPM_TRY(run_demag_gemm(bt, g, s));
        launch_stage1(g.args, j, s);
        BPM_TRY(run_demag_gemm(bt, g, s));
        launch_stage2(g.args, j, s);
    }
    return BPM_OK;
}

// Stage launches of a multi-group batch: the groups, largest mesh first, cut into
// classes within which every group keeps the resident CTAs per SM it would have
// in a launch of its own (the class's shared memory is its largest group's).
struct StageLaunches {
    std::vector<StageGroups> launch;
    std::vector<size_t> smem;
    int threads = 256;
};

int build_stage_launches(const bpm_batch* bt, StageLaunches* out, const std::vector<int>* subset = nullptr) {
    out->launch.clear();
    out->smem.clear();
    out->threads = bt->groups[0].args.threads;
    const int ipb = stage_islands_per_cta(bt->groups[0].args);
    std::vector<int> order;
    if (subset) {
        order = *subset;
    } else {
        order.resize(bt->groups.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return bt->groups[x].mesh->n_pad > bt->groups[y].mesh->n_pad;
    });
    int class_occ = -1;
    for (int gi : order) {
        const Group& g = bt->groups[gi];
        const size_t sb = ipb * stage_smem_bytes(g.args);
        int occ = 0;
        BPM_TRY(stage_blocks_per_sm(out->threads, ipb, sb, &occ));
        if (out->launch.empty() || occ != class_occ || out->launch.back().ng == kMaxStageGroups) {
            out->launch.emplace_back();
            std::memset(&out->launch.back(), 0, sizeof(StageGroups));
            out->smem.push_back(sb);
            class_occ = occ;
        }
        StageGroups& G = out->launch.back();
        G.a[G.ng] = g.args;
        G.block_begin[G.ng + 1] = G.block_begin[G.ng] + (g.B + ipb - 1) / ipb;
        ++G.ng;
    }
    return BPM_OK;
}

// Heun stage (1 or 2) of every group: one launch per group of a single-group
// batch, one launch per class otherwise
void launch_stage_all(bpm_batch* bt, const StageLaunches& L, int stage, int j, cudaStream_t s) {
    if (bt->groups.size() == 1) {
        if (stage == 1)
            launch_stage1(bt->groups[0].args, j, s);
        else
            launch_stage2(bt->groups[0].args, j, s);
        return;
    }
    for (size_t c = 0; c < L.launch.size(); ++c) {
        if (stage == 1)
            launch_stage1_groups(L.launch[c], L.threads, L.smem[c], j, s);
        else
            launch_stage2_groups(L.launch[c], L.threads, L.smem[c], j, s);
    }
}

// one output interval of every group; groups of a multi-mesh batch are forked
// over side streams so that their kernels can run concurrently
int enqueue_interval(bpm_batch* bt, cudaStream_t s) {
    if (bt->chains > 0) {
        // one chain per chunk of islands: chunk 0 on s, chunk c on chain_stream[c - 1] (forked
        // from and joined into s); each chain runs the Heun steps of its own islands in order, so
        // one chain's GEMM can run while another chain's stage kernels do
        BPM_CK(cudaEventRecord(bt->chain_ev[0], s));
        for (int c = 1; c < bt->chains; ++c) BPM_CK(cudaStreamWaitEvent(bt->chain_stream[c - 1], bt->chain_ev[0], 0));
        for (int c = 0; c < bt->chains; ++c) {
            cudaStream_t sc = c ? bt->chain_stream[c - 1] : s;
            // a chunk of the one group, one group of a multi-mesh batch, or several groups (one
            // stage launch per occupancy class, as for the whole batch)
            const std::vector<int>& cg = bt->chain_groups[c];
            StageLaunches L;
            if (cg.size() > 1) BPM_TRY(build_stage_launches(bt, &L, &cg));
            const StepArgs& one = cg.empty() ? bt->chain_args[c] : bt->groups[cg[0]].args;
            for (int j = 0; j < bt->p.substeps; ++j) {
                for (int k = 1; k <= 2; ++k) {
                    BPM_TRY(grouped_gemm_launch(sc, bt->gg_chain[c], bt->ctx->sm_count, bt->gemm_err));
                    if (cg.size() > 1) {
                        for (size_t q = 0; q < L.launch.size(); ++q)
                            (k == 1 ? launch_stage1_groups : launch_stage2_groups)(L.launch[q], L.threads, L.smem[q],
                                                                                   j, sc);
                    } else {
                        (k == 1 ? launch_stage1 : launch_stage2)(one, j, sc);
                    }
                }
            }
        }
        for (int c = 1; c < bt->chains; ++c) {
            BPM_CK(cudaEventRecord(bt->chain_ev[c], bt->chain_stream[c - 1]));
            BPM_CK(cudaStreamWaitEvent(s, bt->chain_ev[c], 0));
        }
    } else if (tensor_core_precision(bt)) {
        // one grouped GEMM launch and one stage launch per class per Heun stage
        StageLaunches L;
        if (bt->groups.size() > 1) BPM_TRY(build_stage_launches(bt, &L));
        for (int j = 0; j < bt->p.substeps; ++j) {
            BPM_TRY(run_demag_all(bt, s));
            launch_stage_all(bt, L, 1, j, s);
            BPM_TRY(run_demag_all(bt, s));
            launch_stage_all(bt, L, 2, j, s);
        }
    } else if (bt->groups.size() == 1) {
        BPM_TRY(enqueue_group_interval(bt, bt->groups[0], s));
    } else {
        const int ns = (int)bt->side.size();
        BPM_CK(cudaEventRecord(bt->ev[0], s));
        for (int k = 0; k < ns; ++k) BPM_CK(cudaStreamWaitEvent(bt->side[k], bt->ev[0], 0));
        for (size_t gi = 0; gi < bt->groups.size(); ++gi)
            BPM_TRY(enqueue_group_interval(bt, bt->groups[gi], bt->side[gi % ns]));
        for (int k = 0; k < ns; ++k) {
            BPM_CK(cudaEventRecord(bt->ev[1 + k], bt->side[k]));
            BPM_CK(cudaStreamWaitEvent(s, bt->ev[1 + k], 0));
        }
    }
    launch_interval_tick(bt->interval, s);
    BPM_CK(cudaGetLastError());
    return BPM_OK;
}

void free_group(Group& g) {
    void* ptrs[] = {g.d_idx, g.isl, g.m, g.k1, g.Hd, g.A32, g.Ahi, g.Alo, g.mz_prev, g.t_sw, g.crossed, g.status};
    for (void* p : ptrs) cudaFree(p);
}

void drop_graph(bpm_batch* bt) {
    if (bt->exec) {
        cudaGraphExecDestroy(bt->exec);
        bt->exec = nullptr;
    }
    if (bt->graph) {
        cudaGraphDestroy(bt->graph);
        bt->graph = nullptr;
    }
}

void free_batch(bpm_batch* bt) {
    if (!bt) return;
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    for (auto& g : bt->groups) free_group(g);
    grouped_gemm_free(&bt->gg);
    for (auto& h : bt->gg_chain) grouped_gemm_free(&h);
    for (auto st : bt->chain_stream)
        if (st) cudaStreamDestroy(st);
    for (auto e : bt->chain_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(bt->gemm_err);
    cudaFree(bt->interval);
    for (auto s : bt->side) cudaStreamDestroy(s);
    for (auto e : bt->ev) cudaEventDestroy(e);
    delete bt;
}

template <class T>
int dalloc(T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T));
    if (e != cudaSuccess) {
        set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return BPM_ERR_OOM;
    }
    e = cudaMemset(*p, 0, std::max<size_t>(1, count) * sizeof(T));
    if (e != cudaSuccess) {
        set_error("cudaMemset failed: %s", cudaGetErrorString(e));
        return BPM_ERR_CUDA;
    }
    return BPM_OK;
}

// the batch's interval graph, captured on first use
int ensure_graph(bpm_batch* bt) {
    if (bt->exec) return BPM_OK;
    cudaStream_t s = bt->ctx->stream;
    BPM_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int r = enqueue_interval(bt, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (r != BPM_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (e != cudaSuccess) {
        set_error("graph capture failed: %s", cudaGetErrorString(e));
        return BPM_ERR_CUDA;
    }
    bt->graph = g;
    BPM_CK(cudaGraphInstantiate(&bt->exec, g, 0));
    return BPM_OK;
}

// average time (ms, CUDA events) of `reps` launches of the interval graph; the state advances,
// the batch clock (the device interval counter) is put back
int time_intervals(bpm_batch* bt, int reps, double* ms) {
    BPM_TRY(ensure_graph(bt));
    cudaStream_t s = bt->ctx->stream;
    long long it0 = 0;
    BPM_CK(cudaMemcpyAsync(&it0, bt->interval, sizeof(long long), cudaMemcpyDeviceToHost, s));
    BPM_CK(cudaStreamSynchronize(s));
    cudaEvent_t e0, e1;
    BPM_CK(cudaEventCreate(&e0));
    BPM_CK(cudaEventCreate(&e1));
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; ++i) cudaGraphLaunch(bt->exec, s);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bt->interval, &it0, sizeof(long long), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("interval timing: %s", cudaGetErrorString(e));
        return BPM_ERR_CUDA;
    }
    *ms = t / reps;
    return BPM_OK;
}

}  // namespace

extern "C" {

const char* bpm_last_error(void) { return g_err; }

int bpm_substeps_for_bound(double field_bound_T, double dt_ps, double alpha, int32_t* substeps) {
    if (!substeps || !(field_bound_T >= 0) || !(dt_ps > 0) || !(alpha >= 0)) {
        set_error("bad step-rule arguments (bound >= 0, dt > 0, alpha >= 0, substeps not null)");
        return BPM_ERR_ARG;
    }
    *substeps = substeps_for_bound(field_bound_T, dt_ps, alpha);
    return BPM_OK;
}

int bpm_stable_substeps(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p, int32_t* substeps,
                        double* field_bound_T) {
    if (!substeps) {
        set_error("substeps is null");
        return BPM_ERR_ARG;
    }
    int k = 0;
    BPM_TRY(stable_substeps(ctx, isl, B, p, &k, field_bound_T));
    *substeps = k;
    return BPM_OK;
}

int bpm_context_stream(bpm_ctx* ctx, void** cuda_stream) {
    if (!ctx || !cuda_stream) {
        set_error("null argument");
        return BPM_ERR_ARG;
    }
    *cuda_stream = static_cast<void*>(ctx->stream);
    return BPM_OK;
}
const char* bpm_version(void) { return "bpmllg 0.1 (sm_103a)"; }

int bpm_create(bpm_ctx** out, int device, void* cuda_stream) {
    if (!out) {
        set_error("out is null");
        return BPM_ERR_ARG;
    }
    *out = nullptr;
    int ndev = 0;
    BPM_CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) {
        set_error("device %d not present (%d devices)", device, ndev);
        return BPM_ERR_ARG;
    }
    cudaDeviceProp prop;
    BPM_CK(cudaGetDeviceProperties(&prop, device));
    if (!(prop.major == 10 && prop.minor == 3)) {
        set_error("device %d is sm_%d%d; this library is built for sm_103a only", device, prop.major, prop.minor);
        return BPM_ERR_CUDA;
    }
    BPM_CK(cudaSetDevice(device));
    BPM_TRY(configure_step_kernels());
    bpm_ctx* c = new bpm_ctx();
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    c->l2_bytes = (size_t)prop.l2CacheSize;
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            set_error("cudaStreamCreate: %s", cudaGetErrorString(e));
            return BPM_ERR_CUDA;
        }
        c->own_stream = true;
    }
    *out = c;
    return BPM_OK;
}

void bpm_destroy(bpm_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (bpm_batch* b : live_batches(ctx)) free_batch(b);
    live_batches(ctx).clear();
    for (Mesh* m : ctx->meshes) free_mesh(m);
    for (Mlp* m : ctx->mlps) free_mlp(m);
    for (Gp* g : ctx->gps) free_gp(g);
    for (HeadMap* h : ctx->maps) {
        if (h) {
            if (h->tex) cudaDestroyTextureObject(h->tex);
            if (h->arr) cudaFreeArray(h->arr);
            cudaFree(h->B);
        }
        delete h;
    }
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int bpm_mesh_upload(bpm_ctx* ctx, const double* xyz_nm, int32_t n_nodes, const int32_t* tets, int32_t n_tets,
                    const int32_t* tet_region, const bpm_region_mat* mats, int32_t n_regions, uint32_t flags,
                    int32_t* mesh_id_out) {
    if (!ctx || !xyz_nm || !tets || !tet_region || !mats || !mesh_id_out) {
        set_error("null argument");
        return BPM_ERR_ARG;
    }
    if (n_nodes < 4 || n_nodes > kMaxNodes || n_tets < 1 || n_regions < 1) {
        set_error("mesh sizes out of range: n_nodes=%d (4..%d), n_tets=%d, n_regions=%d", n_nodes, kMaxNodes,
                  n_tets, n_regions);
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(ctx));
    Mesh* M = new Mesh();
    M->n = n_nodes;
    M->n_pad = round_up(n_nodes, kNodePad);
    M->k_pad = round_up(3 * M->n_pad, kKPad);
    M->n_tets = n_tets;
    int r = assemble_mesh(ctx, M, xyz_nm, tets, n_tets, tet_region, mats, n_regions, flags);
    if (r != BPM_OK) {
        free_mesh(M);
        return r;
    }
    ctx->meshes.push_back(M);
    *mesh_id_out = (int32_t)ctx->meshes.size() - 1;
    return BPM_OK;
}

int bpm_mesh_info_get(bpm_ctx* ctx, int32_t mesh_id, bpm_mesh_info* out) {
    Mesh* M = get_mesh(ctx, mesh_id);
    if (!M || !out) return BPM_ERR_ARG;
    *out = M->info;
    return BPM_OK;
}

int bpm_mesh_get_operator(bpm_ctx* ctx, int32_t mesh_id, int32_t which, void* dst) {
    Mesh* M = get_mesh(ctx, mesh_id);
    if (!M || !dst) return BPM_ERR_ARG;
    BPM_TRY(ensure_device(ctx));
    const int n = M->n, np = M->n_pad;
    switch (which) {
        case BPM_OP_EXCHANGE_F32: {
            float* S = static_cast<float*>(dst);
            std::memset(S, 0, sizeof(float) * (size_t)n * n);
            for (int i = 0; i < n; ++i) {
                double diag = 0;
                for (int e = M->rowptr[i]; e < M->rowptr[i + 1]; ++e) {
                    if (M->col[e] == i) continue;
                    S[(size_t)i * n + M->col[e]] = -M->exch_val[e];
                    diag += M->exch_val[e];
                }
                S[(size_t)i * n + i] = (float)diag;
            }
            return BPM_OK;
        }
        case BPM_OP_DEMAG_F64:
            if (!M->N64) {
                set_error("FP64 demag matrix not kept (upload with BPM_MESH_KEEP_F64)");
                return BPM_ERR_STATE;
            }
            BPM_CK(cudaMemcpy(dst, M->N64, sizeof(double) * 9 * (size_t)n * n, cudaMemcpyDeviceToHost));
            return BPM_OK;
        case BPM_OP_DEMAG_F32: {
            float* D = static_cast<float*>(dst);
            const int K = M->K();
            for (int c = 0; c < 3; ++c)
                for (int c2 = 0; c2 < 3; ++c2)
                    BPM_CK(cudaMemcpy2D(D + (size_t)c * n * 3 * n + (size_t)c2 * n, 3 * n * sizeof(float),
                                        M->N32 + (size_t)c * np * K + (size_t)c2 * np, K * sizeof(float),
                                        n * sizeof(float), n, cudaMemcpyDeviceToHost));
            return BPM_OK;
        }
        case BPM_OP_VOLUMES_F64:
            std::memcpy(dst, M->V.data(), sizeof(double) * n);
            return BPM_OK;
        case BPM_OP_NODAL_MS_F64:
            std::memcpy(dst, M->Ms.data(), sizeof(double) * n);
            return BPM_OK;
        case BPM_OP_NODAL_KU_F64:
            std::memcpy(dst, M->Ku.data(), sizeof(double) * n);
            return BPM_OK;
        default:
            set_error("unknown operator %d", which);
            return BPM_ERR_ARG;
    }
}

int bpm_mesh_release(bpm_ctx* ctx, int32_t mesh_id) {
    Mesh* M = get_mesh(ctx, mesh_id);
    if (!M) return BPM_ERR_ARG;
    for (const bpm_batch* b : live_batches(ctx))
        for (const auto& g : b->groups)
            if (g.mesh == M) {
                set_error("mesh %d is used by a live batch", mesh_id);
                return BPM_ERR_STATE;
            }
    BPM_TRY(ensure_device(ctx));
    BPM_CK(cudaStreamSynchronize(ctx->stream));   // work queued on the mesh's buffers finishes first
    free_mesh(M);
    ctx->meshes[mesh_id] = nullptr;
    return BPM_OK;
}

int bpm_headmap_release(bpm_ctx* ctx, int32_t map_id) {
    if (!ctx || map_id < 0 || map_id >= (int)ctx->maps.size() || !ctx->maps[map_id]) {
        set_error("unknown head map id %d", map_id);
        return BPM_ERR_ARG;
    }
    HeadMap* H = ctx->maps[map_id];
    for (const bpm_batch* b : live_batches(ctx))
        if (b->map == H) {
            set_error("head map %d is used by a live batch", map_id);
            return BPM_ERR_STATE;
        }
    BPM_TRY(ensure_device(ctx));
    BPM_CK(cudaStreamSynchronize(ctx->stream));
    if (H->tex) cudaDestroyTextureObject(H->tex);
    if (H->arr) cudaFreeArray(H->arr);
    cudaFree(H->B);
    delete H;
    ctx->maps[map_id] = nullptr;
    return BPM_OK;
}

int bpm_headmap_upload(bpm_ctx* ctx, const float* B_T, int32_t nx, int32_t ny, int32_t nz, float h_nm,
                       const float origin_nm[3], int32_t* map_id_out) {
    if (!ctx || !B_T || !origin_nm || !map_id_out || nx < 2 || ny < 2 || nz < 2 || !(h_nm > 0)) {
        set_error("bad head map arguments (need nx, ny, nz >= 2, h > 0)");
        return BPM_ERR_ARG;
    }
    if ((size_t)nx * ny * nz > (size_t)1 << 26) {
        set_error("head map too large");
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(ctx));
    size_t N = (size_t)nx * ny * nz;
    std::vector<float4> v(N);
    double max_norm = 0;
    for (size_t k = 0; k < N; ++k) {
        v[k] = make_float4(B_T[3 * k], B_T[3 * k + 1], B_T[3 * k + 2], 0.f);
        const double bx = B_T[3 * k], by = B_T[3 * k + 1], bz = B_T[3 * k + 2];
        max_norm = std::max(max_norm, std::sqrt(bx * bx + by * by + bz * bz));
    }
    HeadMap* H = new HeadMap();
    H->max_norm = max_norm;
    H->nx = nx;
    H->ny = ny;
    H->nz = nz;
    H->h = h_nm;
    for (int a = 0; a < 3; ++a) H->origin[a] = origin_nm[a];
    cudaError_t e = cudaMalloc(&H->B, N * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemcpy(H->B, v.data(), N * sizeof(float4), cudaMemcpyHostToDevice);
    cudaChannelFormatDesc cd = cudaCreateChannelDesc<float4>();
    cudaExtent ext = make_cudaExtent(nx, ny, nz);
    if (e == cudaSuccess) e = cudaMalloc3DArray(&H->arr, &cd, ext);
    if (e == cudaSuccess) {
        cudaMemcpy3DParms cp = {};
        cp.srcPtr = make_cudaPitchedPtr(v.data(), nx * sizeof(float4), nx, ny);
        cp.dstArray = H->arr;
        cp.extent = ext;
        cp.kind = cudaMemcpyHostToDevice;
        e = cudaMemcpy3D(&cp);
    }
    if (e == cudaSuccess) {
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = H->arr;
        cudaTextureDesc td = {};
        td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&H->tex, &rd, &td, nullptr);
    }
    if (e != cudaSuccess) {
        if (H->arr) cudaFreeArray(H->arr);
        cudaFree(H->B);
        delete H;
        set_error("head map upload: %s", cudaGetErrorString(e));
        return BPM_ERR_CUDA;
    }
    ctx->maps.push_back(H);
    *map_id_out = (int32_t)ctx->maps.size() - 1;
    return BPM_OK;
}

int bpm_batch_create(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p, bpm_batch** out) {
    if (!ctx || !isl || !p || !out || B < 1) {
        set_error("bad batch arguments");
        return BPM_ERR_ARG;
    }
    *out = nullptr;
    if (p->substeps < 0 || !(p->dt_ps > 0) || p->precision < 0 || p->precision > 3) {
        set_error("bad run parameters (substeps >= 0, dt > 0, precision 0..3)");
        return BPM_ERR_ARG;
    }
    int k_steps = 0;
    BPM_TRY(run_substeps(ctx, isl, B, p, &k_steps));
    HeadMap* H = nullptr;
    if (p->map_id >= 0) {
        if (p->map_id >= (int)ctx->maps.size() || !ctx->maps[p->map_id]) {
            set_error("unknown head map id %d", p->map_id);
            return BPM_ERR_ARG;
        }
        H = ctx->maps[p->map_id];
    }
    // group the islands by mesh, in order of first appearance
    std::vector<int> mesh_of_group;
    std::vector<std::vector<int>> members;
    for (int b = 0; b < B; ++b) {
        const bpm_island& I = isl[b];
        if (!get_mesh(ctx, I.mesh_id)) return BPM_ERR_ARG;
        if (!(I.Ms_scale > 0) || !(I.Ku_scale >= 0)) {
            set_error("island %d: Ms_scale must be > 0 and Ku_scale >= 0", b);
            return BPM_ERR_ARG;
        }
        size_t gi = 0;
        while (gi < mesh_of_group.size() && mesh_of_group[gi] != I.mesh_id) ++gi;
        if (gi == mesh_of_group.size()) {
            mesh_of_group.push_back(I.mesh_id);
            members.emplace_back();
        }
        members[gi].push_back(b);
    }
    BPM_TRY(ensure_device(ctx));
    bpm_batch* bt = new bpm_batch();
    bt->ctx = ctx;
    bt->map = H;
    bt->B = B;
    bt->p = *p;
    bt->p.substeps = k_steps;
    bt->t0 = p->t0_ps;
    int r = BPM_OK;
    auto chk = [&](int rr) {
        if (r == BPM_OK) r = rr;
    };
    chk(dalloc(&bt->gemm_err, 4));
    chk(dalloc(&bt->interval, 1));
    bt->groups.resize(mesh_of_group.size());
    for (size_t gi = 0; gi < bt->groups.size() && r == BPM_OK; ++gi) {
        Group& g = bt->groups[gi];
        Mesh* M = ctx->meshes[mesh_of_group[gi]];
        g.mesh = M;
        g.user_idx = members[gi];
        g.B = (int)g.user_idx.size();
        g.Bp = round_up(g.B, kIslandPad);
        bt->n_max = std::max(bt->n_max, M->n);
        const size_t S = (size_t)g.Bp * M->K();
        chk(dalloc(&g.d_idx, g.B));
        chk(dalloc(&g.isl, 3 * (size_t)g.B));
        chk(dalloc(&g.m, S));
        chk(dalloc(&g.k1, S));
        chk(dalloc(&g.Hd, S));
        if (p->precision == BPM_PREC_FP32) {
            chk(dalloc(&g.A32, S));
        } else {
            chk(dalloc(&g.Ahi, S));
            chk(dalloc(&g.Alo, S));
        }
        chk(dalloc(&g.mz_prev, g.B));
        chk(dalloc(&g.t_sw, g.B));
        chk(dalloc(&g.crossed, g.B));
        chk(dalloc(&g.status, g.B));
        if (r != BPM_OK) break;
        std::vector<float4> ip(3 * (size_t)g.B);
        for (int k = 0; k < g.B; ++k) {
            const bpm_island& I = isl[g.user_idx[k]];
            ip[3 * k] = make_float4(1.f / I.Ms_scale, I.Ku_scale / I.Ms_scale, I.Ms_scale, 0.f);
            ip[3 * k + 1] = make_float4(I.u[0], I.u[1], I.u[2], I.pos_nm[0]);
            ip[3 * k + 2] = make_float4(I.pos_nm[1], I.Hext_T[0], I.Hext_T[1], I.Hext_T[2]);
        }
        cudaError_t e = cudaMemcpy(g.isl, ip.data(), ip.size() * sizeof(float4), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(g.d_idx, g.user_idx.data(), g.B * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            set_error("island upload: %s", cudaGetErrorString(e));
            r = BPM_ERR_CUDA;
            break;
        }
        StepArgs& a = g.args;
        a.B = g.B;
        a.n = M->n;
        a.n_pad = M->n_pad;
        a.kp = M->k_pad;
        a.node_pos = M->node_pos;
        a.node_mat = M->node_mat;
        a.sell_off = M->sell_off;
        a.sell_ent = M->sell_ent;
        a.sell_il = M->sell_il;
        a.isl = g.isl;
        a.map = H ? H->B : nullptr;
        a.tex = H ? H->tex : 0;
        a.mx = H ? H->nx : 2;
        a.my = H ? H->ny : 2;
        a.mz = H ? H->nz : 2;
        a.mh = H ? H->h : 1.f;
        a.mox = H ? H->origin[0] : 0.f;
        a.moy = H ? H->origin[1] : 0.f;
        a.moz = H ? H->origin[2] : 0.f;
        a.m = g.m;
        a.k1 = g.k1;
        a.Hd = g.Hd;
        a.A32 = g.A32;
        a.Ahi = g.Ahi;
        a.Alo = g.Alo;
        a.prec = p->precision;
        a.mz_prev = g.mz_prev;
        a.t_sw = g.t_sw;
        a.crossed = g.crossed;
        a.status = g.status;
        a.interval = bt->interval;
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
        a.threads = 256;
        a.ipb = 2;
    }
    if (r == BPM_OK && bt->groups.size() > 1) {
        const int ns = (int)std::min<size_t>(4, bt->groups.size());
        bt->side.resize(ns, nullptr);
        bt->ev.resize(ns + 1, nullptr);
        for (auto& st : bt->side)
            if (r == BPM_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) r = BPM_ERR_CUDA;
        for (auto& e : bt->ev)
            if (r == BPM_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) r = BPM_ERR_CUDA;
        if (r != BPM_OK) set_error("stream/event creation failed");
    }
    if (r == BPM_OK && tensor_core_precision(bt)) r = setup_grouped_gemm(bt);
    // two chains by default for a one-mesh batch; a multi-mesh batch starts as one chain (dealing
    // its groups to chains measured slower on the uneven batch: more stage launches per interval)
    bt->streams = bt->groups.size() == 1 ? 2 : 1;
    if (r == BPM_OK) r = setup_chains(bt);
    if (r != BPM_OK) {
        free_batch(bt);
        return r;
    }
    live_batches(ctx).push_back(bt);
    r = bpm_batch_set_state(bt, nullptr, 0, p->t0_ps, 0);
    if (r != BPM_OK) {
        bpm_batch_destroy(bt);
        return r;
    }
    *out = bt;
    return BPM_OK;
}

namespace {
__global__ void k_fill_plus_z(int n, int n_pad, float* m) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int b = blockIdx.y;
    if (i >= n) return;
    size_t base = (size_t)b * 3 * n_pad;
    m[base + i] = 0.f;
    m[base + n_pad + i] = 0.f;
    m[base + 2 * n_pad + i] = 1.f;
}
// user layout [B][3][ld] <-> group layout [Bg][3][n_pad], rows mapped through idx
__global__ void k_gather_state(int n, int n_pad, int ld, const int* __restrict__ idx, const float* __restrict__ user,
                               float* __restrict__ m) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y, b = row / 3, c = row % 3;
    if (i >= n) return;
    m[(size_t)row * n_pad + i] = user[((size_t)idx[b] * 3 + c) * ld + i];
}
__global__ void k_scatter_state(int n, int n_pad, int ld, const int* __restrict__ idx, const float* __restrict__ m,
                                float* __restrict__ user) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y, b = row / 3, c = row % 3;
    if (i >= n) return;
    user[((size_t)idx[b] * 3 + c) * ld + i] = m[(size_t)row * n_pad + i];
}
__global__ void k_scatter_flags(int Bg, const int* __restrict__ idx, const float* mz_prev, const float* t_sw,
                                const int* status, uint8_t* switched, float* tsw_out, int* status_out, float* mz_out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Bg) return;
    int b = idx[k];
    if (switched) switched[b] = mz_prev[k] <= 0.f ? 1 : 0;
    if (tsw_out) tsw_out[b] = t_sw[k];
    if (status_out) status_out[b] = status[k];
    if (mz_out) mz_out[b] = mz_prev[k];
}
}  // namespace

int bpm_batch_set_state(bpm_batch* bt, const float* m, int32_t ld, double t0_ps, int on_device) {
    if (!bt) {
        set_error("null batch");
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(bt->ctx));
    cudaStream_t s = bt->ctx->stream;
    if (m && ld < bt->n_max) {
        set_error("ld %d < largest n_nodes %d", ld, bt->n_max);
        return BPM_ERR_ARG;
    }
    float* src = const_cast<float*>(m);
    if (m && !on_device) {
        BPM_CK(cudaMallocAsync(&src, sizeof(float) * 3 * (size_t)bt->B * ld, s));
        BPM_CK(cudaMemcpyAsync(src, m, sizeof(float) * 3 * (size_t)bt->B * ld, cudaMemcpyHostToDevice, s));
    }
    for (auto& g : bt->groups) {
        const int n = g.mesh->n, np = g.mesh->n_pad;
        if (m)
            k_gather_state<<<dim3((n + 255) / 256, 3 * g.B), 256, 0, s>>>(n, np, ld, g.d_idx, src, g.m);
        else
            k_fill_plus_z<<<dim3((n + 255) / 256, g.B), 256, 0, s>>>(n, np, g.m);
    }
    if (m && !on_device) cudaFreeAsync(src, s);
    BPM_CK(cudaMemsetAsync(bt->interval, 0, sizeof(long long), s));
    bt->t0 = t0_ps;
    bt->intervals_done = 0;
    for (auto& g : bt->groups) g.args.t0 = t0_ps;
    // the interval graph bakes t0 into its kernel arguments: drop it
    drop_graph(bt);
    for (auto& g : bt->groups) launch_init(g.args, s);
    BPM_CK(cudaGetLastError());
    if (!on_device) BPM_CK(cudaStreamSynchronize(s));
    return BPM_OK;
}

int bpm_batch_advance(bpm_batch* bt, int32_t n_intervals) {
    if (!bt || n_intervals < 0) {
        set_error("bad advance arguments");
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(bt->ctx));
    cudaStream_t s = bt->ctx->stream;
    if (n_intervals > 0) BPM_TRY(ensure_graph(bt));
    for (int i = 0; i < n_intervals; ++i) BPM_CK(cudaGraphLaunch(bt->exec, s));
    bt->intervals_done += n_intervals;
    return BPM_OK;
}

int bpm_batch_graph_kernels(bpm_batch* bt, int32_t* n_kernels) {
    if (!bt || !n_kernels) {
        set_error("null argument");
        return BPM_ERR_ARG;
    }
    if (!bt->graph) {
        set_error("no interval graph yet: advance the batch first");
        return BPM_ERR_STATE;
    }
    size_t n = 0;
    BPM_CK(cudaGraphGetNodes(bt->graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    BPM_CK(cudaGraphGetNodes(bt->graph, nodes.data(), &n));
    int k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        BPM_CK(cudaGraphNodeGetType(nd, &t));
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    *n_kernels = k;
    return BPM_OK;
}

int bpm_batch_read(bpm_batch* bt, float* m, int32_t ld, uint8_t* switched, float* t_sw_ps, int32_t* status, float* mz,
                   int on_device) {
    if (!bt) {
        set_error("null batch");
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(bt->ctx));
    cudaStream_t s = bt->ctx->stream;
    const int B = bt->B;
    if (m && ld < bt->n_max) {
        set_error("ld %d < largest n_nodes %d", ld, bt->n_max);
        return BPM_ERR_ARG;
    }
    // device staging of the outputs in the caller's island order
    float *dm = on_device ? m : nullptr, *dtsw = on_device ? t_sw_ps : nullptr, *dmz = on_device ? mz : nullptr;
    uint8_t* dsw = on_device ? switched : nullptr;
    int* dst = on_device ? status : nullptr;
    if (!on_device) {
        if (m) {
            BPM_CK(cudaMallocAsync(&dm, sizeof(float) * 3 * (size_t)B * ld, s));
            BPM_CK(cudaMemsetAsync(dm, 0, sizeof(float) * 3 * (size_t)B * ld, s));
        }
        BPM_CK(cudaMallocAsync(&dtsw, sizeof(float) * B, s));
        BPM_CK(cudaMallocAsync(&dmz, sizeof(float) * B, s));
        BPM_CK(cudaMallocAsync(&dsw, B, s));
        BPM_CK(cudaMallocAsync(&dst, sizeof(int) * B, s));
    }
    for (auto& g : bt->groups) {
        const int n = g.mesh->n, np = g.mesh->n_pad;
        if (dm) k_scatter_state<<<dim3((n + 255) / 256, 3 * g.B), 256, 0, s>>>(n, np, ld, g.d_idx, g.m, dm);
        k_scatter_flags<<<(g.B + 255) / 256, 256, 0, s>>>(g.B, g.d_idx, g.mz_prev, g.t_sw, g.status, dsw, dtsw, dst,
                                                        dmz);
    }
    BPM_CK(cudaGetLastError());
    if (on_device) return BPM_OK;
    int gerr = 0;
    BPM_CK(cudaMemcpyAsync(&gerr, bt->gemm_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (m) BPM_CK(cudaMemcpyAsync(m, dm, sizeof(float) * 3 * (size_t)B * ld, cudaMemcpyDeviceToHost, s));
    std::vector<float> tsw(B), mzv(B);
    std::vector<int> stv(B);
    std::vector<uint8_t> swv(B);
    BPM_CK(cudaMemcpyAsync(tsw.data(), dtsw, sizeof(float) * B, cudaMemcpyDeviceToHost, s));
    BPM_CK(cudaMemcpyAsync(mzv.data(), dmz, sizeof(float) * B, cudaMemcpyDeviceToHost, s));
    BPM_CK(cudaMemcpyAsync(swv.data(), dsw, B, cudaMemcpyDeviceToHost, s));
    BPM_CK(cudaMemcpyAsync(stv.data(), dst, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
    if (dm) cudaFreeAsync(dm, s);
    cudaFreeAsync(dtsw, s);
    cudaFreeAsync(dmz, s);
    cudaFreeAsync(dsw, s);
    cudaFreeAsync(dst, s);
    BPM_CK(cudaStreamSynchronize(s));
    if (gerr) {
        set_error("a bounded wait in the tensor-core demag GEMM gave up (code %d); results are invalid", gerr);
        return BPM_ERR_TIMEOUT;
    }
    for (int b = 0; b < B; ++b) {
        if (switched) switched[b] = swv[b];
        if (t_sw_ps) t_sw_ps[b] = tsw[b];
        if (status) status[b] = stv[b];
        if (mz) mz[b] = mzv[b];
    }
    return BPM_OK;
}

int bpm_batch_energy(bpm_batch* bt, double* E_J, float* max_torque_T) {
    if (!bt || !E_J) {
        set_error("bad energy arguments");
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(bt->ctx));
    cudaStream_t s = bt->ctx->stream;
    const double t = bt->t0 + bt->intervals_done * bt->p.dt_ps;
    int r = BPM_OK;
    if (bt->p.term_mask & BPM_TERM_DEMAG) r = run_demag_all(bt, s);   // B_d of the current state
    for (auto& g : bt->groups) {
        if (r != BPM_OK) break;
        double* dE = nullptr;
        float* dT = nullptr;
        cudaError_t e = cudaMallocAsync(&dE, g.B * sizeof(double), s);
        if (e == cudaSuccess) e = cudaMallocAsync(&dT, g.B * sizeof(float), s);
        if (e != cudaSuccess) {
            set_error("energy scratch: %s", cudaGetErrorString(e));
            r = BPM_ERR_OOM;
        } else {
            launch_energy(g.args, t, g.mesh->info.volume_nm3 * 1e-21, dE, dT, s);
            std::vector<double> hE(g.B);
            std::vector<float> hT(g.B);
            e = cudaMemcpyAsync(hE.data(), dE, g.B * sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hT.data(), dT, g.B * sizeof(float), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                set_error("energy: %s", cudaGetErrorString(e));
                r = BPM_ERR_CUDA;
            } else {
                for (int k = 0; k < g.B; ++k) {
                    E_J[g.user_idx[k]] = hE[k];
                    if (max_torque_T) max_torque_T[g.user_idx[k]] = hT[k];
                }
            }
        }
        if (dE) cudaFreeAsync(dE, s);
        if (dT) cudaFreeAsync(dT, s);
    }
    if (r == BPM_OK) {
        int herr = 0;
        BPM_CK(cudaMemcpy(&herr, bt->gemm_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr) {
            set_error("tensor-core GEMM wait timed out (code %d)", herr);
            r = BPM_ERR_TIMEOUT;
        }
    }
    return r;
}

int bpm_batch_field(bpm_batch* bt, double t_ps, uint32_t term_mask, float* B_out, int32_t ld, int on_device) {
    if (!bt || !B_out || ld < bt->n_max) {
        set_error("bad field arguments");
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(bt->ctx));
    cudaStream_t s = bt->ctx->stream;
    const size_t user_bytes = sizeof(float) * 3 * (size_t)bt->B * ld;
    float* dout = B_out;
    if (!on_device) {
        BPM_CK(cudaMallocAsync(&dout, user_bytes, s));
        BPM_CK(cudaMemsetAsync(dout, 0, user_bytes, s));
    }
    int r = BPM_OK;
    if (term_mask & BPM_TERM_DEMAG) r = run_demag_all(bt, s);
    for (auto& g : bt->groups) {
        if (r != BPM_OK) break;
        const int n = g.mesh->n, np = g.mesh->n_pad;
        float* tmp = nullptr;
        cudaError_t e = cudaMallocAsync(&tmp, (size_t)g.Bp * 3 * np * sizeof(float), s);
        if (e != cudaSuccess) {
            set_error("field scratch: %s", cudaGetErrorString(e));
            r = BPM_ERR_OOM;
            break;
        }
        if (r == BPM_OK) {
            launch_field(g.args, t_ps, term_mask, tmp, s);
            k_scatter_state<<<dim3((n + 255) / 256, 3 * g.B), 256, 0, s>>>(n, np, ld, g.d_idx, tmp, dout);
        }
        cudaFreeAsync(tmp, s);
        if (r != BPM_OK) break;
    }
    if (r == BPM_OK && !on_device) {
        cudaError_t e = cudaMemcpyAsync(B_out, dout, user_bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
            set_error("field copy: %s", cudaGetErrorString(e));
            r = BPM_ERR_CUDA;
        }
    }
    if (!on_device) cudaFreeAsync(dout, s);
    if (r != BPM_OK) return r;
    if (!on_device) BPM_CK(cudaStreamSynchronize(s));
    return BPM_OK;
}

int bpm_batch_kernel_times(bpm_batch* bt, int32_t reps, double* gemm_ms, double* stage1_ms, double* stage2_ms) {
    if (!bt || reps < 1) {
        set_error("bad kernel timing arguments");
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(bt->ctx));
    cudaStream_t s = bt->ctx->stream;
    cudaEvent_t ev[5];
    for (auto& e : ev) BPM_CK(cudaEventCreate(&e));
    double acc[3] = {0, 0, 0};
    StageLaunches L;
    int r = bt->groups.size() > 1 && tensor_core_precision(bt) ? build_stage_launches(bt, &L) : BPM_OK;
    auto stage = [&](int k, int j) {
        if (tensor_core_precision(bt)) {
            launch_stage_all(bt, L, k, j, s);
            return;
        }
        for (auto& g : bt->groups) (k == 1 ? launch_stage1 : launch_stage2)(g.args, j, s);
    };
    for (int q = 0; q < reps && r == BPM_OK; ++q) {
        int j = q % bt->p.substeps;
        cudaEventRecord(ev[0], s);
        r = run_demag_all(bt, s);
        cudaEventRecord(ev[1], s);
        stage(1, j);
        cudaEventRecord(ev[2], s);
        if (r == BPM_OK) r = run_demag_all(bt, s);
        cudaEventRecord(ev[3], s);
        stage(2, j);
        cudaEventRecord(ev[4], s);
        cudaError_t e = cudaEventSynchronize(ev[4]);
        if (e != cudaSuccess) {
            set_error("kernel timing: %s", cudaGetErrorString(e));
            r = BPM_ERR_CUDA;
            break;
        }
        float t[4];
        for (int k = 0; k < 4; ++k) cudaEventElapsedTime(&t[k], ev[k], ev[k + 1]);
        acc[0] += 0.5 * (t[0] + t[2]);
        acc[1] += t[1];
        acc[2] += t[3];
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (r != BPM_OK) return r;
    if (gemm_ms) *gemm_ms = acc[0] / reps;
    if (stage1_ms) *stage1_ms = acc[1] / reps;
    if (stage2_ms) *stage2_ms = acc[2] / reps;
    return BPM_OK;
}

int bpm_batch_set_tuning(bpm_batch* bt, const bpm_tuning* t) {
    if (!bt || !t || (t->gemm_tile_n != 128 && t->gemm_tile_n != 256) ||
        (t->stage_threads != 128 && t->stage_threads != 256 && t->stage_threads != 512) ||
        (t->gemm_raster != BPM_RASTER_AUTO && t->gemm_raster != BPM_RASTER_M && t->gemm_raster != BPM_RASTER_N) ||
        t->stage_islands < 0 || t->stage_islands > 2 || (t->stage_islands == 2 && t->stage_threads != 256) ||
        (t->gemm_k_block != 0 && t->gemm_k_block != 32 && t->gemm_k_block != 64) || t->gemm_pair < 0 ||
        t->gemm_pair > 1 || (t->gemm_pair == 1 && t->gemm_tile_n != 256) || t->streams < 0 ||
        t->streams > kMaxChains) {
        set_error("bad tuning (gemm_tile_n 128|256, stage_threads 128|256|512, gemm_raster 0|1|2, "
                  "stage_islands 0|1|2 with 2 only at 256 threads, gemm_k_block 0|32|64, gemm_pair 0|1 with 1 "
                  "only at gemm_tile_n 256, streams 0 .. 4)");
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(bt->ctx));
    BPM_CK(cudaStreamSynchronize(bt->ctx->stream));
    bt->tile_n = t->gemm_tile_n;
    bt->raster = t->gemm_raster;
    bt->k_block = t->gemm_k_block == 64 ? 64 : 32;
    bt->pair = t->gemm_pair;
    bt->streams = std::max(1, (int)t->streams);
    for (auto& g : bt->groups) {
        g.args.threads = t->stage_threads;
        g.args.ipb = t->stage_islands == 2 ? 2 : 1;
    }
    drop_graph(bt);   // the graph holds the old launch configurations
    if (tensor_core_precision(bt)) BPM_TRY(setup_grouped_gemm(bt));
    BPM_TRY(setup_chains(bt));
    for (auto& h : bt->gg_chain) h.wait_ns = bt->gg.wait_ns;
    return BPM_OK;
}

int bpm_batch_autotune(bpm_batch* bt, int32_t reps, bpm_tuning* chosen) {
    if (!bt || reps < 1) {
        set_error("bad autotune arguments");
        return BPM_ERR_ARG;
    }
    // (tile width, CTA pair): one-SM tiles 256 or 128 wide, or 256 x 256 tiles on CTA pairs
    const int tiles[3] = {256, 128, 256};
    const int pairs[3] = {0, 0, 1};
    const int rasters[3] = {BPM_RASTER_AUTO, BPM_RASTER_M, BPM_RASTER_N};
    const int kblocks[2] = {64, 32};
    const int threads[3] = {256, 128, 512};
    const bool tc = tensor_core_precision(bt);
    double best_g = 1e300, best_s = 1e300;
    int bt_n = 256, bt_r = BPM_RASTER_AUTO, bt_t = 256, bt_k = 64, bt_p = 0;
    // the GEMM candidates at the default stage CTA size, then the stage CTA sizes at the best GEMM
    for (int ti = 0; ti < (tc ? 3 : 1); ++ti)
        for (int ri = 0; ri < (tc ? 3 : 1); ++ri)
            for (int ki = 0; ki < (tc ? 2 : 1); ++ki) {
                bpm_tuning t{tiles[ti], 256, rasters[ri], 1, kblocks[ki], pairs[ti], 1, 0, 0};
                BPM_TRY(bpm_batch_set_tuning(bt, &t));
                double g = 0, s1 = 0, s2 = 0;
                BPM_TRY(bpm_batch_kernel_times(bt, 1, &g, &s1, &s2));   // warm-up
                BPM_TRY(bpm_batch_kernel_times(bt, reps, &g, &s1, &s2));
                if (g < best_g) {
                    best_g = g;
                    bt_n = tiles[ti];
                    bt_r = rasters[ri];
                    bt_k = kblocks[ki];
                    bt_p = pairs[ti];
                }
            }
    // stage candidates: one island per CTA at each CTA size, two islands per 256-thread CTA
    int bt_i = 1;
    for (int hi = 0; hi < 4; ++hi) {
        const int nt = hi < 3 ? threads[hi] : 256, ipb = hi < 3 ? 1 : 2;
        bpm_tuning t{bt_n, nt, bt_r, ipb, bt_k, bt_p, 1, 0, 0};
        BPM_TRY(bpm_batch_set_tuning(bt, &t));
        double g = 0, s1 = 0, s2 = 0;
        BPM_TRY(bpm_batch_kernel_times(bt, 1, &g, &s1, &s2));
        BPM_TRY(bpm_batch_kernel_times(bt, reps, &g, &s1, &s2));
        if (s1 + s2 < best_s) {
            best_s = s1 + s2;
            bt_t = nt;
            bt_i = ipb;
        }
    }
    // one chain or several: whole intervals of the interval graph, where several chains apply
    int bt_s = 1;
    if (tensor_core_precision(bt) && (bt->groups.size() > 1 || bt->groups[0].B > kIslandPad)) {
        double best_i = 1e300;
        for (int ns = 1; ns <= kMaxChains; ++ns) {
            bpm_tuning t{bt_n, bt_t, bt_r, bt_i, bt_k, bt_p, ns, 0, 0};
            BPM_TRY(bpm_batch_set_tuning(bt, &t));
            double ms = 0;
            BPM_TRY(time_intervals(bt, 1, &ms));   // capture and warm-up
            BPM_TRY(time_intervals(bt, reps, &ms));
            if (ms < best_i) {
                best_i = ms;
                bt_s = ns;
            }
        }
    }
    bpm_tuning t{bt_n, bt_t, bt_r, bt_i, bt_k, bt_p, bt_s, best_g, best_s};
    BPM_TRY(bpm_batch_set_tuning(bt, &t));
    if (chosen) *chosen = t;
    return BPM_OK;
}

int bpm_debug_set_gemm_error(bpm_batch* bt, int32_t code) {
    if (!bt) {
        set_error("null batch");
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(bt->ctx));
    BPM_CK(cudaMemcpyAsync(bt->gemm_err, &code, sizeof(int32_t), cudaMemcpyHostToDevice, bt->ctx->stream));
    BPM_CK(cudaStreamSynchronize(bt->ctx->stream));
    return BPM_OK;
}

int bpm_debug_set_gemm_wait(bpm_batch* bt, double wait_ns) {
    if (!bt || !(wait_ns >= 0) || wait_ns > 1e10) {
        set_error("bad wait limit (0 for the default, else up to 1e10 ns)");
        return BPM_ERR_ARG;
    }
    BPM_TRY(ensure_device(bt->ctx));
    BPM_CK(cudaStreamSynchronize(bt->ctx->stream));
    bt->gg.wait_ns = (unsigned long long)wait_ns;
    for (auto& h : bt->gg_chain) h.wait_ns = bt->gg.wait_ns;
    drop_graph(bt);   // the graph holds the old kernel arguments
    return BPM_OK;
}

int bpm_batch_time(bpm_batch* bt, double* t_ps) {
    if (!bt || !t_ps) {
        set_error("null argument");
        return BPM_ERR_ARG;
    }
    *t_ps = bt->t0 + bt->intervals_done * bt->p.dt_ps;
    return BPM_OK;
}

int bpm_batch_destroy(bpm_batch* bt) {
    if (!bt) return BPM_OK;
    cudaSetDevice(bt->ctx->device);
    cudaStreamSynchronize(bt->ctx->stream);
    auto& v = live_batches(bt->ctx);
    v.erase(std::remove(v.begin(), v.end(), bt), v.end());
    free_batch(bt);
    return BPM_OK;
}

int bpm_run_batch(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p, int32_t n_intervals,
                  float* m_final, int32_t ld, uint8_t* switched, float* t_sw_ps, int32_t* status) {
    bpm_batch* bt = nullptr;
    BPM_TRY(bpm_batch_create(ctx, isl, B, p, &bt));
    int r = bpm_batch_advance(bt, n_intervals);
    if (r == BPM_OK) r = bpm_batch_read(bt, m_final, ld, switched, t_sw_ps, status, nullptr, 0);
    bpm_batch_destroy(bt);
    return r;
}

int bpm_run_batch_dev(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p, int32_t n_intervals,
                      float* m_final, int32_t ld, uint8_t* switched, float* t_sw_ps, int32_t* status) {
    bpm_batch* bt = nullptr;
    BPM_TRY(bpm_batch_create(ctx, isl, B, p, &bt));
    int r = bpm_batch_advance(bt, n_intervals);
    if (r == BPM_OK) r = bpm_batch_read(bt, m_final, ld, switched, t_sw_ps, status, nullptr, 1);
    int gerr = 0;
    if (r == BPM_OK && cudaMemcpyAsync(&gerr, bt->gemm_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) !=
                           cudaSuccess) {
        set_error("reading the GEMM error flag failed");
        r = BPM_ERR_CUDA;
    }
    bpm_batch_destroy(bt);   // synchronises the stream before it frees the batch
    if (r == BPM_OK && gerr) {
        set_error("a bounded wait in the tensor-core GEMM gave up (code %d)", gerr);
        r = BPM_ERR_TIMEOUT;
    }
    return r;
}

}  // extern "C"
